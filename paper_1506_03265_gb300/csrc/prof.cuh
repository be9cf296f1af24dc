// Launch accounting and optional CUDA-event timing per kernel class.
//
// Every kernel launch of the library goes through CLD_K(class, stream, launch):
// the launch is counted and, when timing is enabled for its class, bracketed
// by CUDA events on the launching stream.  Callers attribute the algorithmic
// bytes a launch had to move with prof_add_bytes once they know them.
#pragma once

#include "common.cuh"

namespace cld {

enum KClass : int {
    K_RELAX = 0,
    K_SNAPSHOT,
    K_REBUILD,
    K_SELECT,
    K_FINALIZE,
    K_GROWABLE,
    K_RADIX_HIST,
    K_RADIX_SCATTER,
    K_SCAN,
    K_CSR,
    K_CC,
    K_QUOTIENT,
    K_FW,
    K_SSSP,
    K_REDUCE,
    K_MISC,
    K_PULL,
    K_NCLASS
};

const char* kclass_name(int c);
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);
void prof_add_bytes(int cls, double bytes);
// Resolve finished event pairs into milliseconds (call after a stream sync).
void prof_flush();

struct ProfScope {
    int cls;
    cudaStream_t s;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st) { prof_begin(cls, s); }
    ~ProfScope() { prof_end(cls, s); }
};

#define CLD_K(cls, stream, ...)                      \
    do {                                             \
        ::cld::ProfScope cld_ps_((cls), (stream));   \
        __VA_ARGS__;                                 \
    } while (0)

}  // namespace cld
