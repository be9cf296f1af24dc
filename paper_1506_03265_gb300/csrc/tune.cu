// Process-wide tuning knobs (launch shapes and cut-overs between equivalent
// forms of a step).  Every knob is result-invariant.
#include <mutex>

#include "internal.cuh"

namespace cld {

namespace {

std::mutex g_tmu;
cldiam_tuning g_tuning{};  // zero = defaults

}  // namespace

cldiam_tuning tuning_defaults_filled(const cldiam_tuning& t) {
    cldiam_tuning r = t;
    if (r.pull_ratio == 0.f) r.pull_ratio = 0.3f;
    if (r.pull_ratio < 0.f) r.pull_ratio = 0.f;  // never
    if (r.dense_quotient_k == 0) r.dense_quotient_k = 4096;
    if (r.apsp_fw_density == 0) r.apsp_fw_density = 8;
    if (r.batch_fw_k == 0) r.batch_fw_k = 200;
    if (r.sssp_delta_scale == 0.f) r.sssp_delta_scale = 1.f;
    return r;
}

cldiam_status tuning_check(const cldiam_tuning& t) {
    if (!(t.pull_ratio == t.pull_ratio)) return fail(CLDIAM_ERR_INVALID_ARG, "pull_ratio is NaN");
    if (t.relax_ctas_per_sm > 64) return fail(CLDIAM_ERR_INVALID_ARG, "relax_ctas_per_sm > 64");
    if (t.dense_quotient_k > 65535) return fail(CLDIAM_ERR_INVALID_ARG, "dense_quotient_k > 65535");
    if (t.apsp_sources_per_cta != 0 && t.apsp_sources_per_cta != 1 && t.apsp_sources_per_cta != 4 &&
        t.apsp_sources_per_cta != 8)
        return fail(CLDIAM_ERR_INVALID_ARG, "apsp_sources_per_cta must be 0, 1, 4 or 8");
    if (t.batch_fw_k > 200) return fail(CLDIAM_ERR_INVALID_ARG, "batch_fw_k > 200");
    if (!(t.sssp_delta_scale == 0.f || t.sssp_delta_scale >= 1.f) || !(t.sssp_delta_scale < 1e9f))
        return fail(CLDIAM_ERR_INVALID_ARG, "sssp_delta_scale must be 0 or in [1, 1e9)");
    for (uint32_t r : t.reserved)
        if (r) return fail(CLDIAM_ERR_INVALID_ARG, "reserved tuning fields must be 0");
    return CLDIAM_OK;
}

cldiam_tuning tuning_current() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return tuning_defaults_filled(g_tuning);
}

}  // namespace cld

using namespace cld;

extern "C" {

cldiam_status cldiam_tuning_get(cldiam_tuning* out) {
    if (!out) return fail(CLDIAM_ERR_INVALID_ARG, "NULL out");
    *out = tuning_current();
    return CLDIAM_OK;
}

cldiam_status cldiam_tuning_set(const cldiam_tuning* t) {
    cldiam_tuning v{};
    if (t) {
        CLD_TRY(tuning_check(*t));
        v = *t;
    }
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tuning = v;
    return CLDIAM_OK;
}

}  // extern "C"
