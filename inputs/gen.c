/*
 * Seeded synthetic graph generators for the CL-DIAM workloads.
 *
 * This file produces INPUTS only (edge lists with uint32 weights).  It holds
 * none of the diameter method's arithmetic and is shared by the CPU oracle and
 * the CUDA path as the single source of test and benchmark graphs.
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), keyed by the 64-bit seed and driven by
 * a counter that names (item index, stream, call), so every draw is a pure
 * function of its coordinates.  Results are independent of the thread count.
 *
 * Workload shapes follow the paper's synthetic graphs (Section 5, Table 1):
 * square meshes, R-MAT power-law graphs (Chakrabarti et al.), plus a road-like
 * mesh with deleted edges and random chords standing in for the road networks.
 * Weights are integers w = 1 + floor(r * W / 2^32), uniform in [1, W].
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

#define GEN_STREAM_WEIGHT 1u
#define GEN_STREAM_RMAT 2u
#define GEN_STREAM_DELETE 3u
#define GEN_STREAM_CHORD 4u
#define GEN_STREAM_PERM 5u
#define GEN_STREAM_MIX 6u
#define GEN_STREAM_SUBSEED 7u
#define GEN_STREAM_QUERY 8u

typedef struct { uint32_t v[4]; } gen_u4;

static inline gen_u4 gen_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    gen_u4 o = {{x0, x1, x2, x3}};
    return o;
}

static inline uint32_t gen_weight(uint64_t seed, uint64_t e, uint32_t W)
{
    gen_u4 r = gen_philox(seed, (uint32_t)e, (uint32_t)(e >> 32), GEN_STREAM_WEIGHT, 0);
    return 1u + (uint32_t)(((uint64_t)r.v[0] * W) >> 32);
}

/* Raw Philox block, exported so tests can check the generator's stream. */
void gen_philox4x32(uint64_t seed, const uint32_t ctr[4], uint32_t out[4])
{
    gen_u4 r = gen_philox(seed, ctr[0], ctr[1], ctr[2], ctr[3]);
    for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

/*
 * side x side 4-neighbour mesh: horizontal edges row-major, then vertical
 * edges row-major.  m = 2*side*(side-1).  Node id = row*side + col.
 */
int64_t gen_grid(uint32_t side, uint32_t W, uint64_t seed,
                 uint32_t* src, uint32_t* dst, uint32_t* w)
{
    if (side == 0) return 0;
    int64_t S = side;
    int64_t mh = S * (S - 1);
    int64_t m = 2 * mh;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t u, v;
        if (e < mh) { int64_t r = e / (S - 1), c = e % (S - 1); u = r * S + c; v = u + 1; }
        else { int64_t f = e - mh; int64_t r = f / S, c = f % S; u = r * S + c; v = u + S; }
        src[e] = (uint32_t)u; dst[e] = (uint32_t)v; w[e] = gen_weight(seed, (uint64_t)e, W);
    }
    return m;
}

/*
 * Road-like mesh: the side x side mesh above with each edge deleted
 * independently with probability p_del, plus floor(chord_frac * m_grid) chords
 * between uniform random node pairs.  Weights are drawn by generation index
 * (grid edge index e, chord j at index m_grid + j) before deletion, so a kept
 * edge's weight does not depend on which others were deleted.  Output: kept
 * grid edges in order, then the chords.  Returns the edge count; the caller
 * sizes the buffers with gen_road_mesh_max_edges().
 */
int64_t gen_road_mesh_max_edges(uint32_t side, double chord_frac)
{
    int64_t S = side;
    int64_t mg = 2 * S * (S - 1);
    return mg + (int64_t)floor(chord_frac * (double)mg);
}

int64_t gen_road_mesh(uint32_t side, double p_del, double chord_frac, uint32_t W, uint64_t seed,
                      uint32_t* src, uint32_t* dst, uint32_t* w)
{
    if (side == 0) return 0;
    int64_t S = side, n = S * S;
    int64_t mh = S * (S - 1);
    int64_t mg = 2 * mh;
    uint64_t thr = (uint64_t)floor(p_del * 4294967296.0);
    int64_t out = 0;
    /* sequential compaction keeps the output order independent of threads */
    for (int64_t e = 0; e < mg; ++e) {
        gen_u4 r = gen_philox(seed, (uint32_t)e, (uint32_t)((uint64_t)e >> 32), GEN_STREAM_DELETE, 0);
        if ((uint64_t)r.v[0] < thr) continue;
        int64_t u, v;
        if (e < mh) { int64_t rr = e / (S - 1), c = e % (S - 1); u = rr * S + c; v = u + 1; }
        else { int64_t f = e - mh; int64_t rr = f / S, c = f % S; u = rr * S + c; v = u + S; }
        src[out] = (uint32_t)u; dst[out] = (uint32_t)v; w[out] = gen_weight(seed, (uint64_t)e, W);
        ++out;
    }
    int64_t nc = (int64_t)floor(chord_frac * (double)mg);
    for (int64_t j = 0; j < nc; ++j) {
        gen_u4 r = gen_philox(seed, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), GEN_STREAM_CHORD, 0);
        src[out] = (uint32_t)(((uint64_t)r.v[0] * (uint64_t)n) >> 32);
        dst[out] = (uint32_t)(((uint64_t)r.v[1] * (uint64_t)n) >> 32);
        w[out] = gen_weight(seed, (uint64_t)(mg + j), W);
        ++out;
    }
    return out;
}

/*
 * R-MAT(scale, edge factor): m = ef * 2^scale directed draws, each choosing one
 * quadrant per level with probabilities (a, b, c, 1-a-b-c), most significant
 * bit first (Chakrabarti, Zhan, Faloutsos, SDM'04).  One Philox word per
 * level.  With permute != 0 the vertex labels are relabelled by a seeded
 * Fisher-Yates permutation (as Graph500 does) so ids carry no locality.
 * Self-loops and duplicates are left in: the CSR builder removes them.
 */
int64_t gen_rmat(uint32_t scale, uint32_t ef, uint32_t W, uint64_t seed,
                 double a, double b, double c, int permute,
                 uint32_t* src, uint32_t* dst, uint32_t* w, uint32_t* perm_scratch)
{
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)ef * n;
    uint64_t ta = (uint64_t)floor(a * 4294967296.0);
    uint64_t tab = (uint64_t)floor((a + b) * 4294967296.0);
    uint64_t tabc = (uint64_t)floor((a + b + c) * 4294967296.0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        gen_u4 r = {{0, 0, 0, 0}};
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            if ((lvl & 3u) == 0)
                r = gen_philox(seed, (uint32_t)e, (uint32_t)((uint64_t)e >> 32), GEN_STREAM_RMAT, lvl >> 2);
            uint64_t x = r.v[lvl & 3u];
            uint32_t sb, db;
            if (x < ta) { sb = 0; db = 0; }
            else if (x < tab) { sb = 0; db = 1; }
            else if (x < tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            u = (u << 1) | sb;
            v = (v << 1) | db;
        }
        src[e] = u; dst[e] = v; w[e] = gen_weight(seed, (uint64_t)e, W);
    }
    if (permute && perm_scratch) {
        for (int64_t i = 0; i < n; ++i) perm_scratch[i] = (uint32_t)i;
        for (int64_t i = n - 1; i > 0; --i) {
            gen_u4 r = gen_philox(seed, (uint32_t)i, 0, GEN_STREAM_PERM, 0);
            int64_t j = (int64_t)(((uint64_t)r.v[0] * (uint64_t)(i + 1)) >> 32);
            uint32_t t = perm_scratch[i]; perm_scratch[i] = perm_scratch[j]; perm_scratch[j] = t;
        }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < m; ++e) { src[e] = perm_scratch[src[e]]; dst[e] = perm_scratch[dst[e]]; }
    }
    return m;
}

/*
 * Mixture used for the many-graph workloads: graph g is an R-MAT (edge factor
 * 8, scale uniform in {8..16}) with probability 1/2, else a mesh whose side is
 * round(2^U) with U uniform in [5, 9) (sides 32..512, log-uniform).  Each
 * graph gets its own 64-bit sub-seed.
 */
void gen_mix_params(uint64_t seed, uint32_t g, uint32_t* kind, uint32_t* scale, uint32_t* side,
                    uint64_t* subseed)
{
    gen_u4 r = gen_philox(seed, g, 0, GEN_STREAM_MIX, 0);
    *kind = (r.v[0] < 0x80000000u) ? 0u : 1u; /* 0 = R-MAT, 1 = mesh */
    *scale = 8u + (uint32_t)(((uint64_t)r.v[1] * 9u) >> 32);
    double u = (double)r.v[2] / 4294967296.0;
    *side = (uint32_t)llround(pow(2.0, 5.0 + 4.0 * u));
    gen_u4 s = gen_philox(seed, g, 0, GEN_STREAM_SUBSEED, 0);
    *subseed = ((uint64_t)s.v[1] << 32) | s.v[0];
}

/*
 * Query stream for the serving workload: query q arrives after an exponential
 * gap of mean 1/rate seconds; with probability p_big it asks for the large
 * graph (index n_small), else for graph floor(u * n_small) of the mixture.
 */
void gen_queries(uint64_t seed, uint32_t count, double rate, double p_big, uint32_t n_small,
                 double* arrival, uint32_t* graph)
{
    double t = 0.0;
    uint64_t tbig = (uint64_t)floor(p_big * 4294967296.0);
    for (uint32_t q = 0; q < count; ++q) {
        gen_u4 r = gen_philox(seed, q, 0, GEN_STREAM_QUERY, 0);
        double u = ((double)r.v[0] + 1.0) / 4294967297.0; /* (0,1) */
        t += -log(u) / rate;
        arrival[q] = t;
        graph[q] = ((uint64_t)r.v[1] < tbig) ? n_small : (uint32_t)(((uint64_t)r.v[2] * n_small) >> 32);
    }
}
