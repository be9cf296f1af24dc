/*
 * CL-DIAM reference oracle: a plain, sequential, obviously-correct CPU
 * restatement of the diameter-approximation method of Ceccarello,
 * Pietracaprina, Pucci and Upfal, "A Practical Parallel Algorithm for Diameter
 * Approximation of Massive Weighted Graphs" (arXiv 1506.03265).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, helper or table with the CUDA library; the two agree only through
 * the paper.  Integer arithmetic throughout (distances in uint64), so results
 * are exact.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_philox4x32_10   pinned: an independent Philox4x32-10 (Triton's, CPU interpreter)
 *   orc_build_csr       pinned: numpy unique/lexsort + scipy connected_components
 *   orc_growth_steps    pinned: brute-force enumeration of bounded walks (Section 3 step),
 *                       with frozen nodes at distance 0 or, cumulative mode, at their D
 *   orc_cluster         pinned by invariants (coverage, radius bounds, D >= true distance,
 *                       stage-count bound) and by the special cases that reduce to exact
 *                       APSP; the random trajectory itself has no printed example
 *                       ("parity unpinned" beyond these invariants)
 *   orc_cluster_opts    the same, plus: a step cap at least as long as the longest
 *                       uncapped growth changes nothing, cap 1 bounds every growth to one
 *                       step, the cumulative mode keeps every D within the final Delta and
 *                       above the true distance, and its first stage equals the default's
 *   orc_cluster2        pinned: a global-offset multi-source Dijkstra restatement of
 *                       Algorithm 2 (same draws), plus coverage / path-length invariants
 *                       and the R_CL = 0 case (all singletons)
 *   orc_quotient        pinned: independent dictionary recomputation + symmetry
 *   orc_apsp_max        pinned: scipy shortest_path
 *   orc_dijkstra        pinned: scipy dijkstra
 *   orc_delta0          pinned: numpy sum / min
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF_KEY 0xFFFFFFFFFFFFFFFFull
#define ORC_NONE 0xFFFFFFFFu
#define ORC_DELTA_MAX 0x80000000u /* Delta saturates at 2^31 */
#define ORC_MAX_STAGES 100000u
#define ORC_GAMMA 2.772588722239781 /* 4 ln 2, Algorithm 1 */

/* error codes (negative) */
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_DIVERGED (-8)

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): the counter-based generator that the
 * center-selection rule of Algorithm 1 draws from.  key = (seed lo, seed hi).
 * Round: (hi,lo) = M0*x0 and M1*x2; the four words become
 *   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)),
 * with the Weyl key bump k += (W0, W1) after each round.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(uint64_t seed, const uint32_t ctr_in[4], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    uint32_t k1 = (uint32_t)(seed >> 32);
    uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)x[0];
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)x[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y[4];
        y[0] = hi1 ^ x[1] ^ k0;
        y[1] = lo1;
        y[2] = hi0 ^ x[3] ^ k1;
        y[3] = lo0;
        memcpy(x, y, sizeof x);
        k0 += W0;
        k1 += W1;
    }
    memcpy(out, x, sizeof x);
}

static uint32_t philox_x0(uint64_t seed, uint32_t c0, uint32_t c1)
{
    uint32_t ctr[4] = {c0, c1, 0, 0}, out[4];
    orc_philox4x32_10(seed, ctr, out);
    return out[0];
}

/* ---------------------------------------------------------------------------
 * CSR construction.  Graph model of Section 2: undirected, positive integral
 * weights.  Self-loops carry no distance and are dropped; parallel edges are
 * merged keeping the minimum weight (only the lightest can lie on a shortest
 * path).  With lcc != 0 only the largest connected component is kept (the
 * diameter of a disconnected graph is taken per component, Section 2); ties
 * go to the component containing the smallest node id.  Kept nodes are
 * renumbered by increasing original id.  Rows are sorted by column.
 * ------------------------------------------------------------------------- */
typedef struct { uint32_t a, b, w; } orc_trip;

static int cmp_trip(const void* p, const void* q)
{
    const orc_trip* x = (const orc_trip*)p;
    const orc_trip* y = (const orc_trip*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

/* returns number of directed CSR entries, or < 0 on error.
 * Buffers: off_out[n+1], col_out[2m], wt_out[2m], orig_out[n]. */
int64_t orc_build_csr(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                      int lcc, uint32_t* n_out, uint64_t* off_out, uint32_t* col_out, uint32_t* wt_out,
                      uint32_t* orig_out)
{
    if (n == 0) return ORC_ERR_ARG;
    for (uint64_t e = 0; e < m; ++e)
        if (src[e] >= n || dst[e] >= n || w[e] == 0) return ORC_ERR_ARG;

    /* 1. undirected pairs (min, max), self-loops dropped */
    orc_trip* und = (orc_trip*)malloc(sizeof(orc_trip) * (m ? m : 1));
    if (!und) return ORC_ERR_OOM;
    uint64_t mu = 0;
    for (uint64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        uint32_t a = src[e] < dst[e] ? src[e] : dst[e];
        uint32_t b = src[e] < dst[e] ? dst[e] : src[e];
        und[mu].a = a; und[mu].b = b; und[mu].w = w[e];
        ++mu;
    }
    /* 2. sort by (a, b, w); keep the first (= lightest) of each pair */
    qsort(und, mu, sizeof(orc_trip), cmp_trip);
    uint64_t md = 0;
    for (uint64_t i = 0; i < mu; ++i) {
        if (md > 0 && und[md - 1].a == und[i].a && und[md - 1].b == und[i].b) continue;
        und[md++] = und[i];
    }
    /* 3. both directions, sorted by (row, col) */
    orc_trip* dir = (orc_trip*)malloc(sizeof(orc_trip) * (2 * md ? 2 * md : 1));
    if (!dir) { free(und); return ORC_ERR_OOM; }
    for (uint64_t i = 0; i < md; ++i) {
        dir[2 * i].a = und[i].a; dir[2 * i].b = und[i].b; dir[2 * i].w = und[i].w;
        dir[2 * i + 1].a = und[i].b; dir[2 * i + 1].b = und[i].a; dir[2 * i + 1].w = und[i].w;
    }
    free(und);
    uint64_t nnz = 2 * md;
    qsort(dir, nnz, sizeof(orc_trip), cmp_trip);
    uint64_t* off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!off) { free(dir); return ORC_ERR_OOM; }
    for (uint64_t i = 0; i < nnz; ++i) off[dir[i].a + 1]++;
    for (uint32_t v = 0; v < n; ++v) off[v + 1] += off[v];

    /* 4. optional largest connected component by breadth-first search */
    uint32_t* newid = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!newid) { free(dir); free(off); return ORC_ERR_OOM; }
    if (lcc) {
        uint32_t* comp = (uint32_t*)malloc(sizeof(uint32_t) * n);
        uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * n);
        if (!comp || !queue) { free(comp); free(queue); free(dir); free(off); free(newid); return ORC_ERR_OOM; }
        for (uint32_t v = 0; v < n; ++v) comp[v] = ORC_NONE;
        uint32_t best_root = 0;
        uint64_t best_size = 0;
        for (uint32_t r = 0; r < n; ++r) {
            if (comp[r] != ORC_NONE) continue;
            uint64_t head = 0, tail = 0;
            queue[tail++] = r;
            comp[r] = r;
            while (head < tail) {
                uint32_t u = queue[head++];
                for (uint64_t j = off[u]; j < off[u + 1]; ++j) {
                    uint32_t v = dir[j].b;
                    if (comp[v] == ORC_NONE) { comp[v] = r; queue[tail++] = v; }
                }
            }
            if (tail > best_size) { best_size = tail; best_root = r; } /* strict: first (smallest) root wins ties */
        }
        uint32_t next = 0;
        for (uint32_t v = 0; v < n; ++v) newid[v] = (comp[v] == best_root) ? next++ : ORC_NONE;
        free(comp);
        free(queue);
    } else {
        for (uint32_t v = 0; v < n; ++v) newid[v] = v;
    }

    /* 5. emit the kept rows, columns renumbered (renumbering is monotone, so rows stay sorted) */
    uint32_t nk = 0;
    uint64_t pos = 0;
    off_out[0] = 0;
    for (uint32_t v = 0; v < n; ++v) {
        if (newid[v] == ORC_NONE) continue;
        orig_out[nk] = v;
        for (uint64_t j = off[v]; j < off[v + 1]; ++j) {
            col_out[pos] = newid[dir[j].b];
            wt_out[pos] = dir[j].w;
            ++pos;
        }
        off_out[++nk] = pos;
    }
    *n_out = nk;
    free(dir);
    free(off);
    free(newid);
    return (int64_t)pos;
}

/* ---------------------------------------------------------------------------
 * Initial Delta.  Algorithm 1 starts from the minimum edge weight; the
 * experiments of Section 5 start from the average edge weight instead.
 * mode 0: floor(sum of weights / number of undirected edges), at least 1.
 * mode 1: minimum weight.  A graph without edges gets 1.
 * ------------------------------------------------------------------------- */
uint32_t orc_delta0(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt, int mode)
{
    uint64_t nnz = off[n];
    if (nnz == 0) return 1;
    if (mode == 1) {
        uint32_t mn = 0xFFFFFFFFu;
        for (uint64_t j = 0; j < nnz; ++j) if (wt[j] < mn) mn = wt[j];
        return mn;
    }
    /* each undirected edge appears twice; sum over the u < v copy */
    uint64_t sum = 0, cnt = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t j = off[u]; j < off[u + 1]; ++j)
            if (u < col[j]) { sum += wt[j]; ++cnt; }
    uint64_t avg = sum / cnt;
    if (avg < 1) avg = 1;
    if (avg > ORC_DELTA_MAX) avg = ORC_DELTA_MAX;
    return (uint32_t)avg;
}

/* ---------------------------------------------------------------------------
 * One Delta-growing step (Section 3), synchronous: every candidate is formed
 * from the state as it was at the start of the step (snapshot S).
 *   relaxers: unfrozen u with d_u < Delta, and every frozen u, which stands for
 *             its contracted cluster center c_u at distance 0 (Procedure
 *             Contract replaces (u,v) by (c_u,v) with weight w(u,v)); in the
 *             cumulative contract mode (Dfrozen != NULL) a frozen u relaxes
 *             with its own bound D_u instead, if D_u < Delta;
 *   for each relaxer u and edge (u,v) with v unfrozen: if d_u + w <= Delta,
 *             v takes (d_u + w, c_u) if that is lexicographically smaller than
 *             its current (d_v, c_v): smallest distance first, then smallest
 *             center index.
 * key(d, c) = d * 2^32 + c orders pairs exactly that way.  Returns the number
 * of nodes whose key decreased; *newly_covered counts those that had none.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n;
    const uint64_t* off;
    const uint32_t* col;
    const uint32_t* wt;
} orc_graph;

static uint64_t mkkey(uint64_t d, uint32_t c) { return (d << 32) | c; }

static uint64_t growing_step(const orc_graph* g, uint64_t* key, uint64_t* snap, const uint8_t* frozen,
                             const uint32_t* center, const uint64_t* Dfrozen, uint32_t delta,
                             uint64_t* newly_covered, uint64_t* edges_examined)
{
    uint32_t n = g->n;
    memcpy(snap, key, sizeof(uint64_t) * n);
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t du;
        uint32_t cu;
        if (frozen[u] && !Dfrozen) { du = 0; cu = center[u]; }
        else if (frozen[u] && Dfrozen[u] < delta) { du = Dfrozen[u]; cu = center[u]; }
        else if (frozen[u]) continue;
        else if (snap[u] != ORC_INF_KEY && (snap[u] >> 32) < delta) { du = snap[u] >> 32; cu = (uint32_t)snap[u]; }
        else continue;
        for (uint64_t j = g->off[u]; j < g->off[u + 1]; ++j) {
            uint32_t v = g->col[j];
            ++*edges_examined;
            if (frozen[v]) continue;
            uint64_t cand = du + g->wt[j];
            if (cand > delta) continue;
            uint64_t k = mkkey(cand, cu);
            if (k < key[v]) key[v] = k;
        }
    }
    uint64_t updated = 0;
    for (uint32_t v = 0; v < n; ++v) {
        if (frozen[v]) continue;
        if (key[v] < snap[v]) {
            ++updated;
            if (snap[v] == ORC_INF_KEY) ++*newly_covered;
        }
    }
    return updated;
}

/* Exposed for the brute-force pin: t synchronous steps at fixed Delta.
 * key[] holds unfrozen nodes' keys (ORC_INF_KEY = no center yet); frozen[v]
 * marks contracted nodes whose center is center[v]; Dfrozen (NULL: the
 * default contract mode) holds their bounds for the cumulative mode.
 * Per-step updated counts go to updated_out[t]. */
void orc_growth_steps(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt,
                      uint64_t* key, const uint8_t* frozen, const uint32_t* center, const uint64_t* Dfrozen,
                      uint32_t delta, uint32_t steps, uint64_t* updated_out)
{
    orc_graph g = {n, off, col, wt};
    uint64_t* snap = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint64_t cov = 0, ex = 0;
    for (uint32_t t = 0; t < steps; ++t)
        updated_out[t] = growing_step(&g, key, snap, frozen, center, Dfrozen, delta, &cov, &ex);
    free(snap);
}

/* ---------------------------------------------------------------------------
 * CLUSTER(G, tau), Algorithm 1, with the choices of Section 5 (initial Delta
 * given by the caller).  Readings fixed here where the paper leaves room:
 *  - log n = log2 of this graph's node count; gamma = 4 ln 2.
 *  - "uncovered" U = unfrozen nodes at the stage start; both half-tests are
 *    the integer test 2*covered >= |U|, covered = nodes of U holding a key.
 *  - center draw: v in U is selected iff Philox(seed; ctr = (v, stage, 0, 0))
 *    word 0 < thr, thr = floor(p * 2^32) (2^32 when p >= 1),
 *    p = gamma * tau * log n / |U|.  thr = 0 ends the loop (no node can be drawn).
 *  - contracted clusters of earlier stages relax as (0, c_u) from every frozen u.
 *  - a stage whose growth reached a fixed point with coverage still under half
 *    doubles Delta only while that can still cover a node: Delta below its cap
 *    2^31 and some covered or frozen node adjacent to an uncovered one.
 *  - D_v = d_v + R[c_v] is an upper bound on dist_G(c_v, v), R[c] being the
 *    largest D of c's cluster before the stage (d_v alone bounds the distance
 *    in the contracted graph only).
 * Outputs: center_out[v] (a node id) and D_out[v]; counters in *st; an
 * optional event trace (stage starts, steps, doublings, guard exits,
 * finalizations) in trace[0..trace_cap).
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t stages, steps, doublings, delta_end;
    uint32_t guard_exits, pad;
    uint64_t node_updates;
    uint64_t edges_examined;
    uint64_t centers_drawn;
} orc_stats;

typedef struct {
    uint32_t kind;   /* 0 step, 1 doubling, 2 finalize, 3 guard exit, 4 stage start */
    uint32_t stage;
    uint32_t delta;
    uint32_t pad;
    uint64_t a;      /* step: updated;  finalize: nodes frozen; stage start: |U| */
    uint64_t b;      /* step: covered after the step; stage start: centers drawn */
} orc_trace;

static int exists_growable_edge(const orc_graph* g, const uint64_t* key, const uint8_t* frozen)
{
    for (uint32_t u = 0; u < g->n; ++u) {
        if (!frozen[u] && key[u] == ORC_INF_KEY) continue; /* u must be covered or frozen */
        for (uint64_t j = g->off[u]; j < g->off[u + 1]; ++j) {
            uint32_t v = g->col[j];
            if (!frozen[v] && key[v] == ORC_INF_KEY) return 1;
        }
    }
    return 0;
}

/* Options beyond Algorithm 1's defaults (both off by default):
 *  - contract_mode 1 (cumulative): contracted nodes relax with their own
 *    distance bound D_u (not 0), so a new node's distance d_v already bounds
 *    dist_G(c_v, v) and D_v = d_v; every D then stays within the final Delta.
 *  - step_cap > 0: each execution of PartialGrowth performs at most step_cap
 *    growing steps (the O(n / tau) limit of Section 3's closing remark); if
 *    fewer than half of the nodes are covered afterwards, Delta doubles as
 *    when growth stops. */
int orc_cluster_opts(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt, double tau,
                     uint64_t seed, uint32_t delta0, int contract_mode, uint32_t step_cap, uint32_t* center_out,
                     uint64_t* D_out, orc_stats* st, orc_trace* trace, uint64_t trace_cap, uint64_t* trace_len)
{
    if (contract_mode != 0 && contract_mode != 1) return ORC_ERR_ARG;
    if (n == 0 || !(tau > 0.0) || delta0 == 0) return ORC_ERR_ARG;
    orc_graph g = {n, off, col, wt};
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint64_t* snap = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint8_t* frozen = (uint8_t*)calloc(n, 1);
    uint64_t* R = (uint64_t*)calloc(n, sizeof(uint64_t));
    uint64_t* newD = (uint64_t*)malloc(sizeof(uint64_t) * n);
    if (!key || !snap || !frozen || !R || !newD) {
        free(key); free(snap); free(frozen); free(R); free(newD);
        return ORC_ERR_OOM;
    }
    memset(st, 0, sizeof *st);
    uint64_t tl = 0;
#define TRACE(K, A, B)                                                                   \
    do {                                                                                 \
        if (trace && tl < trace_cap) {                                                   \
            trace[tl].kind = (K); trace[tl].stage = stage; trace[tl].delta = delta;      \
            trace[tl].pad = 0; trace[tl].a = (A); trace[tl].b = (B);                     \
        }                                                                                \
        ++tl;                                                                            \
    } while (0)

    const double L = log2((double)n);
    uint32_t delta = delta0 > ORC_DELTA_MAX ? ORC_DELTA_MAX : delta0;
    for (uint32_t v = 0; v < n; ++v) { center_out[v] = ORC_NONE; D_out[v] = 0; key[v] = ORC_INF_KEY; }
    uint32_t stage = 1;
    int rc = 0;
    for (;;) {
        uint64_t U = 0;
        for (uint32_t v = 0; v < n; ++v) U += frozen[v] ? 0 : 1;
        if (U == 0) break;
        if ((double)U < 8.0 * tau * L) break; /* outer while test of Algorithm 1 */
        double p = ORC_GAMMA * tau * L / (double)U;
        uint64_t thr = (p >= 1.0) ? 4294967296ull : (uint64_t)floor(p * 4294967296.0);
        if (thr == 0) break;
        if (stage > ORC_MAX_STAGES) { rc = ORC_ERR_DIVERGED; break; }

        /* selection and state reset */
        uint64_t covered = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (frozen[v]) continue;
            if ((uint64_t)philox_x0(seed, v, stage) < thr) { key[v] = mkkey(0, v); ++covered; }
            else key[v] = ORC_INF_KEY;
        }
        st->centers_drawn += covered;
        TRACE(4, U, covered);

        /* inner while loop with PartialGrowth */
        for (;;) {
            uint64_t updated;
            uint32_t growth_steps = 0;
            do {
                updated = growing_step(&g, key, snap, frozen, center_out, contract_mode ? D_out : NULL, delta,
                                       &covered, &st->edges_examined);
                st->steps++;
                st->node_updates += updated;
                ++growth_steps;
                TRACE(0, updated, covered);
            } while (updated != 0 && 2 * covered < U && (step_cap == 0 || growth_steps < step_cap));
            if (2 * covered >= U) break;
            if (delta >= ORC_DELTA_MAX || !exists_growable_edge(&g, key, frozen)) {
                st->guard_exits++;
                TRACE(3, 0, covered);
                break;
            }
            delta = (delta > ORC_DELTA_MAX / 2) ? ORC_DELTA_MAX : 2 * delta;
            st->doublings++;
            TRACE(1, 0, covered);
        }

        /* assign covered nodes to their clusters and contract */
        uint64_t nf = 0, stage_max_D = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (frozen[v] || key[v] == ORC_INF_KEY) continue;
            uint32_t c = (uint32_t)key[v];
            newD[v] = (key[v] >> 32) + (contract_mode ? 0 : R[c]);
        }
        for (uint32_t v = 0; v < n; ++v) {
            if (frozen[v] || key[v] == ORC_INF_KEY) continue;
            uint32_t c = (uint32_t)key[v];
            frozen[v] = 1;
            center_out[v] = c;
            D_out[v] = newD[v];
            if (newD[v] > R[c]) R[c] = newD[v];
            if (newD[v] > stage_max_D) stage_max_D = newD[v];
            ++nf;
        }
        TRACE(2, nf, stage_max_D);
        st->stages++;
        ++stage;
    }
    /* remaining uncovered nodes become singleton clusters */
    for (uint32_t v = 0; v < n; ++v)
        if (!frozen[v]) { frozen[v] = 1; center_out[v] = v; D_out[v] = 0; }
    st->delta_end = delta;
    if (trace_len) *trace_len = tl;
#undef TRACE
    free(key); free(snap); free(frozen); free(R); free(newD);
    return rc;
}

int orc_cluster(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt, double tau,
                uint64_t seed, uint32_t delta0, uint32_t* center_out, uint64_t* D_out, orc_stats* st,
                orc_trace* trace, uint64_t trace_cap, uint64_t* trace_len)
{
    return orc_cluster_opts(n, off, col, wt, tau, seed, delta0, 0, 0, center_out, D_out, st, trace, trace_cap,
                            trace_len);
}

/* ---------------------------------------------------------------------------
 * CLUSTER2(G, tau), Algorithm 2 (Section 4), with PartialGrowth2 and Contract2
 * taken literally: the current graph G_i is an explicit list of undirected
 * edges whose ends are clusters formed so far (named by their center) or
 * nodes not yet covered.  Readings fixed here where the paper leaves room:
 *  - R_CL = largest D_v of CLUSTER(G, tau) run with the same options (its radius);
 *    Delta = 2 R_CL throughout.
 *  - the for loop runs i = 1..L, L = the least i >= 1 with 2^i >= n (log n rounded
 *    up), so the last iteration draws every node still uncovered.
 *  - center draw in iteration i: an uncovered v is drawn iff
 *    Philox(seed; ctr = (v, i, 1, 0)) word 0 < thr_i, thr_i = floor(2^i 2^32 / n)
 *    (2^32 when 2^i >= n).
 *  - growing steps as in CLUSTER (synchronous; (distance, center id) order;
 *    a relaxation is kept when d_u + w <= Delta); centers keep (0, c).
 *  - G_1 holds the edges of G of weight <= 2 R_CL: heavier ones are never used.
 *  - Contract2 keeps an edge between two uncovered nodes, maps an edge with
 *    exactly one covered end a (cluster c_a, distance d_a) to (c_a, b) with
 *    weight d_a + w - 2 R_CL, and drops an edge with both ends covered.
 *  - D_v = d_v + (i_v - i_c) 2 R_CL, v reached at distance d_v in G_{i_v} and its
 *    center drawn in iteration i_c: by induction over the contractions, the
 *    length of a path of G from c_v to v.
 * Outputs center_out[v], D_out[v]; counters in *st.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t iterations, steps;
    uint64_t centers_drawn;
    uint64_t node_updates;
    uint64_t r_cl;
} orc_c2_stats;

int orc_cluster2(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt, double tau,
                 uint64_t seed, uint32_t delta0, int contract_mode, uint32_t step_cap, uint32_t* center_out,
                 uint64_t* D_out, orc_c2_stats* st)
{
    memset(st, 0, sizeof *st);
    orc_stats s1;
    int rc = orc_cluster_opts(n, off, col, wt, tau, seed, delta0, contract_mode, step_cap, center_out, D_out, &s1,
                              NULL, 0, NULL);
    if (rc != 0) return rc;
    uint64_t R = 0;
    for (uint32_t v = 0; v < n; ++v) if (D_out[v] > R) R = D_out[v];
    const uint64_t delta = 2 * R;
    st->r_cl = R;

    /* G_1: undirected edges (a, b, w), a < b, w <= Delta */
    uint64_t m = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t j = off[u]; j < off[u + 1]; ++j)
            if (u < col[j] && wt[j] <= delta) ++m;
    uint32_t* ea = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* eb = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t* ew = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint8_t* cov = (uint8_t*)calloc(n, 1);        /* covered (a center or reached) */
    uint32_t* ccov = (uint32_t*)malloc(sizeof(uint32_t) * n);  /* center of a covered node */
    uint32_t* it_sel = (uint32_t*)calloc(n, sizeof(uint32_t)); /* iteration a center was drawn */
    uint32_t* it_cov = (uint32_t*)calloc(n, sizeof(uint32_t)); /* iteration a node was covered */
    uint64_t* dcov = (uint64_t*)calloc(n, sizeof(uint64_t));   /* its distance in that G_i */
    uint64_t* kd = (uint64_t*)malloc(sizeof(uint64_t) * n);    /* state (d, c) of the nodes of G_i */
    uint32_t* kc = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* sd = (uint64_t*)malloc(sizeof(uint64_t) * n);    /* its snapshot at a step start */
    uint32_t* sc = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint8_t* upd = (uint8_t*)malloc(n);
    if (!ea || !eb || !ew || !cov || !ccov || !it_sel || !it_cov || !dcov || !kd || !kc || !sd || !sc || !upd) {
        rc = ORC_ERR_OOM;
        goto done;
    }
    m = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t j = off[u]; j < off[u + 1]; ++j)
            if (u < col[j] && wt[j] <= delta) { ea[m] = u; eb[m] = col[j]; ew[m] = wt[j]; ++m; }

    uint32_t L = 1;
    while (((uint64_t)1 << L) < (uint64_t)n) ++L;
    st->iterations = L;
    for (uint32_t i = 1; i <= L; ++i) {
        const uint64_t thr = (((uint64_t)1 << i) >= (uint64_t)n) ? 4294967296ull : ((uint64_t)1 << (32 + i)) / n;
        /* new centers among the uncovered nodes */
        for (uint32_t v = 0; v < n; ++v) {
            if (cov[v]) continue;
            uint32_t ctr[4] = {v, i, 1, 0}, out[4];
            orc_philox4x32_10(seed, ctr, out);
            if ((uint64_t)out[0] < thr) {
                cov[v] = 1; ccov[v] = v; it_sel[v] = i; it_cov[v] = i; dcov[v] = 0;
                st->centers_drawn++;
            }
        }
        /* states of G_i's nodes: every center (0, c); uncovered nodes (inf, nil) */
        for (uint32_t v = 0; v < n; ++v) {
            if (cov[v] && ccov[v] == v) { kd[v] = 0; kc[v] = v; }
            else { kd[v] = UINT64_MAX; kc[v] = ORC_NONE; }
        }
        /* PartialGrowth2: growing steps until no state is updated */
        for (;;) {
            memcpy(sd, kd, sizeof(uint64_t) * n);
            memcpy(sc, kc, sizeof(uint32_t) * n);
            memset(upd, 0, n);
            for (uint64_t e = 0; e < m; ++e) {
                for (int dir = 0; dir < 2; ++dir) {
                    const uint32_t a = dir ? eb[e] : ea[e], b = dir ? ea[e] : eb[e];
                    if (sd[a] == UINT64_MAX || cov[b]) continue;  /* b must be an uncovered node */
                    const uint64_t cand = sd[a] + ew[e];
                    if (cand > delta) continue;
                    if (cand < kd[b] || (cand == kd[b] && sc[a] < kc[b])) { kd[b] = cand; kc[b] = sc[a]; upd[b] = 1; }
                }
            }
            uint64_t u = 0;
            for (uint32_t v = 0; v < n; ++v) u += upd[v];
            st->steps++;
            st->node_updates += u;
            if (u == 0) break;
        }
        /* the reached nodes join their clusters */
        for (uint32_t v = 0; v < n; ++v) {
            if (cov[v] || kd[v] == UINT64_MAX) continue;
            cov[v] = 2;  /* covered in this iteration (kept distinct until the contraction below) */
            ccov[v] = kc[v]; it_cov[v] = i; dcov[v] = kd[v];
        }
        /* Contract2 */
        uint64_t m2 = 0;
        for (uint64_t e = 0; e < m; ++e) {
            const uint32_t a = ea[e], b = eb[e];
            const int ca = cov[a] != 0, cb = cov[b] != 0;
            if (ca && cb) continue;
            if (!ca && !cb) { ea[m2] = a; eb[m2] = b; ew[m2] = ew[e]; ++m2; continue; }
            const uint32_t x = ca ? a : b, y = ca ? b : a;  /* x covered, y not */
            const uint64_t dx = kd[x];                     /* 0 for a center, else its distance this iteration */
            if (dx + ew[e] <= delta) { rc = ORC_ERR_DIVERGED; goto done; }  /* y would have been reached */
            ea[m2] = ccov[x]; eb[m2] = y; ew[m2] = dx + ew[e] - delta; ++m2;
        }
        m = m2;
        for (uint32_t v = 0; v < n; ++v) if (cov[v] == 2) cov[v] = 1;
    }
    for (uint32_t v = 0; v < n; ++v) {
        if (!cov[v]) { rc = ORC_ERR_DIVERGED; goto done; }  /* the last iteration draws every uncovered node */
        center_out[v] = ccov[v];
        D_out[v] = dcov[v] + (uint64_t)(it_cov[v] - it_sel[ccov[v]]) * delta;
    }
done:
    free(ea); free(eb); free(ew); free(cov); free(ccov); free(it_sel); free(it_cov); free(dcov);
    free(kd); free(kc); free(sd); free(sc); free(upd);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Weighted quotient graph (Section 4): one node per cluster, numbered by
 * increasing center id; for each edge (u,v) of G with c_u != c_v an edge
 * between their clusters of weight w(u,v) + D_u + D_v, keeping the minimum
 * per cluster pair.  Output is a symmetric CSR sorted by (row, col).
 * Buffers: cid_out[n], q_off[k+1] (k <= n), q_col/q_w[nnz(G)].
 * Returns the number of directed quotient entries.
 * ------------------------------------------------------------------------- */
typedef struct { uint32_t a, b; uint64_t w; } orc_qtrip;

static int cmp_qtrip(const void* p, const void* q)
{
    const orc_qtrip* x = (const orc_qtrip*)p;
    const orc_qtrip* y = (const orc_qtrip*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

int64_t orc_quotient(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt,
                     const uint32_t* center, const uint64_t* D, uint32_t* cid_out, uint32_t* k_out,
                     uint64_t* q_off, uint32_t* q_col, uint64_t* q_w)
{
    uint32_t* rank = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!rank) return ORC_ERR_OOM;
    uint32_t k = 0;
    for (uint32_t v = 0; v < n; ++v) rank[v] = (center[v] == v) ? k++ : ORC_NONE;
    for (uint32_t v = 0; v < n; ++v) cid_out[v] = rank[center[v]];
    free(rank);
    *k_out = k;

    uint64_t cap = off[n] ? off[n] : 1;
    orc_qtrip* t = (orc_qtrip*)malloc(sizeof(orc_qtrip) * cap);
    if (!t) return ORC_ERR_OOM;
    uint64_t nt = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t j = off[u]; j < off[u + 1]; ++j) {
            uint32_t v = col[j];
            if (cid_out[u] == cid_out[v]) continue;
            t[nt].a = cid_out[u];
            t[nt].b = cid_out[v];
            t[nt].w = D[u] + (uint64_t)wt[j] + D[v];
            ++nt;
        }
    }
    /* both directions of every edge are present already (the CSR is symmetric) */
    qsort(t, nt, sizeof(orc_qtrip), cmp_qtrip);
    uint64_t nq = 0;
    for (uint32_t a = 0; a <= k; ++a) q_off[a] = 0;
    for (uint64_t i = 0; i < nt; ++i) {
        if (nq > 0 && i > 0 && t[i].a == t[i - 1].a && t[i].b == t[i - 1].b) continue; /* first = min */
        q_col[nq] = t[i].b;
        q_w[nq] = t[i].w;
        q_off[t[i].a + 1]++;
        ++nq;
    }
    for (uint32_t a = 0; a < k; ++a) q_off[a + 1] += q_off[a];
    free(t);
    return (int64_t)nq;
}

/* ---------------------------------------------------------------------------
 * Dijkstra with a binary heap (lazy deletion).  Distances in uint64,
 * UINT64_MAX = unreachable.  Exactly one of wt32 / wt64 is non-null.
 * ------------------------------------------------------------------------- */
typedef struct { uint64_t d; uint32_t v; } orc_hn;

static void heap_push(orc_hn* h, uint64_t* sz, orc_hn x)
{
    uint64_t i = (*sz)++;
    h[i] = x;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d < h[i].d || (h[p].d == h[i].d && h[p].v <= h[i].v)) break;
        orc_hn t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static orc_hn heap_pop(orc_hn* h, uint64_t* sz)
{
    orc_hn top = h[0];
    h[0] = h[--*sz];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *sz && (h[l].d < h[s].d || (h[l].d == h[s].d && h[l].v < h[s].v))) s = l;
        if (r < *sz && (h[r].d < h[s].d || (h[r].d == h[s].d && h[r].v < h[s].v))) s = r;
        if (s == i) break;
        orc_hn t = h[s]; h[s] = h[i]; h[i] = t;
        i = s;
    }
    return top;
}

int orc_dijkstra(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt32,
                 const uint64_t* wt64, uint32_t source, uint64_t* dist)
{
    if (source >= n) return ORC_ERR_ARG;
    uint64_t nnz = off[n];
    orc_hn* h = (orc_hn*)malloc(sizeof(orc_hn) * (nnz + 2));
    uint8_t* done = (uint8_t*)calloc(n, 1);
    if (!h || !done) { free(h); free(done); return ORC_ERR_OOM; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = UINT64_MAX;
    uint64_t sz = 0;
    dist[source] = 0;
    orc_hn s0 = {0, source};
    heap_push(h, &sz, s0);
    while (sz > 0) {
        orc_hn x = heap_pop(h, &sz);
        if (done[x.v]) continue;
        done[x.v] = 1;
        for (uint64_t j = off[x.v]; j < off[x.v + 1]; ++j) {
            uint32_t v = col[j];
            uint64_t w = wt32 ? wt32[j] : wt64[j];
            uint64_t nd = x.d + w;
            if (nd < dist[v]) {
                dist[v] = nd;
                orc_hn y = {nd, v};
                heap_push(h, &sz, y);
            }
        }
    }
    free(h);
    free(done);
    return 0;
}

/* Phi of a graph given as CSR with uint64 weights: the largest finite
 * shortest-path distance (Section 2; per component if disconnected), by one
 * Dijkstra per node.  Used on the quotient graph G_C (Section 4). */
int orc_apsp_max(uint32_t k, const uint64_t* q_off, const uint32_t* q_col, const uint64_t* q_w, uint64_t* phi)
{
    uint64_t* dist = (uint64_t*)malloc(sizeof(uint64_t) * (k ? k : 1));
    if (!dist) return ORC_ERR_OOM;
    uint64_t best = 0;
    for (uint32_t s = 0; s < k; ++s) {
        int rc = orc_dijkstra(k, q_off, q_col, NULL, q_w, s, dist);
        if (rc) { free(dist); return rc; }
        for (uint32_t v = 0; v < k; ++v)
            if (dist[v] != UINT64_MAX && dist[v] > best) best = dist[v];
    }
    free(dist);
    *phi = best;
    return 0;
}

/* Source of the SSSP-based 2-approximation (Section 5, "starting from a random
 * node"): Philox(seed; ctr = (2^32-1, 2^32-1, 0, 0)) word 0 mod n. */
uint32_t orc_sssp_source(uint64_t seed, uint32_t n)
{
    return philox_x0(seed, 0xFFFFFFFFu, 0xFFFFFFFFu) % n;
}

/* Eccentricity of a node = largest finite distance from it. */
static uint64_t ecc_of(const uint64_t* dist, uint32_t n, uint32_t* far)
{
    uint64_t e = 0;
    uint32_t f = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (dist[v] != UINT64_MAX && dist[v] > e) { e = dist[v]; f = v; }
    if (far) *far = f;
    return e;
}

/* Lower bound on Phi(G) used for the approximation ratios of Table 2: repeated
 * exact SSSP, each from the node farthest from the previous source (lowest id
 * among equals).  Returns the largest eccentricity seen; ecc_first gets the
 * first source's eccentricity (half the SSSP 2-approximation upper bound). */
int orc_lower_bound(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* wt, uint32_t source,
                    uint32_t sweeps, uint64_t* lb, uint64_t* ecc_first)
{
    uint64_t* dist = (uint64_t*)malloc(sizeof(uint64_t) * n);
    if (!dist) return ORC_ERR_OOM;
    uint64_t best = 0;
    uint32_t s = source;
    for (uint32_t i = 0; i < sweeps; ++i) {
        int rc = orc_dijkstra(n, off, col, wt, NULL, s, dist);
        if (rc) { free(dist); return rc; }
        uint32_t far;
        uint64_t e = ecc_of(dist, n, &far);
        if (i == 0 && ecc_first) *ecc_first = e;
        if (e > best) best = e;
        s = far;
    }
    free(dist);
    *lb = best;
    return 0;
}
