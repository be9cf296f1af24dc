"""Benchmark of the GB300 CL-DIAM hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload rmat24]

One step = the whole CL-DIAM pass on one synthetic graph whose edge list is
already resident in HBM: CSR build (dedup, symmetrise, LCC), initial Delta,
CLUSTER(tau), quotient contraction and the estimate Phi(G_C) + 2R.  value =
m_LCC / step time in GTEPS (undirected edges of the processed graph).  The
headline workload is R-MAT scale 24 (the paper's R-MAT(24) row, Table 2; its
3.2 GB edge list and 6.2 GB CSR are far larger than the 129 MB L2, so no flush
is needed between steps).

Also reported on the same line: the end-to-end rate through cldiam_run with
pinned host buffers (H2D copies inside the timed region), the roofline of the
dominant kernel class and of the Delta-growing step (both of its forms) from
live CUDA-event timing, the same step on the R-MAT 20 and road-mesh workloads,
the Delta-stepping baseline, the many-graph and served forms, SM clocks
sampled during the timed region, and the CPU oracle timed on one host thread.

With --impl reference the CPU oracle (a sequential program written from the
paper) is timed instead, on a bounded sample (R-MAT scale 17, about a second a
step).  Under torchrun (N > 1) every rank runs an independent replica (weak
scaling; the single-graph path has no exchange step), and rank 0 prints the
line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS and graphs/sec (batched+served vs plain) at bit-exact; HBM % peak; p99 ms"
SAMPLE_SCALE = 17  # CPU oracle sample: R-MAT scale 17 with the rmat20 recipe
BASE_TUNING = {}  # --tuning: process-wide knobs for the whole run


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat24")
    ap.add_argument("--secondary", default="rmat20,roadmesh4096",
                    help="other single-graph workloads timed the same way on the same line ('' = none)")
    ap.add_argument("--secondary-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", default="",
                    help="process-wide tuning knobs for the whole run, e.g. pull_ratio=0.5,relax_ctas_per_sm=4")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-batched", action="store_true", help="skip the many-graph leg")
    ap.add_argument("--batched-count", type=int, default=2000)
    ap.add_argument("--no-served", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000")
    ap.add_argument("--plain-sample-every", type=int, default=10)
    ap.add_argument("--no-delta0-experiment", action="store_true", help="skip the initial-Delta experiment")
    ap.add_argument("--no-cluster2", action="store_true", help="skip the CLUSTER2 (Algorithm 2) leg")
    ap.add_argument("--no-tuned-cluster", action="store_true",
                    help="skip the autotuned CLUSTER + quotient + estimate leg on the headline graph")
    ap.add_argument("--profile-pass", action="store_true",
                    help="run one pipeline pass on the workload and exit (for ncu captures)")
    ap.add_argument("--profile-sssp", action="store_true",
                    help="build the workload's CSR, run one Delta-stepping SSSP and exit (for ncu captures)")
    ap.add_argument("--profile-cluster2", action="store_true",
                    help="build the workload's CSR, run CLUSTER2 + quotient + estimate once and exit")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="pack this many mixture graphs into an arena, run one batch and exit")
    ap.add_argument("--profile-apsp", type=int, default=0,
                    help="Phi of one dense random k-node graph (the blocked Floyd-Warshall path) and exit")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_pass(e, tau, seed):
    """One oracle pass (CSR build + LCC + CLUSTER + quotient + estimate); returns (seconds, m_LCC, n_LCC)."""
    import oracle
    t0 = time.perf_counter()
    g = oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=True)
    d0 = oracle.delta0(g)
    cl = oracle.cluster(g, tau, seed, d0)
    q = oracle.quotient(g, cl)
    oracle.estimate(q, cl)
    return time.perf_counter() - t0, g.m, g.n


def oracle_sample_run(scale: int = SAMPLE_SCALE):
    """One oracle pass on the bounded R-MAT sample; returns (seconds, m_LCC, describe)."""
    import inputs
    from inputs.workloads import WORKLOADS
    wl = WORKLOADS["rmat20"]
    e = inputs.rmat(scale, 16, 1 << 20, wl.seed)
    dt, m, n = oracle_pass(e, wl.tau, wl.seed)
    return dt, m, (f"R-MAT scale {scale} (edge factor 16, w in [1,2^20], seed {wl.seed}, LCC n={n}, "
                   f"m={m}), tau {wl.tau}: CSR build + CLUSTER + quotient + estimate, one thread")


def cpu_baseline_leg():
    """The oracle, as it stands, on one host thread: one full pass over the R-MAT 20 workload (the headline's
    R-MAT family at 1/16 of its edges; the R-MAT 24 pass takes about ten minutes)."""
    from inputs.workloads import WORKLOADS
    wl = WORKLOADS["rmat20"]
    e = wl.make()
    dt, m, n = oracle_pass(e, wl.tau, wl.seed)
    return {"value": round(m / dt / 1e9, 6), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": (f"the rmat20 workload ({wl.describe}; LCC n={n}, m={m}), tau {wl.tau}, one full pass: "
                       f"CSR build + LCC + CLUSTER + quotient + estimate on one thread, {dt:.1f} s")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_run()
    times, m, desc = [], 0, ""
    for _ in range(args.steps):
        dt, m, desc = oracle_sample_run()
        times.append(dt)
    t = sum(times) / len(times)
    v = m / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": round(v, 6), "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 6), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def wait_first(self, timeout=5.0):
        t0 = time.time()
        while self.proc and not self.rows and time.time() - t0 < timeout:
            time.sleep(0.05)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=3)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = [r for (t, r) in self.rows if t0 <= t <= t1 + 0.15]
        window = True
        if not rows:
            rows = [r for (_, r) in self.rows[-3:]]
            window = False
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, val in zip(names, r[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "in_window": window,
                "power_w_max": max(float(r[4]) for r in rows if r[4].replace(".", "").isdigit()) if rows else None}


# ----------------------------------------------------------------------------- many-graph leg
def mix_shard(count, rank, world):
    """Graph indices of this rank: largest-first bin packing on the generator's edge counts."""
    import inputs
    from inputs.workloads import MIX_SEED
    from paper_1506_03265_gb300.shard import lpt_partition
    if world == 1:
        return list(range(count))
    sizes = []
    for g in range(count):
        kind, scale, side, _ = inputs.mix_params(MIX_SEED, g)
        sizes.append(8 * (1 << scale) if kind == 0 else 2 * side * (side - 1))
    return lpt_partition(sizes, world)[rank]


def build_mix_arena(cd, stream, count, budget=0, rank=0, world=1):
    """This rank's share of the many-graph workload packed into one arena:
    (arena, ids, taus, seeds, undirected edges, seconds)."""
    import inputs
    from inputs.workloads import MIX_SEED, mixture_tau
    arena = cd.arena_create(hbm_budget_bytes=budget, stream=stream)
    ids, taus, seeds, edges = [], [], [], 0
    t0 = time.perf_counter()
    for g in mix_shard(count, rank, world):
        e = inputs.mix_graph(MIX_SEED, g, 1000)
        gid = arena.add(e.src, e.dst, e.w, e.n)
        view = arena.graph(gid)
        n = view.n
        edges += view.nnz // 2
        view.free()
        ids.append(gid)
        taus.append(mixture_tau(n))
        seeds.append(MIX_SEED * 1000 + g)
    return arena, ids, taus, seeds, edges, time.perf_counter() - t0


def batched_leg(cd, stream, mix, sample_every, reps=3, dist=None, total_count=None):
    """graphs/s of one persistent batch launch vs the plain one-graph-per-call loop (same jobs).
    With several ranks each runs its share; the batch time is the max over ranks."""
    import torch

    from inputs.workloads import MIX_DESCRIBE
    from paper_1506_03265_gb300.shard import max_over_ranks, sum_over_ranks
    arena, ids, taus, seeds, edges, build_s = mix
    count = len(ids)
    res, st = arena.run(ids, taus, seeds)  # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    cd.profile_reset()
    e0.record(stream)
    for _ in range(reps):
        res2, _ = arena.run(ids, taus, seeds)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    launches = sum(v["launches"] for v in cd.profile_get().values()) / reps
    assert res2 == res
    # per-job device times of the last batch: the tail of the persistent launch
    js, je = arena.job_times(count)
    jt = je - js
    ctas = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    job_times = {"job_ms_p50": round(1e3 * float(np.percentile(jt, 50)), 3),
                 "job_ms_p99": round(1e3 * float(np.percentile(jt, 99)), 3),
                 "job_ms_max": round(1e3 * float(jt.max()), 3),
                 "makespan_ms": round(1e3 * float(je.max()), 3),
                 "balanced_ms": round(1e3 * float(jt.sum()) / ctas, 3),
                 "last_job_start_ms": round(1e3 * float(js.max()), 3),
                 "what": ("device time per job (one CTA each: no graph of this batch outweighs the per-CTA average); "
                          f"balanced_ms = the sum of job times over the {ctas} CTAs, the makespan a perfect split "
                          "would give")}
    # a small batch (the first 50 jobs) is bound by its largest job: one CTA per job vs CTA groups
    small = {}
    sids, staus, sseeds = ids[:50], taus[:50], seeds[:50]
    for split in (1, 2):
        cd.tuning_set(**{**BASE_TUNING, "batch_split": split})
        ref_small, _ = arena.run(sids, staus, sseeds)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            rs, _ = arena.run(sids, staus, sseeds)
        e1.record(stream)
        torch.cuda.synchronize()
        sj, sje = arena.job_times(len(sids))
        small["split" if split == 2 else "all_in_launch"] = {
            "ms_per_batch": round(e0.elapsed_time(e1) / reps, 3), "makespan_ms": round(1e3 * float(sje.max()), 3),
            "job_ms_max": round(1e3 * float((sje - sj).max()), 3), "identical": bool(rs == ref_small)}
        small.setdefault("results", []).append(rs)
    cd.tuning_set(**BASE_TUNING)
    small_same = small.pop("results")
    small["identical_across_forms"] = bool(small_same[0] == small_same[1])
    small["what"] = ("the mixture's first 50 jobs: batch_split = 1 (every graph in the persistent launch, one CTA "
                     "each) vs 2, the default (a graph that outweighs the per-CTA average runs first on the "
                     "one-graph path with the whole device)")
    # autotuned: the many-graph knobs picked on these jobs (cached for the batch's size class), then timed
    tuned = arena.autotune(ids, taus, seeds, reps=2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        res3, _ = arena.run(ids, taus, seeds)
    e1.record(stream)
    torch.cuda.synchronize()
    t_tuned = e0.elapsed_time(e1) / 1e3 / reps
    tuned_same = res3 == res
    # plain loop over a sample of the same jobs
    sample = list(range(0, count, sample_every))
    same = True
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    for i in sample:
        g = arena.graph(ids[i])
        r = cd.estimate(cd.quotient_build(cd.cluster(g, taus[i], seeds[i])))
        same &= all(r[f] == res[i][f] for f in r)
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - p0) / len(sample)
    if dist is not None and dist.is_initialized():
        dev = torch.device("cuda", torch.cuda.current_device())
        t_batch = max_over_ranks(t_batch, dist, dev)
        edges = int(sum_over_ranks(edges, dist, dev))
        count = int(sum_over_ranks(count, dist, dev))
    gps = count / t_batch
    if dist is not None and dist.is_initialized():
        t_tuned = max_over_ranks(t_tuned, dist, dev)
    return {"workload": "mix2000", "describe": MIX_DESCRIBE, "graphs": count, "undirected_edges": edges,
            "job_times": job_times, "small_batch": small,
            "tuned": {"graphs_per_s": round(count / t_tuned, 1), "ms_per_batch": round(t_tuned * 1e3, 2),
                      "knobs": {"batch_fw_k": tuned["batch_fw_k"], "batch_split": tuned["batch_split"]},
                      "identical_to_default": bool(tuned_same),
                      "what": "cldiam_autotune_batch on the same jobs (median of 2 runs per candidate), then "
                              "the same timed loop with the cached choice"},
            "scaling": "strong (the 2,000 graphs are split across ranks by size)",
            "graphs_per_s": round(gps, 1), "gteps": round(edges / t_batch / 1e9, 4),
            "ms_per_batch": round(t_batch * 1e3, 2), "kernel_launches_per_batch": launches,
            "plain_graphs_per_s": round(1.0 / t_plain, 1), "speedup_vs_plain": round(gps * t_plain, 2),
            "plain_sample": f"every {sample_every}th job ({len(sample)} graphs), cldiam_cluster + "
                            "cldiam_quotient_build + cldiam_estimate per graph on the same GPU",
            "identical_to_plain_on_sample": bool(same), "arena_build_s": round(build_s, 1)}


def served_leg(cd, mix, rates, count=20000, plain_count=1000, seed=5):
    """Poisson query stream over the mixture + 1% R-MAT 20: continuous-batching server vs plain FIFO loop."""
    import inputs
    from inputs.workloads import WORKLOADS
    arena, ids, taus, seeds, _, _ = mix
    wl = WORKLOADS["rmat20"]
    e = wl.make()
    big = arena.add(e.src, e.dst, e.w, e.n)
    g_ids = list(ids) + [big]
    g_taus = list(taus) + [wl.tau]
    srv = cd.server_create(arena, hbm_budget_bytes=150 * 10**9)
    out = {"workload": "serve20k", "describe": (f"{count} queries, seed {seed}, exponential inter-arrival times; "
                                                "each on a graph of the 2,000-graph mixture (p = 0.99) or on the "
                                                "R-MAT 20 workload graph (p = 0.01); HBM budget 150 GB"),
           "queries": count, "arena_device_bytes": arena.info()[1], "rates": []}
    same = True
    for rate in rates:
        arr, gsel = inputs.queries(seed, count, float(rate), 0.01, len(ids))
        q_ids = [g_ids[x] for x in gsel]
        q_taus = [g_taus[x] for x in gsel]
        q_seeds = [seed * 100000 + i for i in range(count)]
        res, lat, el = srv.replay(q_ids, q_taus, q_seeds, arr)
        k = plain_count
        res_p, lat_p, el_p = srv.replay(q_ids[:k], q_taus[:k], q_seeds[:k], arr[:k], plain=True)
        same &= res[:k] == res_p
        out["rates"].append({
            "rate_qps": rate, "qps": round(count / el, 1), "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
            "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3), "big_queries": int((gsel == len(ids)).sum()),
            "plain_qps": round(k / el_p, 1), "plain_p50_ms": round(1e3 * float(np.percentile(lat_p, 50)), 3),
            "plain_p99_ms": round(1e3 * float(np.percentile(lat_p, 99)), 3)})
    srv.free()
    out["plain"] = (f"the first {plain_count} queries of each trace served one at a time in arrival order "
                    "(cldiam_cluster + cldiam_quotient_build + cldiam_estimate per query) on the same GPU")
    out["identical_to_plain"] = bool(same)
    best = max(out["rates"], key=lambda r: r["qps"])
    out["speedup_qps_vs_plain"] = round(best["qps"] / max(r["plain_qps"] for r in out["rates"]), 2)
    return out


# ----------------------------------------------------------------------------- initial-Delta experiment
def delta0_leg(cd, side=2048, tau=5.4, seed=7):
    """The initial-Delta experiment of Section 5 on a mesh with two edge weights (integer form of the
    paper's 1 with probability 0.1 and 1e-6 otherwise): CL-DIAM started at the minimum weight (Delta
    grows by doubling) against CL-DIAM started at the graph's diameter (no doubling); each ratio is
    Phi_approx over a lower bound from farthest-node SSSP sweeps (exact Delta-stepping distances)."""
    import inputs
    e = inputs.grid(side, 10, seed)
    w = np.where(e.w == 1, 1_000_000, 1).astype(np.uint32)  # a uniform draw in [1, 10] is 1 w.p. 0.1
    g = cd.build_csr(e.src, e.dst, w, e.n)
    # lower bound on the diameter: four farthest-node sweeps from the Philox source
    src = cd.sssp_source(g, seed)
    lb = 0
    for _ in range(4):
        dist, ecc, _ = cd.sssp_delta(g, src)
        lb = max(lb, int(ecc))
        src = int(np.argmax(np.where(dist == 0xFFFFFFFF, 0, dist)))
    out = {"workload": f"mesh {side}x{side}, w = 10^6 with probability 0.1 else 1, seed {seed}, tau {tau}",
           "diameter_lower_bound": lb}
    for name, mode, d0, cm in (("delta0_min", cd.DELTA0_MIN, 0, cd.CONTRACT_RESET),
                               ("delta0_diameter", cd.DELTA0_EXPLICIT, lb, cd.CONTRACT_RESET),
                               ("delta0_min_cumulative", cd.DELTA0_MIN, 0, cd.CONTRACT_CUMULATIVE),
                               ("delta0_diameter_cumulative", cd.DELTA0_EXPLICIT, lb, cd.CONTRACT_CUMULATIVE)):
        t0 = time.perf_counter()
        c = cd.cluster(g, tau, seed, delta0_mode=mode, delta0=d0, contract_mode=cm)
        r = cd.estimate(cd.quotient_build(c))
        out[name] = {"delta0": int(d0) if d0 else 1, "delta_end": r["delta_end"], "doublings": r["doublings"],
                     "steps": r["steps"], "k": r["k"], "phi_approx": r["phi_approx"],
                     "ratio": round(r["phi_approx"] / lb, 4), "ms": round((time.perf_counter() - t0) * 1e3, 2)}
    out["paper"] = "Section 5: ratio 1.0001 (start at the minimum weight) vs about 2.5 (start at the diameter)"
    return out


# ----------------------------------------------------------------------------- GPU leg
RELAX_CLASSES = ("relax", "relax_pull")  # the two forms of the Delta-growing step (row a5)


def load_peaks():
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pk)) if os.path.exists(pk) else {}


def stored_traffic(workload, cls, alg_bytes_per_launch=None):
    """DRAM bytes per launch of a kernel class from the committed ncu summary, while its source is unchanged:
    either captured on the workload itself, or (a workload too large to capture under the size rule)
    captured on a smaller one above the L2 size and scaled by the algorithmic bytes per launch, i.e. by the
    units a launch processes."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None
    ent = json.load(open(tpath)).get(workload, {}).get(cls)
    if not ent:
        return None
    src = os.path.join(ROOT, ent.get("source_file", ""))
    same = os.path.isfile(src) and hashlib.sha256(open(src, "rb").read()).hexdigest() == ent.get("source_sha256")
    if not same:
        return None
    if "dram_bytes_per_launch" in ent:
        return ent["dram_bytes_per_launch"]
    if "dram_per_alg_byte" in ent and alg_bytes_per_launch:
        return round(ent["dram_per_alg_byte"] * alg_bytes_per_launch)
    return None


def roofline_of(prof, classes, peak, peaks, workload, tkey=None):
    """HBM roofline of one kernel class (or the sum of several): algorithmic bytes of its launches in the
    timed region / their CUDA-event time (events on the library's stream)."""
    b = sum(prof[c]["bytes"] for c in classes)
    ms = sum(prof[c]["ms"] for c in classes)
    launches = sum(prof[c]["launches"] for c in classes)
    achieved = b / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"bound": "hbm", "kernel": "+".join(classes), "achieved": round(achieved, 1) if achieved else None,
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
            "traffic": stored_traffic(workload, tkey or classes[0], b / max(1, launches)), "launches": launches,
            "alg_bytes_per_launch": round(b / max(1, launches)),
            "avg_launch_us": round(1e3 * ms / max(1, launches), 2),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}


def combined_traffic(roof):
    """Traffic per launch of several kernel classes together: the forms' values weighed by their launches
    (null unless every form that launched has one)."""
    forms = [f for f in roof["forms"].values() if f["launches"]]
    if forms and all(f["traffic"] is not None for f in forms):
        roof["traffic"] = round(sum(f["traffic"] * f["launches"] for f in forms) / sum(f["launches"] for f in forms))
    return roof


def tuned_cluster_leg(cd, g, tau, seed, stream, reps=5):
    """CLUSTER + quotient + estimate on a built CSR with the library's default knobs, then after
    cldiam_autotune_graph picked and cached knobs for this size class; same results required."""
    import torch
    cd.profile_set_timing([])

    def timed():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        r = None
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            r = cd.estimate(cd.quotient_build(cd.cluster(g, tau, seed)))
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    cd.tuning_cache_clear()
    timed()  # warm-up
    ms_def, r_def = timed()
    best = cd.autotune_graph(g, tau, seed, reps=2)
    ms_tuned, r_tuned = timed()
    cd.tuning_cache_clear()
    keys = ("pull_ratio", "relax_ctas_per_sm", "dense_quotient_k", "apsp_sources_per_cta", "apsp_fw_density")
    return {"default_ms": round(ms_def, 3), "tuned_ms": round(ms_tuned, 3),
            "knobs": {k: (round(best[k], 3) if isinstance(best[k], float) else best[k]) for k in keys},
            "identical": bool(r_def == r_tuned),
            "what": ("CLUSTER + quotient + estimate on the built CSR (CUDA events, mean of 5 runs) with the default "
                     "knobs, then with the knobs cldiam_autotune_graph picked and cached for this size class")}


def measure_workload(cd, name, steps, warmup, stream, dist, local, sampler=None, tune=False):
    """Time `steps` whole CL-DIAM passes (CSR build .. estimate) on one workload with its edge list resident
    in HBM; check the first pass against the oracle's stored result."""
    import torch

    from inputs.workloads import WORKLOADS
    wl = WORKLOADS[name]
    e = wl.make()
    with torch.cuda.stream(stream):
        src_d = torch.from_numpy(e.src.view(np.int32)).cuda()
        dst_d = torch.from_numpy(e.dst.view(np.int32)).cuda()
        w_d = torch.from_numpy(e.w.view(np.int32)).cuda()
    stream.synchronize()

    def step(mid_event=None):
        g = cd.build_csr(src_d, dst_d, w_d, e.n, lcc=True, stream=stream)
        if mid_event is not None:
            mid_event.record(stream)  # end of the CSR build (row a1) on the device timeline
        c = cd.cluster(g, wl.tau, wl.seed)
        q = cd.quotient_build(c)
        r = cd.estimate(q)
        return g, c, q, r

    # warm-up; the first pass is profiled per kernel class and checked against the oracle's stored result
    cd.profile_set_timing(cd.KERNEL_CLASSES)
    cd.profile_reset()
    g, c, q, r = step()
    prof_warm = cd.profile_get()
    n_lcc, nnz = g.n, g.nnz
    m_lcc = nnz // 2
    center, D, cid = c.copy()
    qoff, qcol, qw = q.copy()
    parity = "unchecked (no stored oracle result for this workload)"
    gold_path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.json")
    if os.path.exists(gold_path):
        gold = json.load(open(gold_path))
        ok = (gold["n"] == n_lcc and gold["nnz"] == nnz and gold["k"] == r["k"] and
              gold["phi_approx"] == r["phi_approx"] and gold["center_sha256"] == digest(center) and
              gold["D_sha256"] == digest(D) and gold["cid_sha256"] == digest(cid) and
              gold["quotient"]["col_sha256"] == digest(qcol) and gold["quotient"]["w_sha256"] == digest(qw) and
              all(gold["stats"][k] == r[k] for k in gold["stats"]))
        parity = ("bit-exact vs the CPU oracle's stored result (centers, D, cluster ids, quotient CSR, estimate)"
                  if ok else "MISMATCH vs the CPU oracle's stored result")
    del g, c, q, center, D, cid
    for _ in range(max(0, warmup - 1)):
        g, c, q, r2 = step()
        del g, c, q
        assert r2["phi_approx"] == r["phi_approx"]

    shares = {k: v["ms"] for k, v in prof_warm.items() if v["ms"] > 0}
    tot = sum(shares.values()) or 1.0
    dominant = max((k for k in shares if prof_warm[k]["bytes"] > 0), key=lambda k: shares[k])

    # timed region: the dominant class and both growing-step forms are bracketed by CUDA events
    cd.profile_set_timing(sorted({dominant, *RELAX_CLASSES}))
    cd.profile_reset()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev_mid = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev_end = [torch.cuda.Event(enable_timing=True) for _ in range(steps - 1)] + [ev1]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    for i in range(steps):
        g, c, q, r2 = step(ev_mid[i])
        del g, c, q
        ev_end[i].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / steps
    ms_csr = sum((ev0 if i == 0 else ev_end[i - 1]).elapsed_time(ev_mid[i]) for i in range(steps)) / steps
    ms_rest = sum(ev_mid[i].elapsed_time(ev_end[i]) for i in range(steps)) / steps
    prof = cd.profile_get()
    if dist:
        from paper_1506_03265_gb300.shard import max_over_ranks
        dev = torch.device("cuda", local)
        ms, ms_csr, ms_rest = (max_over_ranks(x, dist, dev) for x in (ms, ms_csr, ms_rest))
    ws = dist.get_world_size() if dist else 1
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    relax_ms = sum(prof[c]["ms"] for c in RELAX_CLASSES) / steps
    scanned = r["edges_scanned"]
    out = {
        "workload": name, "describe": wl.describe, "tau": wl.tau, "seed": wl.seed, "n_lcc": n_lcc, "m_lcc": m_lcc,
        "ms_per_step": round(ms, 3), "gteps": round(ws * m_lcc / (ms * 1e-3) / 1e9, 4),
        "result": {k: r[k] for k in ("k", "phi_gc", "radius", "phi_approx", "stages", "steps", "doublings",
                                     "delta_end", "node_updates", "edges_scanned", "quotient_edges")},
        "parity": parity,
        "step_split": {"csr_build_ms": round(ms_csr, 3), "cluster_quotient_estimate_ms": round(ms_rest, 3),
                       "gteps_excluding_csr_build": round(ws * m_lcc / (ms_rest * 1e-3) / 1e9, 4),
                       "what": "m_LCC / time of CLUSTER + quotient + estimate on a built CSR (the same timed steps)"},
        "roofline": roofline_of(prof, [dominant], peak, peaks, name),
        "relax_roofline": combined_traffic(dict(
            roofline_of(prof, list(RELAX_CLASSES), peak, peaks, name, tkey="relax_steps"),
            traffic_note=("per form below: DRAM bytes per algorithmic byte from one-kernel ncu captures on R-MAT 22 "
                          "(inputs above the L2 size, a few GB on the device), times this workload's algorithmic "
                          "bytes per launch; the combined value weighs the forms by their launches"),
            what=("both forms of the Delta-growing step (pushed relax and dense relax_pull) over the timed "
                  "steps: algorithmic bytes = 16 B per adjacency entry a launch reads + per-entry/row/changed-"
                  "node terms, as the library counts them per launch / CUDA-event time"),
            ms_per_step=round(relax_ms, 4),
            forms={c: {"launches": prof[c]["launches"], "ms": round(prof[c]["ms"] / steps, 4),
                       "gbs": round(prof[c]["bytes"] / (prof[c]["ms"] * 1e-3) / 1e9, 1) if prof[c]["ms"] else None,
                       "frac": round(prof[c]["bytes"] / (prof[c]["ms"] * 1e-3) / 1e9 / peak, 4) if prof[c]["ms"]
                       else None,
                       "alg_bytes_per_launch": round(prof[c]["bytes"] / max(1, prof[c]["launches"])),
                       "traffic": stored_traffic(name, c, prof[c]["bytes"] / max(1, prof[c]["launches"]))}
                   for c in RELAX_CLASSES},
            edges_scanned_per_step=scanned,
            scanned_16B_gbs=round(16.0 * scanned / (relax_ms * 1e-3) / 1e9, 1) if relax_ms else None,
            scanned_16B_frac=round(16.0 * scanned / (relax_ms * 1e-3) / 1e9 / peak, 4) if relax_ms else None,
            relax_gteps=round(scanned / (relax_ms * 1e-3) / 1e9, 3) if relax_ms else None)),
        "kernel_shares": {k: round(v / tot, 4) for k, v in sorted(shares.items(), key=lambda x: -x[1])},
        "kernel_ms_per_step": {k: round(v, 4) for k, v in sorted(shares.items(), key=lambda x: -x[1])},
        "gpu_launches": sum(v["launches"] for v in prof.values()),
        "tuned_cluster": None,
        "wall": (t_wall0, t_wall1),
        "in_bytes": 12 * e.m, "nnz": nnz,
    }
    if tune:
        g = cd.build_csr(src_d, dst_d, w_d, e.n, lcc=True, stream=stream)
        out["tuned_cluster"] = tuned_cluster_leg(cd, g, wl.tau, wl.seed, stream)
        del g
    return out, (e, src_d, dst_d, w_d, r)


def run_gpu(args):
    import torch

    import paper_1506_03265_gb300 as cd
    from inputs.workloads import WORKLOADS

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cd.load()
    if args.tuning:
        BASE_TUNING.update({k: float(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))})
        cd.tuning_set(**BASE_TUNING)
    stream = torch.cuda.Stream()
    wl = WORKLOADS[args.workload]

    sampler = ClockSampler(local)
    sampler.wait_first()
    head, (e, src_d, dst_d, w_d, r) = measure_workload(cd, args.workload, args.steps, args.warmup, stream, dist, local,
                                                       tune=not args.no_tuned_cluster)
    t_wall0, t_wall1 = head.pop("wall")
    clocks = sampler.summary(t_wall0, t_wall1)
    in_bytes = head.pop("in_bytes")
    nnz = head.pop("nnz")
    m_lcc = head["m_lcc"]
    ms = head["ms_per_step"]
    value = head["gteps"]
    launches = head["gpu_launches"]

    # end to end through the public API with pinned host buffers
    src_h = torch.from_numpy(e.src.view(np.int32)).pin_memory()
    dst_h = torch.from_numpy(e.dst.view(np.int32)).pin_memory()
    w_h = torch.from_numpy(e.w.view(np.int32)).pin_memory()
    cd.profile_set_timing([])
    cd.run(src_h, dst_h, w_h, e.n, wl.tau, wl.seed, stream=stream)
    torch.cuda.synchronize()
    # one call in flight: each step's host read, then its compute
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        re = cd.run(src_h, dst_h, w_h, e.n, wl.tau, wl.seed, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = e0.elapsed_time(e1) / args.e2e_steps
    assert re["phi_approx"] == r["phi_approx"]
    # two calls in flight (two host threads, two streams): one step's edge list crosses the host link while
    # the other step computes; every step still copies its inputs and reads its result inside the timed
    # region, which is wall clock between two device-wide synchronisations
    streams = [stream, torch.cuda.Stream()]
    per_thread = max(1, (args.e2e_steps + 1) // 2)
    outs, errs = [[], []], []

    def worker(j):
        try:
            for _ in range(per_thread):
                outs[j].append(cd.run(src_h, dst_h, w_h, e.n, wl.tau, wl.seed, stream=streams[j]))
        except Exception as ex:  # surfaced below
            errs.append(ex)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    threads = [threading.Thread(target=worker, args=(j,)) for j in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    ms_e2e = (time.perf_counter() - t0) * 1e3 / (2 * per_thread)
    if errs:
        raise errs[0]
    assert all(x == re for o in outs for x in o), "concurrent cldiam_run results differ"
    e2e = {"value": round(ws * m_lcc / (ms_e2e * 1e-3) / 1e9, 4), "unit": "GTEPS", "ms_per_step": round(ms_e2e, 3),
           "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": 88,
           "api": "cldiam_run (pinned host edge list in, cldiam_result out)",
           "in_flight": 2,
           "what": ("two cldiam_run calls in flight from two host threads on two streams, wall clock over "
                    f"{2 * per_thread} steps between device-wide synchronisations; results equal to the "
                    "one-call run"),
           "one_in_flight": {"value": round(ws * m_lcc / (ms_one * 1e-3) / 1e9, 4), "ms_per_step": round(ms_one, 3),
                             "what": "one call at a time on one stream, CUDA events"}}
    del src_h, dst_h, w_h

    # Delta-stepping baseline (Section 5) on the same graph
    g = cd.build_csr(src_d, dst_d, w_d, e.n, lcc=True, stream=stream)
    s = cd.sssp_source(g, wl.seed)
    cd.sssp_delta(g, s, want_dist=False)
    torch.cuda.synchronize()
    cd.profile_set_timing(["delta_stepping"])
    cd.profile_reset()
    reps = 5
    t_each = []
    for _ in range(reps):
        t0 = time.perf_counter()
        _, ecc, rounds = cd.sssp_delta(g, s, want_dist=False)
        t_each.append(time.perf_counter() - t0)
    t_ds = statistics.median(t_each)
    pds = cd.profile_get()["delta_stepping"]
    peaks = load_peaks()
    sssp = {"what": "Delta-stepping SSSP from the Philox source, 2*ecc = upper bound; wall clock of one call, "
                    "median of 5 (min and max beside it)",
            "ms": round(t_ds * 1e3, 3), "ms_min": round(min(t_each) * 1e3, 3), "ms_max": round(max(t_each) * 1e3, 3),
            "gteps": round(m_lcc / t_ds / 1e9, 4), "ecc": ecc,
            "upper_bound": 2 * ecc, "rounds": rounds,
            "roofline": roofline_of({"delta_stepping": pds}, ["delta_stepping"], peaks.get("hbm_gbs", 6800.0),
                                    peaks, args.workload)}
    cd.profile_set_timing([])
    cl2 = None
    if not args.no_cluster2:
        # CLUSTER2 (Algorithm 2) + quotient + estimate on the same CSR: the provable variant of Section 4
        r2 = cd.estimate(cd.quotient_build(cd.cluster2(g, wl.tau, wl.seed)))
        torch.cuda.synchronize()
        t_each = []
        for _ in range(3):
            t0 = time.perf_counter()
            r2 = cd.estimate(cd.quotient_build(cd.cluster2(g, wl.tau, wl.seed)))
            t_each.append(time.perf_counter() - t0)
        t_c2 = statistics.median(t_each)
        cl2 = {"what": "CLUSTER2 (Algorithm 2: CLUSTER for R_CL, then log2 n iterations of PartialGrowth2 / "
                       "Contract2) + quotient + estimate on the built CSR, wall clock, median of 3",
               "ms": round(t_c2 * 1e3, 3), "ms_min": round(min(t_each) * 1e3, 3),
               "gteps": round(m_lcc / t_c2 / 1e9, 4),
               "k": r2["k"], "radius": r2["radius"], "phi_gc": r2["phi_gc"], "phi_approx": r2["phi_approx"],
               "iterations": r2["stages"], "growth_rounds": r2["steps"], "r_cl": r2["delta_end"] // 2,
               "phi_approx_over_cluster": round(r2["phi_approx"] / r["phi_approx"], 4)}
    del g, src_d, dst_d, w_d, e
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "describe": head["describe"], "tau": head["tau"], "seed": head["seed"],
                   "n_lcc": head["n_lcc"], "m_lcc": m_lcc, "parallelism": f"replicas x{ws}",
                   "step": "CSR build + LCC + CLUSTER + quotient + estimate, edge list resident in HBM",
                   "l2": f"no flush: edge list {in_bytes / 1e6:.0f} MB and CSR {nnz * 12 / 1e6:.0f} MB exceed the 129 MB L2"},
        "result": head["result"],
        "parity": head["parity"],
        "step_split": head["step_split"],
        "e2e": e2e,
        "roofline": head["roofline"],
        "relax_roofline": head["relax_roofline"],
        "tuned_cluster": head["tuned_cluster"],
        "kernel_shares": head["kernel_shares"],
        "kernel_ms_per_step": head["kernel_ms_per_step"],
        "clocks": clocks,
        "gpu_launches": launches,
        "sssp_baseline": sssp,
    }
    if cl2:
        line["cluster2"] = cl2
    # the other single-graph workloads: same step, same checks, fewer steps
    if args.secondary:
        sec = {}
        for name in [x for x in args.secondary.split(",") if x and x != args.workload]:
            sm = ClockSampler(local)
            sm.wait_first()
            res, keep = measure_workload(cd, name, args.secondary_steps, args.warmup, stream, dist, local)
            del keep
            w0, w1 = res.pop("wall")
            res.pop("in_bytes"); res.pop("nnz")
            res["clocks"] = sm.summary(w0, w1)
            sm.stop()
            for k in ("kernel_shares", "tuned_cluster"):
                res.pop(k)
            sec[name] = res
            torch.cuda.empty_cache()
        line["secondary_workloads"] = sec
    if not args.no_delta0_experiment and rank == 0:
        line["initial_delta_experiment"] = delta0_leg(cd)
    if not args.no_batched:
        mix = build_mix_arena(cd, stream, args.batched_count, budget=150 * 10**9, rank=rank, world=ws)
        line["batched"] = batched_leg(cd, stream, mix, args.plain_sample_every, dist=dist)
        if not args.no_served and ws == 1:
            # the serving leg runs on a single GPU: its query stream is one queue
            line["served"] = served_leg(cd, mix, [int(x) for x in args.serve_rates.split(",")])
        mix[0].free()
    sampler.stop()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def profile_pass(args):
    """One CL-DIAM pass (CSR build .. estimate) on the workload, nothing else: the ncu capture target."""
    import torch

    import paper_1506_03265_gb300 as cd
    from inputs.workloads import WORKLOADS
    wl = WORKLOADS[args.workload]
    e = wl.make()
    ts = [torch.from_numpy(a.view(np.int32)).cuda() for a in (e.src, e.dst, e.w)]
    cd.profile_reset()
    g = cd.build_csr(ts[0], ts[1], ts[2], e.n, lcc=True)
    r = cd.estimate(cd.quotient_build(cd.cluster(g, wl.tau, wl.seed)))
    # launches and algorithmic bytes per kernel class of this pass: the denominators of the DRAM captures
    prof = {c: {"launches": v["launches"], "bytes": v["bytes"]} for c, v in cd.profile_get().items() if v["launches"]}
    print(json.dumps({"workload": args.workload, "k": r["k"], "phi_approx": r["phi_approx"], "m": int(e.src.size),
                      "nnz_lcc": g.nnz, "n_lcc": g.n, "classes": prof}))


def profile_other(args):
    """One Delta-stepping SSSP, one CLUSTER2 pass or one many-graph batch, nothing else: ncu capture targets."""
    import torch

    import paper_1506_03265_gb300 as cd
    from inputs.workloads import WORKLOADS
    if args.profile_apsp:
        k = args.profile_apsp
        rng = np.random.default_rng(k)
        iu = np.triu_indices(k, 1)
        keep = rng.random(iu[0].size) < 0.5
        s_, d_ = iu[0][keep].astype(np.uint32), iu[1][keep].astype(np.uint32)
        w_ = rng.integers(1, 1 << 20, s_.size).astype(np.uint32)
        g = cd.build_csr(s_, d_, w_, k, lcc=False)
        off, col, w, _ = g.copy()
        print(json.dumps({"k": k, "nnz": int(off[-1]), "phi": cd.apsp_max(k, off, col, w)}))
        return
    if args.profile_batch:
        mix = build_mix_arena(cd, None, args.profile_batch)
        arena, ids, taus, seeds, edges, _ = mix
        res, st = arena.run(ids, taus, seeds)
        torch.cuda.synchronize()
        print(json.dumps({"batch": len(ids), "undirected_edges": edges, "ok": all(x == 0 for x in st)}))
        return
    wl = WORKLOADS[args.workload]
    e = wl.make()
    ts = [torch.from_numpy(a.view(np.int32)).cuda() for a in (e.src, e.dst, e.w)]
    g = cd.build_csr(ts[0], ts[1], ts[2], e.n, lcc=True)
    if args.profile_sssp:
        src = cd.sssp_source(g, wl.seed)
        _, ecc, rounds, scanned = cd.sssp_delta(g, src, want_dist=False, with_scanned=True)
        print(json.dumps({"workload": args.workload, "ecc": ecc, "rounds": rounds, "edges_scanned": scanned}))
    else:
        r = cd.estimate(cd.quotient_build(cd.cluster2(g, wl.tau, wl.seed)))
        print(json.dumps({"workload": args.workload, "k": r["k"], "phi_approx": r["phi_approx"]}))


def main():
    args = parse()
    if args.profile_pass:
        profile_pass(args)
    elif args.profile_sssp or args.profile_cluster2 or args.profile_batch or args.profile_apsp:
        profile_other(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
