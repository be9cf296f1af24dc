"""Write expected CL-DIAM results for the named workloads from the CPU oracle only.

    python tests/golden/make_golden.py rmat20 grid64

Each tests/golden/<workload>_oracle.json holds the oracle's CSR size, cluster
counters, estimate and SHA-256 digests of its per-node arrays (center as
uint32, D as uint32, cid as uint32) and of the quotient CSR, so full-size GPU
runs can be checked bit-exactly without rerunning the oracle.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402
from inputs.workloads import WORKLOADS  # noqa: E402


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def expected(name: str) -> dict:
    wl = WORKLOADS[name]
    e = wl.make()
    t0 = time.time()
    g = oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=True)
    d0 = oracle.delta0(g)
    cl = oracle.cluster(g, wl.tau, wl.seed, d0)
    q = oracle.quotient(g, cl)
    res = oracle.estimate(q, cl)
    s = oracle.sssp_source(wl.seed, g.n)
    dist = oracle.dijkstra(g, s)
    assert int(cl.D.max()) < 0xFFFFFFFF and int(q.w.max(initial=0)) < 0xFFFFFFFF
    st = cl.stats
    return {
        "workload": name,
        "describe": wl.describe,
        "tau": wl.tau,
        "seed": wl.seed,
        "n": g.n,
        "nnz": g.nnz,
        "delta0": d0,
        "csr_sha256": {"off": digest(g.off), "col": digest(g.col), "w": digest(g.wt)},
        "k": res.k,
        "phi_gc": res.phi_gc,
        "radius": res.radius,
        "phi_approx": res.phi_approx,
        "stats": {f: int(st[f]) for f in ("stages", "steps", "doublings", "delta_end", "guard_exits",
                                          "node_updates", "centers_drawn")},
        "center_sha256": digest(cl.center.astype(np.uint32)),
        "D_sha256": digest(cl.D.astype(np.uint32)),
        "cid_sha256": digest(q.cid.astype(np.uint32)),
        "quotient": {"nnz": int(q.col.size), "off_sha256": digest(q.off.astype(np.uint64)),
                     "col_sha256": digest(q.col.astype(np.uint32)), "w_sha256": digest(q.w.astype(np.uint32))},
        "sssp": {"source": s, "ecc": int(dist[dist != oracle.UNREACHABLE].max()),
                 "dist_sha256": digest(np.where(dist == oracle.UNREACHABLE, 0xFFFFFFFF, dist).astype(np.uint32))},
        "oracle_seconds": round(time.time() - t0, 1),
        "written_by": "tests/golden/make_golden.py (CPU oracle only)",
    }


if __name__ == "__main__":
    for name in sys.argv[1:] or ["grid64", "rmat20"]:
        out = expected(name)
        path = os.path.join(HERE, f"{name}_oracle.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(path, out["k"], out["phi_approx"], out["oracle_seconds"], "s")
