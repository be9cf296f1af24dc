"""Multi-stage CLUSTER pinned to hand-worked examples (Algorithm 1 with Procedure Contract, Section 3).

The expected arrays in tests/golden/multistage_pins.json were derived by hand on unit-weight paths
0 - 1 - ... - (n-1), as written out below; only the seeds were found by a search (so that the
Philox draws of Algorithm 1 pick the listed centers, which the test re-checks).  The cases pin the
bound of a node reached in a later stage through a contracted cluster, D_v = d_v + R_prev[c_v], where
R_prev[c] is the largest D of cluster c before the stage: reading R after the stage's own updates,
adding it twice or dropping it gives different D arrays.

two_stage_reset (n = 10, tau = 0.15, seed 6, Delta0 = average weight = 1; L = log2 10, 8 tau L = 3.99):
  stage 1, U = {0..9}: draws {2}; key(2) = (0, 2).
    step 1 (Delta 1): relaxer 2 (d 0 < 1) gives 1 and 3 the key (1, 2); covered 3, 2*3 < 10.
    step 2: the changed nodes have d = 1 = Delta, so nothing relaxes; no update, coverage under half.
    Delta doubles to 2 (a covered node touches an uncovered one); relaxers 1, 2, 3 (d < 2).
    step 3: 0 and 4 get (2, 2); covered 5, 2*5 >= 10: stop.
    finalize: 0..4 join cluster 2 with D = d + R_prev[2] = d + 0 = 2 1 0 1 2; R[2] = 2.
  stage 2, U = {5..9} (5 >= 3.99): draws {8}.
    step 4 (Delta 2): contracted node 4 relaxes as (0, 2): 5 gets (1, 2); center 8 gives 7 and 9 (1, 8);
    covered 4, 2*4 >= 5: stop.
    finalize: D_5 = 1 + R_prev[2] = 3, D_7 = D_9 = 1 + R_prev[8] = 1, D_8 = 0; R[2] = 3, R[8] = 1.
  stage 3: U = {6}, 1 < 3.99: the loop ends; 6 becomes a singleton (D 0).
  counters: 2 stages, 4 steps, 1 doubling, Delta_end 2, updates 2 + 0 + 2 + 3 = 7, 2 centers drawn.
  quotient (cluster ids by center id: 2 -> 0, 6 -> 1, 8 -> 2): edge (5,6) gives D_5 + 1 + D_6 = 4 between
  0 and 1, edge (6,7) gives 0 + 1 + 1 = 2 between 1 and 2; Phi(G_C) = 6, R = 3, Phi_approx = 6 + 2*3 = 12.

three_stage_reset (n = 14, tau = 0.09, seed 144868, Delta0 = 2 given; 8 tau L = 2.74):
  stage 1, U = {0..13}: draws {1, 4}.
    step 1: 0, 2 get (1, 1); 3, 5 get (1, 4); covered 6, 12 < 14.
    step 2: from 2, 3 would get (2, 1) > (1, 4): no; from 5, 6 gets (2, 4); covered 7, 14 >= 14: stop.
    finalize: D = 1 0 1 | 1 0 1 2 for nodes 0..6 (centers 1 and 4); R[1] = 1, R[4] = 2.
  stage 2, U = {7..13}: draws {11}.
    step 3: contracted 6 (cluster 4) gives 7 the key (1, 4); 11 gives 10 and 12 (1, 11); covered 4 >= 7/2.
    finalize: D_7 = 1 + R_prev[4] = 3; D_10 = D_12 = 1; R[4] = 3, R[11] = 1.
  stage 3, U = {8, 9, 13} (3 >= 2.74): draws {13}.
    step 4: contracted 7 (cluster 4) gives 8 (1, 4); contracted 10 (cluster 11) gives 9 (1, 11); covered 3.
    finalize: D_8 = 1 + R_prev[4] = 1 + 3 = 4 (R of cluster 4 grown in stage 2), D_9 = 1 + R_prev[11] = 2.
  counters: 3 stages, 4 steps, no doubling, updates 4 + 1 + 3 + 2 = 10, 4 centers drawn.
  quotient (1 -> 0, 4 -> 1, 11 -> 2, 13 -> 3): (2,3) 1+1+1 = 3, (8,9) 4+1+2 = 7, (12,13) 1+1+0 = 2;
  Phi(G_C) = 12, R = 4, Phi_approx = 20 (the path's diameter is 13).

three_stage_cumulative (the same graph, seed and Delta0; contracted nodes relax with their own D while
D < Delta, and D_v = d_v):
  stage 1 as above (D = 1 0 1 1 0 1 2).
  stage 2, U = {7..13}: draws {11}.  Node 6 has D = 2 = Delta, so it does not relax: 7 gets nothing.
    step 3: 11 gives 10, 12 (1, 11); covered 3 < 7/2.  step 4: 10 and 12 (d 1 < 2) give 9 and 13 (2, 11);
    covered 5: stop.  D = d: 9 -> 2, 10 -> 1, 11 -> 0, 12 -> 1, 13 -> 2.
  stage 3: U = {7, 8}, 2 < 2.74: the loop ends; 7 and 8 are singletons.
  counters: 2 stages, 4 steps, updates 4 + 1 + 2 + 2 = 9, 3 centers drawn.
  quotient (1, 4, 7, 8, 11 -> 0..4): (2,3) 3, (6,7) 2+1+0 = 3, (7,8) 1, (8,9) 0+1+2 = 3;
  Phi(G_C) = 10, R = 2, Phi_approx = 14.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "multistage_pins.json")))["cases"]
GAMMA = 4 * math.log(2)  # Algorithm 1
UNFROZEN = {  # U at the start of each stage that draws, from the derivations above
    "two_stage_reset": [range(10), range(5, 10)],
    "three_stage_reset": [range(14), range(7, 14), [8, 9, 13]],
    "three_stage_cumulative": [range(14), range(7, 14)],
}


def path(n):
    s = np.arange(n - 1, dtype=np.uint32)
    return s, s + 1, np.ones(n - 1, np.uint32)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_draws_are_the_assumed_centers(case):
    n, tau, seed = case["n"], case["tau"], case["seed"]
    L = math.log2(n)
    for stage, (U, want) in enumerate(zip(UNFROZEN[case["name"]], case["draws"]), 1):
        p = GAMMA * tau * L / len(U)
        thr = 1 << 32 if p >= 1 else int(math.floor(p * 4294967296.0))
        got = [v for v in U if int(oracle.philox4x32_10(seed, [v, stage, 0, 0])[0]) < thr]
        assert got == want, (stage, got, want)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_oracle_matches_hand_derivation(case):
    n = case["n"]
    g = oracle.build_csr(n, *path(n), lcc=True)
    d0 = oracle.delta0(g) if case["delta0"] is None else case["delta0"]
    cl = oracle.cluster(g, case["tau"], case["seed"], d0, contract_mode=case["contract_mode"])
    assert cl.center.tolist() == case["center"]
    assert cl.D.tolist() == case["D"]
    for k, v in case["stats"].items():
        assert cl.stats[k] == v, k
    q = oracle.quotient(g, cl)
    qq = case["quotient"]
    assert q.k == qq["k"] and q.cid.tolist() == qq["cid"]
    assert q.off.tolist() == qq["off"] and q.col.tolist() == qq["col"] and q.w.tolist() == qq["w"]
    r = oracle.estimate(q, cl)
    assert (r.phi_gc, r.radius, r.phi_approx) == (case["phi_gc"], case["radius"], case["phi_approx"])
