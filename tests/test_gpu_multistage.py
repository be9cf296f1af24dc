"""The GPU path on the hand-worked multi-stage examples of tests/golden/multistage_pins.json
(Algorithm 1 with Procedure Contract; derivations in tests/test_oracle_multistage.py), with the
growing steps in the pushed and in the dense pull form.  Integers: bit-exact."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "multistage_pins.json")))["cases"]


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    yield m
    m.tuning_set()


@pytest.mark.parametrize("ratio", [-1.0, 1e-9])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_gpu_matches_hand_derivation(cd, case, ratio):
    cd.tuning_set(pull_ratio=ratio)
    n = case["n"]
    s = np.arange(n - 1, dtype=np.uint32)
    g = cd.build_csr(s, s + 1, np.ones(n - 1, np.uint32), n)
    kw = {} if case["delta0"] is None else {"delta0_mode": cd.DELTA0_EXPLICIT, "delta0": case["delta0"]}
    c = cd.cluster(g, case["tau"], case["seed"], contract_mode=case["contract_mode"], **kw)
    center, D, cid = c.copy()
    assert center.tolist() == case["center"] and D.tolist() == case["D"]
    info = c.info()
    for k, v in case["stats"].items():
        assert info[k] == v, k
    q = cd.quotient_build(c)
    qoff, qcol, qw = q.copy()
    qq = case["quotient"]
    assert cid.tolist() == qq["cid"] and qoff.tolist() == qq["off"]
    assert qcol.tolist() == qq["col"] and qw.tolist() == qq["w"]
    r = cd.estimate(q)
    assert (r["k"], r["phi_gc"], r["radius"], r["phi_approx"]) == (qq["k"], case["phi_gc"], case["radius"],
                                                                    case["phi_approx"])
