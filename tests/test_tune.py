"""The autotuner's host logic (no GPU): the coordinate-descent search over the knobs' candidate
lists driven by a synthetic cost, its result-invariance check, and the tuning cache (which knob a
call uses: process-wide setting, else the cached choice for its device and size class, else the
default; save / load).  The GPU tuners run the same search on real work (tests/test_gpu_tune.py)."""
import os

import pytest

import paper_1506_03265_gb300 as cd

CANDIDATES = {  # the library's fixed candidate lists, restated for the synthetic costs below
    "pull_ratio": [-1.0, 0.15, 0.3, 0.5, 0.8],
    "relax_ctas_per_sm": [0, 2, 4],
    "dense_quotient_k": [1024, 4096, 8192],
    "apsp_sources_per_cta": [0, 1, 4, 8],
    "apsp_fw_density": [4, 8, 16],
    "batch_fw_k": [64, 128, 200],
    "sssp_delta_scale": [1, 2, 4, 8],
    "batch_split": [1, 2],
}
DEFAULTS = {"pull_ratio": 0.3, "relax_ctas_per_sm": 0, "dense_quotient_k": 4096, "apsp_sources_per_cta": 0,
            "apsp_fw_density": 8, "batch_fw_k": 200, "sssp_delta_scale": 1.0,
            "batch_split": 2}


@pytest.fixture(autouse=True)
def clean():
    cd.load()
    cd.tuning_set()
    cd.tuning_cache_clear()
    yield
    cd.tuning_set()
    cd.tuning_cache_clear()


def close(a, b):
    return abs(float(a) - float(b)) < 1e-6


def test_size_class():
    assert [cd.size_class(x) for x in (0, 1, 2, 3, 4, 1023, 1024, 520_758_400)] == [0, 0, 1, 1, 2, 9, 10, 28]


def test_search_finds_the_separable_optimum():
    # cost = sum of independent per-knob terms: coordinate descent reaches the grid minimum
    best_of = {"pull_ratio": 0.5, "relax_ctas_per_sm": 4, "apsp_fw_density": 16}
    calls = []

    def measure(k):
        calls.append(k)
        cost = 1.0
        for name, want in best_of.items():
            cost += 0.0 if close(k[name], want) else 0.5 + 0.1 * CANDIDATES[name].index(
                min(CANDIDATES[name], key=lambda v: abs(v - k[name])))
        return cost, 42

    best, sec = cd.autotune_search(measure, list(best_of))
    for name, want in best_of.items():
        assert close(best[name], want), (name, best)
    for name in set(DEFAULTS) - set(best_of):  # knobs outside the mask keep their (default) value
        assert close(best[name], DEFAULTS[name])
    assert close(sec, 1.0)
    # the start point, then every other candidate of each searched knob once
    assert len(calls) == 1 + sum(len(CANDIDATES[k]) - 1 for k in best_of)


def test_search_keeps_the_start_without_a_two_percent_gain():
    def measure(k):
        return (0.99 if close(k["batch_fw_k"], 64) else 1.0), 7  # 1 % faster only: not taken

    best, _ = cd.autotune_search(measure, ["batch_fw_k"])
    assert best["batch_fw_k"] == 200
    best, _ = cd.autotune_search(lambda k: ((0.97 if close(k["batch_fw_k"], 64) else 1.0), 7), ["batch_fw_k"])
    assert best["batch_fw_k"] == 64


def test_search_starts_from_the_given_knobs():
    best, _ = cd.autotune_search(lambda k: (1.0, 1), ["sssp_delta_scale"], start={"apsp_fw_density": 16,
                                                                                    "sssp_delta_scale": 4})
    assert best["apsp_fw_density"] == 16 and close(best["sssp_delta_scale"], 4)


def test_search_refuses_a_knob_that_changes_the_result():
    def measure(k):
        return 1.0, (1 if close(k["pull_ratio"], 0.3) else 2)

    with pytest.raises(cd.CldiamError) as ei:
        cd.autotune_search(measure, ["pull_ratio"])
    assert ei.value.status == -8  # DIVERGED


def test_search_skips_candidates_that_fail():
    def measure(k):
        if k["dense_quotient_k"] == 1024:
            raise RuntimeError("out of memory")
        return (0.5 if k["dense_quotient_k"] == 8192 else 1.0), 3

    best, sec = cd.autotune_search(measure, ["dense_quotient_k"])
    assert best["dense_quotient_k"] == 8192 and close(sec, 0.5)


def test_search_argument_checks():
    with pytest.raises(cd.CldiamError):
        cd.autotune_search(lambda k: (1.0, 0), [])  # empty mask
    with pytest.raises(cd.CldiamError):
        cd.autotune_search(lambda k: (1.0, 0), ["batch_fw_k"], start={"batch_fw_k": 300})  # out of range


def test_effective_knobs_process_wide_then_cache_then_default():
    assert cd.tuning_effective(0, 20) == pytest.approx(DEFAULTS)
    cd.tuning_cache_put(0, 20, pull_ratio=0.8, apsp_sources_per_cta=4)
    eff = cd.tuning_effective(0, 20)
    assert close(eff["pull_ratio"], 0.8) and eff["apsp_sources_per_cta"] == 4 and eff["dense_quotient_k"] == 4096
    assert cd.tuning_effective(0, 21) == pytest.approx(DEFAULTS)  # other size class
    assert cd.tuning_effective(1, 20) == pytest.approx(DEFAULTS)  # other device
    cd.tuning_set(pull_ratio=-1.0)  # an explicit process-wide value wins over the cache
    eff = cd.tuning_effective(0, 20)
    assert eff["pull_ratio"] < 0 and eff["apsp_sources_per_cta"] == 4
    assert cd.tuning_cache_get(0, 20)["apsp_sources_per_cta"] == 4
    with pytest.raises(cd.CldiamError):
        cd.tuning_cache_get(0, 5)


def test_cache_save_and_load(tmp_path):
    cd.tuning_cache_put(0, 24, pull_ratio=0.5, relax_ctas_per_sm=4)
    cd.tuning_cache_put(0, 64 + 27, batch_fw_k=128)
    path = str(tmp_path / "tuning.txt")
    cd.tuning_cache_save(path)
    cd.tuning_cache_clear()
    with pytest.raises(cd.CldiamError):
        cd.tuning_cache_get(0, 24)
    cd.tuning_cache_load(path)
    a = cd.tuning_cache_get(0, 24)
    assert close(a["pull_ratio"], 0.5) and a["relax_ctas_per_sm"] == 4 and a["batch_fw_k"] == 0
    assert cd.tuning_cache_get(0, 91)["batch_fw_k"] == 128
    bad = str(tmp_path / "bad.txt")
    with open(bad, "w") as f:
        f.write("0 3 0.5 1\n")
    with pytest.raises(cd.CldiamError):
        cd.tuning_cache_load(bad)
    with open(bad, "w") as f:
        f.write("0 3 0.5 0 4096 3 8 200 1 2\n")  # apsp_sources_per_cta = 3 is out of range
    with pytest.raises(cd.CldiamError):
        cd.tuning_cache_load(bad)
    with pytest.raises(cd.CldiamError):
        cd.tuning_cache_load(os.path.join(str(tmp_path), "missing.txt"))


@pytest.mark.parametrize("knobs", [{"relax_ctas_per_sm": 65}, {"dense_quotient_k": 70000},
                                   {"apsp_sources_per_cta": 2}, {"batch_fw_k": 201},
                                   {"sssp_delta_scale": 0.5}, {"pull_ratio": float("nan")},
                                   {"batch_split": 3}])
def test_tuning_set_rejects_out_of_range(knobs):
    with pytest.raises(cd.CldiamError) as ei:
        cd.tuning_set(**knobs)
    assert ei.value.status == -1
    assert cd.tuning_get() == pytest.approx(DEFAULTS)
