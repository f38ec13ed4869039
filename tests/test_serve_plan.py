"""Engine planning of the serving runtime (amg_serve_plan): a host-only
function, called here without a device.

The rule: in mesh order, a mesh is admitted with one engine when its resident
hierarchy plus one engine still fit in the budget; then engines go one at a
time to the admitted mesh with the largest load / engines (ties to the lowest
index) that still fits and has fewer than max_engines. The cases below check
the rule's consequences directly (budget never exceeded, admission order,
the cap, the load split) and against a plain restatement on random inputs.
"""
import numpy as np

from paper_2210_16660_gb300 import binding as B


def _plan(res, eb, budget, cap, loads=None):
    st, eng, tot = B.serve_plan(res, eb, budget, cap, loads=loads)
    return st, list(eng), tot


def _restated(res, eb, budget, cap, loads):
    m = len(res)
    eng = [0] * m
    used = 0
    for i in range(m):
        if used + res[i] + eb[i] <= budget:
            used += res[i] + eb[i]
            eng[i] = 1
    while True:
        cand = [i for i in range(m) if 1 <= eng[i] < cap and used + eb[i] <= budget]
        if not cand:
            break
        best = max(cand, key=lambda i: (loads[i] / eng[i], -i))
        eng[best] += 1
        used += eb[best]
    return eng, used


def test_everything_fits():
    st, eng, tot = _plan([100, 200, 300], [10, 20, 30], 10 ** 9, 3)
    assert st == B.OK and eng == [3, 3, 3] and tot == 600 + 3 * 60


def test_admission_in_mesh_order_and_refusal():
    # mesh 1 does not fit after mesh 0; mesh 2 still does
    st, eng, tot = _plan([100, 500, 50], [10, 10, 10], 200, 1)
    assert st == B.OK and eng == [1, 0, 1] and tot == 170


def test_nothing_fits_is_oom():
    st, eng, tot = _plan([100], [10], 109, 4)
    assert st == B.ERR_OOM and eng == [0] and tot == 0
    assert "budget" in B.last_error()


def test_budget_boundary_is_inclusive():
    st, eng, tot = _plan([100], [10], 110, 4)
    assert st == B.OK and eng == [1] and tot == 110
    st, eng, tot = _plan([100], [10], 140, 4)
    assert eng == [4] and tot == 140


def test_extra_engines_follow_the_load():
    # equal costs; load 3:1 -> the heavy mesh gets engines first, up to the cap
    st, eng, _ = _plan([0, 0], [10, 10], 60, 8, loads=[3.0, 1.0])
    assert eng == [4, 2]
    st, eng, _ = _plan([0, 0], [10, 10], 60, 3, loads=[3.0, 1.0])
    assert eng == [3, 3]


def test_ties_go_to_the_lowest_index():
    st, eng, _ = _plan([0, 0, 0], [10, 10, 10], 40, 4)
    assert eng == [2, 1, 1]


def test_bad_arguments():
    st, _, _ = _plan([], [], 10, 1)
    assert st == B.ERR_ARG
    st, _, _ = _plan([1], [1], 10, 0)
    assert st == B.ERR_ARG


def test_random_cases_match_the_rule():
    rng = np.random.default_rng(7)
    for _ in range(300):
        m = int(rng.integers(1, 6))
        res = [int(v) for v in rng.integers(0, 1000, m)]
        eb = [int(v) for v in rng.integers(1, 400, m)]
        loads = [float(v) for v in rng.integers(1, 5, m)]
        budget = int(rng.integers(0, 5000))
        cap = int(rng.integers(1, 5))
        st, eng, tot = _plan(res, eb, budget, cap, loads)
        want, used = _restated(res, eb, budget, cap, loads)
        assert eng == want
        if any(want):
            assert st == B.OK and tot == used <= budget
        else:
            assert st == B.ERR_OOM
