"""The benchmark's algorithmic byte counts (host logic, no GPU).

Each level-0 kernel's count is the compulsory DRAM traffic of one launch:
every array once. The checks restate the counts for the 128^3 system from
the kernels' reads and writes and check how the shared offset patterns
change them: a slice kept with a pattern costs its values only, plus the
pattern (one index per entry column) and one flag per slice.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_for_tests", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


N0, NNZ0, STORED0, N1 = 2_097_152, 55_321_580, 55_611_136, 520_192
SPTR = 4 * (N0 // 32 + 1)


def test_plain_layout_counts(bench):
    ab = bench.algorithmic_bytes
    # float32 down sweep: value + int16 column per entry; xpre, b, p read, t written
    assert ab("down0", "fcg32", N0, NNZ0, N1, 2) == NNZ0 * 6 + N0 * 16 + SPTR
    # float64 q = A p: value + column; p read, q written
    assert ab("spmv", "fcg32", N0, NNZ0, N1, 2) == NNZ0 * 10 + N0 * 16 + SPTR
    # the post sweep in FCG(1): b, dinv (float32), z written, r and q_old read (float64)
    assert ab("post0", "fcg32", N0, NNZ0, N1, 2) == NNZ0 * 6 + N0 * (2 * 4 + 8) + SPTR + N0 * 16
    # vector kernels do not depend on the layout
    assert ab("update", "fcg32", N0, NNZ0, N1, 2) == N0 * 60
    assert ab("axpy", "pcg64", N0, NNZ0, N1, 2) == N0 * 24


def test_pattern_layout_counts(bench):
    ab = bench.algorithmic_bytes
    full = ab("down0", "fcg32", N0, NNZ0, N1, 2, stored=STORED0, pat_entries=STORED0)
    # every slice with a pattern: values, the pattern (2 bytes per 32 entries) and a flag per slice
    want = NNZ0 * 4 + 2 * (STORED0 / 32 + (N0 + 31) // 32) + N0 * 16 + SPTR
    assert full == pytest.approx(want)
    plain = ab("down0", "fcg32", N0, NNZ0, N1, 2)
    assert plain - full == pytest.approx(NNZ0 * 2 - 2 * (STORED0 / 32 + (N0 + 31) // 32))
    # fewer pattern entries, more bytes; none at all is the plain count
    half = ab("down0", "fcg32", N0, NNZ0, N1, 2, stored=STORED0, pat_entries=STORED0 // 2)
    assert full < half < plain
    assert ab("down0", "fcg32", N0, NNZ0, N1, 2, stored=STORED0, pat_entries=0) == plain
    # the float64 product saves the same index bytes
    s_plain = ab("spmv", "fcg32", N0, NNZ0, N1, 2)
    s_pat = ab("spmv", "fcg32", N0, NNZ0, N1, 2, stored=STORED0, pat_entries=STORED0)
    assert s_plain - s_pat == pytest.approx(plain - full)
    # the true residual reads the columns entry by entry whatever the layout
    assert ab("residual", "fcg32", N0, NNZ0, N1, 2, stored=STORED0, pat_entries=STORED0) == \
        ab("residual", "fcg32", N0, NNZ0, N1, 2)


def test_the_headline_figures(bench):
    """The counts quoted for the 128^3 system: 258.7 MB (down), 292.3 MB (post)
    and 480.0 MB (q = A p) with 55,608,736 of 55,611,136 entries in pattern
    slices."""
    ab = bench.algorithmic_bytes
    kw = dict(stored=STORED0, pat_entries=55_608_736)
    assert ab("down0", "fcg32", N0, NNZ0, N1, 2, **kw) / 1e6 == pytest.approx(258.7, abs=0.05)
    assert ab("post0", "fcg32", N0, NNZ0, N1, 2, **kw) / 1e6 == pytest.approx(292.3, abs=0.05)
    assert ab("spmv", "fcg32", N0, NNZ0, N1, 2, **kw) / 1e6 == pytest.approx(480.0, abs=0.05)
