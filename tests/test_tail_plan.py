"""Host check of the shared-memory cluster tail's planner (``csrc/tail_plan.h``).

``tail_plan_check.cpp`` builds the per-CTA layout and static blob with
``build_plan`` for 16, 8 and 5 CTAs, emulates every phase of the tail kernel on
per-CTA byte arrays (reads of rows another CTA owns go through the packed
owner/row references) and requires the entry level's x to equal, bit for bit,
the same V-cycle computed level by level, in float32 and float64. It runs under
AddressSanitizer/UBSan where the compiler provides them, so an out-of-range
offset in the layout fails the test. The levels come from the oracle's
hierarchy (inputs only).
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2210_16660_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tail_plan_check.cpp")
SMALL_ROWS = 12000   # levels the tail may hold (kSmallRows-sized levels)


def _write(path, h):
    L = h.nlevels - 1
    F = next(l for l in range(1, L) if h.level_size(l)[0] <= SMALL_ROWS)
    with open(path, "wb") as f:
        f.write(struct.pack("ii", F, L))
        for l in range(F, L + 1):
            lv = h.level(l)
            f.write(struct.pack("i", lv["n"]))
            for a, dt in ((lv["row_ptr"], np.int32), (lv["col"], np.int32), (lv["val"], np.float64),
                          (lv["dinv"], np.float64)):
                a = np.ascontiguousarray(a, dt)
                f.write(struct.pack("q", a.size) + a.tobytes())
            if l < L:
                agg, p = h.level_agg(l)
                nc = h.level_size(l + 1)[0]
                keep = agg >= 0
                rptr = np.zeros(nc + 1, np.int64)
                np.add.at(rptr, agg[keep] + 1, 1)
                rptr = np.cumsum(rptr).astype(np.int32)
                order = np.argsort(np.where(keep, agg, nc), kind="stable")
                ridx = order[keep[order]].astype(np.int32)      # members in increasing index
                for a, dt in ((agg, np.int32), (p, np.float64), (rptr, np.int32), (ridx, np.int32)):
                    a = np.ascontiguousarray(a, dt)
                    f.write(struct.pack("q", a.size) + a.tobytes())
        last = h.level(L)
        aL = W.CSR(last["n"], last["row_ptr"], last["col"], last["val"]).to_dense()
        f.write(np.ascontiguousarray(np.linalg.inv(aL), np.float64).tobytes())
    return F, L


def _compile(tmp):
    exe = os.path.join(tmp, "tail_plan_check")
    base = ["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-o", exe, SRC]
    try:
        subprocess.run(base + ["-fsanitize=address,undefined", "-fno-omit-frame-pointer"], check=True,
                       capture_output=True, timeout=300)
        probe = subprocess.run([exe], capture_output=True, timeout=60)   # no argument: returns 2 at once
        if probe.returncode == 2:
            return exe
    except (subprocess.CalledProcessError, subprocess.TimeoutExpired):
        pass
    subprocess.run(base, check=True, capture_output=True, timeout=300)
    return exe


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    return _compile(str(tmp_path_factory.mktemp("tailplan")))


@pytest.mark.parametrize("N,ratio", [(20, 1.04), (32, 1.0), (36, 1.04)])
def test_tail_plan_layout_and_kernel_indexing(checker, tmp_path, N, ratio):
    A = W.make_problem(N, ratio, seed=3).A
    h = O.Hierarchy(A, coarse_max=200, n_pass=2)
    assert h.nlevels >= 3
    path = str(tmp_path / "levels.bin")
    F, L = _write(path, h)
    assert L - F >= 1
    out = subprocess.run([checker, path], capture_output=True, text=True, timeout=600)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("T=")]
    assert out.returncode == 0, out.stdout + out.stderr
    assert len(lines) == 6 and all("mismatches=0 bad_refs=0" in ln for ln in lines), out.stdout
