"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#", "return")):
                names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("amg_setup", "pcg_solve", "amg_destroy", "amg_last_error", "amg_info"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2210_16660_gb300 import binding, build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in sorted(_declared()):
        assert hasattr(lib, name), f"{name} not exported"
    assert set(binding.EXPORTS) == _declared()
    # pure host functions are callable without a device
    lib2 = binding.load()
    p = binding.AmgParams()
    lib2.amg_default_params(ctypes.byref(p))
    assert (p.coarse_max, p.n_pass, p.max_levels, p.mode) == (200, 2, 30, 0)
    assert lib2.amg_last_error() == b""


def test_sources_target_sm103a_only():
    from paper_2210_16660_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_bad_arguments_are_rejected_on_the_host():
    from paper_2210_16660_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.amg_setup(None, None, None, ctypes.byref(h)) == binding.ERR_ARG
    assert lib.pcg_solve(None, None, None, 1e-8, 10, None, None, None) == binding.ERR_ARG
    assert b"NULL handle" in lib.amg_last_error()
    assert lib.amg_set_allocator(ctypes.c_void_p(1), None, None) == binding.ERR_ARG


def test_host_side_checks_of_the_batched_serving_and_tuning_calls():
    """Every entry point that takes a handle, batch or server rejects NULL
    and bad sizes on the host with AMG_ERR_ARG and a message, without a
    device call; the host-only planner and the server defaults need none."""
    from paper_2210_16660_gb300 import binding
    lib = binding.load()
    E = binding.ERR_ARG
    i = ctypes.c_int()
    assert lib.pcg_solve_multi(None, 4, None, None, 1e-8, 10, None, None, None) == E
    out = ctypes.c_void_p()
    assert lib.amg_batch_create(0, None, ctypes.byref(out)) == E
    assert lib.pcg_solve_batch(None, None, None, 1e-8, 10, None, None, None) == E
    assert lib.amg_autotune(None, 5, ctypes.byref(i), None) == E
    shape = (ctypes.c_int * 4)()
    assert lib.amg_level_shape(None, 1, shape) == E
    assert lib.amg_set_level_shape(None, 1, shape) == E
    assert lib.amg_profile_levels(None, 1, None, None) == E
    assert lib.amg_residual_noalloc(None, None, None, None, None, None) == E
    assert lib.amg_refresh(None, None, None) == E
    assert b"NULL handle" in lib.amg_last_error()
    d = ctypes.c_double()
    assert lib.amg_refresh_time(None, ctypes.byref(d)) == E
    p = binding.ServerParams()
    lib.amg_server_default_params(ctypes.byref(p))
    assert (p.mode, p.slots, p.max_engines, p.chunk, p.solo, p.batch_min) == (binding.MODE_FCG32, 4, 2, 4, 1, 3)
    assert lib.amg_server_create(ctypes.byref(p), 0, None, None, ctypes.byref(out)) == E
    t = ctypes.c_int64()
    assert lib.amg_server_submit(None, 0, None, None, None, ctypes.byref(t)) == E
    assert lib.amg_server_progress(None, 0, ctypes.byref(i)) == E
    assert lib.amg_server_result(None, 1, None, None, None, None, None, None) == E
    assert lib.amg_server_info(None, None, None, None, None, None) == E
    assert lib.amg_server_mesh_info(None, 0, None, None, None, None) == E
    assert lib.amg_last_error() != b""
    lib.amg_server_destroy(None)
    lib.amg_batch_destroy(None)
