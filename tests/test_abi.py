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
