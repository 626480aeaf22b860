"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(vofp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1410_1937_gb300 import build as B
    return ctypes.CDLL(B.build())


def test_header_declares_entry_points():
    names = declared_symbols()
    assert {"vofp_create", "vofp_build_operator", "vofp_solve", "vofp_apply", "vofp_destroy"} <= names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1410_1937_gb300 import vofp
    assert declared_symbols() <= set(vofp.EXPORTED)


def test_invalid_arguments_rejected_before_device_use(lib):
    from paper_1410_1937_gb300 import vofp
    import numpy as np
    with pytest.raises(vofp.VofpError) as e:
        vofp.vofp_create(np.ones(0), np.ones(3), np.ones(3), stream=type("S", (), {"cuda_stream": 0})())
    assert e.value.status == vofp.ERR_INVALID_ARG
    with pytest.raises(vofp.VofpError):
        vofp.vofp_create(np.array([1.0, -1.0]), np.ones(3), np.ones(3), stream=type("S", (), {"cuda_stream": 0})())
    assert vofp.vofp_version().startswith("vofp")
    lib.vofp_last_error.restype = ctypes.c_char_p
    assert lib.vofp_last_error(None) == b"null context"


def test_null_context_is_rejected_by_every_entry_point():
    # no device is touched: each call checks its context first
    from paper_1410_1937_gb300 import vofp
    L = vofp._lib
    n = None
    calls = {
        "vofp_build_operator": lambda: L.vofp_build_operator(n, n, n, n, n, n, n, n),
        "vofp_rhs_from_face_velocity": lambda: L.vofp_rhs_from_face_velocity(n, n, n, n, n, n),
        "vofp_project": lambda: L.vofp_project(n, n, n, n, n, n, n, n, n, n, n),
        "vofp_exit_flux": lambda: L.vofp_exit_flux(n, n, n, n, n, 1.0, n, 0, n, n),
        "vofp_vof_flux_correct": lambda: L.vofp_vof_flux_correct(*([n] * 11)),
        "vofp_vof_advect": lambda: L.vofp_vof_advect(*([n] * 9), 0.1, 0, n),
        "vofp_rk2_step": lambda: L.vofp_rk2_step(*([n] * 15), n, 0, n),
        "vofp_apply": lambda: L.vofp_apply(n, n, n),
        "vofp_solve": lambda: L.vofp_solve(n, n, n, n, n),
        "vofp_solve_host": lambda: L.vofp_solve_host(*([n] * 14)),
        "vofp_solve_host_batch": lambda: L.vofp_solve_host_batch(n, 1, n, n, n, n, n),
    }
    for name, call in calls.items():
        assert call() == vofp.ERR_INVALID_ARG, name


def test_binding_fails_loudly_without_the_library(tmp_path):
    # no CPU fallback: the binding refuses to import when libvofp.so is absent
    import shutil
    import subprocess
    import sys
    shutil.copy(os.path.join(ROOT, "paper_1410_1937_gb300", "vofp.py"), tmp_path / "vofp.py")
    r = subprocess.run([sys.executable, "-c", "import vofp"], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0 and "libvofp.so is not built" in r.stderr


def test_host_pointers_only_from_arrays_that_outlive_the_call():
    # a list or another dtype would be converted to a temporary whose memory is freed before the
    # C call reads it: the binding refuses those instead of passing a dangling address
    import numpy as np
    from paper_1410_1937_gb300 import vofp
    hp = vofp.Context._host_ptr
    a = np.arange(4, dtype=np.float64)
    assert hp(a, 4, "a").value == a.ctypes.data
    assert hp(None, 4, "a") is None
    for bad in ([0.0, 1.0, 2.0, 3.0], np.arange(4, dtype=np.float32), np.zeros((4, 2))[:, 0], np.zeros(5)):
        with pytest.raises(ValueError):
            hp(bad, 4, "a")
