"""The C-ABI library builds for sm_103a, loads, and exports every function include/amgc.h declares."""
import ctypes
import subprocess

from paper_1912_09056_gb300 import amgc
from paper_1912_09056_gb300.build import build


def test_library_exports_every_declared_symbol():
    path = build()
    lib = ctypes.CDLL(path)
    declared = amgc.header_symbols()
    assert "amgc_setup" in declared and "amgc_vcycle" in declared and "amgc_solve" in declared
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in declared:
        assert f" T {name}" in out, name


def test_defaults_and_error_strings_without_gpu():
    o = amgc.default_options()
    assert o.levels_max == 10 and o.coarse_max_rows == 5000 and o.transfer == 1
    assert abs(o.sa_omega - 4.0 / 3.0) < 1e-15 and abs(o.simple_alpha - 0.8) < 1e-15 and o.tol == 1e-8
    lib = amgc.load()
    assert lib.amgc_strerror(amgc.AMGC_NOT_CONVERGED) == b"FGMRES did not converge"
    # argument validation happens before any device work
    out = ctypes.c_void_p(0)
    assert lib.amgc_setup(None, None, None, None, None, None, None, None, None, None, None, ctypes.byref(out)) \
        == amgc.AMGC_EINVAL
    assert b"invalid argument" in lib.amgc_last_error()
