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
    # the trailing fields (the binding's struct layout matches the header's)
    assert o.autotune == 0 and o.schur_damping == 0 and o.coarse_solver == 0
    assert ctypes.sizeof(amgc.Options) == 88
    lib = amgc.load()
    assert lib.amgc_strerror(amgc.AMGC_NOT_CONVERGED) == b"FGMRES did not converge"
    # argument validation happens before any device work
    out = ctypes.c_void_p(0)
    assert lib.amgc_setup(None, None, None, None, None, None, None, None, None, None, None, ctypes.byref(out)) \
        == amgc.AMGC_EINVAL
    assert b"invalid argument" in lib.amgc_last_error()


def test_header_is_plain_c_and_matches_the_binding(tmp_path):
    """include/amgc.h compiles as C99 without warnings, and its option and stats structs have the
    sizes the ctypes binding declares."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include <stdio.h>\n#include "amgc.h"\n'
                   'int main(void) { printf("%zu %zu\\n", sizeof(amgc_options), sizeof(amgc_stats_t)); return 0; }\n')
    exe = tmp_path / "t"
    inc = str(amgc.HEADER).rsplit("/", 1)[0]
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    sizes = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    assert int(sizes[0]) == ctypes.sizeof(amgc.Options)
    assert int(sizes[1]) == ctypes.sizeof(amgc.Stats)
