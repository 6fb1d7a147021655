"""The C ABI: libparis.so loads without a GPU, exports every function that
include/paris.h declares, the ctypes binding declares the same set, and the
struct layouts agree with a C compiler's."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paris.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(paris_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_11744_gb300 import _abi
    return _abi.load()


def test_header_declares_the_four_steps():
    fns = declared_functions()
    for name in ("paris_face_coeffs", "paris_divergence", "paris_poisson_solve", "paris_project"):
        assert name in fns


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2012_11744_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(declared_functions())


def test_struct_layouts_match_c(tmp_path):
    from paper_2012_11744_gb300 import _abi
    prog = tmp_path / "sizes.c"
    prog.write_text('#include "paris.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(paris_grid), '
                    'sizeof(paris_opts), sizeof(paris_stats), sizeof(paris_kernel_prof), '
                    'offsetof(paris_opts, inner_tol), offsetof(paris_stats, levels));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ct.sizeof(_abi.Grid), ct.sizeof(_abi.Opts), ct.sizeof(_abi.Stats),
            ct.sizeof(_abi.KernelProf), _abi.Opts.inner_tol.offset, _abi.Stats.levels.offset]
    assert got == want


def test_defaults_and_status_strings(lib):
    from paper_2012_11744_gb300 import _abi
    o = _abi.Opts()
    lib.paris_default_opts(ct.byref(o))
    assert o.tol == 1e-10 and o.precision == _abi.MIXED and o.nu1 == 2 and o.nu2 == 2
    for s in range(7):
        assert lib.paris_status_string(s)
    assert lib.paris_launch_count() >= 0


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2012_11744_gb300 import _abi
    ctx = ct.c_void_p()
    g = _abi.Grid()
    g.nx, g.ny, g.nz, g.h = 1, 8, 8, 0.1
    assert lib.paris_create(ct.byref(ctx), ct.byref(g), None, None) == _abi.PARIS_ERR_INVALID_ARG
    g.nx, g.h = 8, -1.0
    assert lib.paris_create(ct.byref(ctx), ct.byref(g), None, None) == _abi.PARIS_ERR_INVALID_ARG
    g.h = 0.1
    g.bc[1] = 7
    assert lib.paris_create(ct.byref(ctx), ct.byref(g), None, None) == _abi.PARIS_ERR_INVALID_ARG
    g.bc[1] = 0
    o = _abi.Opts()
    lib.paris_default_opts(ct.byref(o))
    o.omega = 2.5
    assert lib.paris_create(ct.byref(ctx), ct.byref(g), ct.byref(o), None) == _abi.PARIS_ERR_INVALID_ARG
    assert lib.paris_face_coeffs(None, None, 1.0, 1.0, None, None, None) == _abi.PARIS_ERR_INVALID_ARG
    assert lib.paris_divergence_noalloc(None, None, None, None, 1.0, None, None, None) == \
        _abi.PARIS_ERR_INVALID_ARG
