"""The C-ABI library builds, loads and exports every symbol include/lb.h
declares; the Python binding carries the same names.  No GPU needed (no
compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="lb.h", prefix="lb_"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_6703_gb300.build import build_library
    return ctypes.CDLL(build_library())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_create", "lb_init", "lb_step", "lb_moments", "lb_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_exports_every_network_symbol(lib):
    names = declared_functions("fno.h", "fno_")
    assert "fno_forward" in names and "fno_backward" in names
    for name in names:
        assert hasattr(lib, name), name


def test_network_binding_has_same_names():
    from paper_1307_6703_gb300 import fno
    for name in declared_functions("fno.h", "fno_"):
        assert callable(getattr(fno, name)), name


def test_binding_has_same_names():
    import paper_1307_6703_gb300 as pkg
    for name in declared_functions():
        assert callable(getattr(pkg, name)), name


def test_params_struct_layout_matches_header():
    from paper_1307_6703_gb300.lb import lb_params
    # 4 int32 + 12 doubles + 1 pointer on LP64
    assert ctypes.sizeof(lb_params) == 4 * 4 + 12 * 8 + 8


def test_create_rejects_bad_parameters_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_1307_6703_gb300 import LB_ERR_ARG, LBError, lb_create, lb_params
    base = dict(nx=8, ny=8, walls=1, precision=1, a=0.375, b=1 / 3, T=0.3, kappa=0.1,
                tau=1.0, A0=0.0, lambda_=0.0, u_bot=0.0, u_top=0.0, N=0.5, Q=1.0,
                rho_ref=0.0, stream=None)
    for bad in (dict(tau=0.5), dict(nx=0), dict(walls=1, ny=2), dict(precision=7), dict(T=-1.0),
                dict(precision=2, nx=12), dict(precision=3, ny=4), dict(precision=2, rho_ref=-1.0)):
        p = lb_params(**{**base, **bad})
        with pytest.raises(LBError) as ei:
            lb_create(p)
        assert ei.value.code == LB_ERR_ARG


def test_null_handles_are_refused_without_gpu(lib):
    """Entry points given a NULL handle return LB_ERR_ARG before any CUDA call."""
    from paper_1307_6703_gb300 import LB_ERR_ARG
    assert lib.lb_set_seg_h(None, 64) == LB_ERR_ARG
    assert lib.lb_reduce_async(None, None) == LB_ERR_ARG
    assert lib.lb_monitor(None, None, 0) == LB_ERR_ARG
    assert lib.lb_step(None, 1) == LB_ERR_ARG


def test_product_path_does_not_touch_oracle():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1307_6703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "lb_oracle" not in text


def test_batch_create_rejects_bad_parameters_without_gpu(lib):
    """Batch argument validation happens before any CUDA call."""
    from paper_1307_6703_gb300 import LB_ERR_ARG, LBError, lb_batch_create, lb_params
    base = dict(nx=8, ny=8, walls=1, precision=1, a=0.375, b=1 / 3, T=0.3, kappa=0.1,
                tau=1.0, A0=0.0, lambda_=0.0, u_bot=0.0, u_top=0.0, N=0.5, Q=1.0,
                rho_ref=0.0, stream=None)
    for bad in ([dict(), dict(precision=2)],          # mixed precision
                [dict(), dict(nx=10)],                # not a sweep lattice
                [dict(precision=0), dict(precision=0)],  # FP64 has no sweep kernel
                [dict(precision=2, nx=12)]):
        ps = [lb_params(**{**base, **b}) for b in bad]
        with pytest.raises(LBError) as ei:
            lb_batch_create(ps)
        assert ei.value.code == LB_ERR_ARG


@pytest.mark.parametrize("header", ["lb.h", "fno.h"])
def test_headers_are_plain_c(header, tmp_path):
    """The boundary is a C ABI: each public header compiles on its own as
    C99 and as C++17 with warnings as errors (no C++ or library types)."""
    import shutil
    import subprocess
    for cc, std, lang in (("gcc", "c99", "c"), ("g++", "c++17", "c++")):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not available")
        src = tmp_path / f"use_{header}.{ 'c' if lang == 'c' else 'cpp'}"
        src.write_text(f'#include "{header}"\nint lb_header_check_dummy;\n')
        r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                            "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
