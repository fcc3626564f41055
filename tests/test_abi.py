"""The C-ABI library loads and exports every entry point declared in include/of.h, and
rejects invalid arguments before touching the GPU (no compute call here)."""
import ctypes as C
import os
import re

import pytest

from paper_1412_8250_gb300 import binding as B, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "of.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(of_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    build_lib.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.exported_symbols()) == names


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    h = C.c_void_p()
    assert lib.of_grid_create(0, 8, 8, 1.0, 1.0, 1.0, 6, None, C.byref(h)) == B.OF_EINVAL
    assert "bad sizes" in B.of_last_error()
    assert lib.of_grid_create(8, 8, 8, 1.0, 1.0, 1.0, 2, None, C.byref(h)) == B.OF_EINVAL
    assert "fd_half_order" in B.of_last_error()
    assert lib.of_grid_create(8, 8, 8, 1.0, -1.0, 1.0, 6, None, C.byref(h)) == B.OF_EINVAL
    assert lib.of_laplacian_apply(None, 0, None, None) == B.OF_EINVAL
    assert lib.of_poisson_solve(None, None, None, None, None) == B.OF_EINVAL
    assert lib.of_forces(None, None, None, None, None) == B.OF_EINVAL
    assert lib.of_grid_destroy(None) == B.OF_OK


def test_default_options(lib):
    o = B.of_default_scf_opts()
    assert o.nlcg_tol == 1e-7 and o.anderson_m == 7 and o.anderson_zeta == 0.3
    assert o.poisson.tol == 1e-10 and o.kernel.max_iter == 20000
