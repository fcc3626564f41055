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
    assert lib.of_relax(None, None, None, None, None, None, None, None, None, None) == B.OF_EINVAL
    assert "of_relax" in B.of_last_error()
    assert lib.of_vacancy_formation(None, None, None, 0, None, None, None, None, None, None, None,
                                    None, None) == B.OF_EINVAL
    assert "of_vacancy_formation" in B.of_last_error()
    x = C.c_double(1.0)
    assert lib.of_alu_peak(7, None, C.byref(x)) == B.OF_EINVAL
    assert "kind 7" in B.of_last_error()
    assert lib.of_alu_peak(B.OF_PEAK_F64, None, None) == B.OF_EINVAL
    assert lib.of_grid_destroy(None) == B.OF_OK


def test_default_options(lib):
    o = B.of_default_scf_opts()
    assert o.nlcg_tol == 1e-7 and o.anderson_m == 7 and o.anderson_zeta == 0.3
    assert o.poisson.tol == 1e-10 and o.kernel.max_iter == 20000


STRUCTS = ["of_solve_opts", "of_solve_info", "of_system", "of_functional", "of_scf_opts",
           "of_scf_result", "of_relax_opts", "of_relax_result", "of_vacancy_result",
           "of_kernel_stat"]


def test_binding_structs_match_the_header(tmp_path):
    # every record the binding passes across the boundary has the header's size and field
    # offsets (a C program built from include/of.h prints them)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "of.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(B, name)
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {cname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        name, field, value = line.split()
        cls = getattr(B, name)
        got = C.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)
        seen += 1
    assert seen > 60
