"""CPU-side checks of the C-ABI library: it loads, exports every entry point
declared in include/fsim.h, and rejects bad arguments without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_02999_gb300 import build, fsim
    build.build()
    return fsim.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "fsim.h")).read()
    return sorted(set(re.findall(r"^fsim_status\s+(fsim_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2312_02999_gb300 import fsim
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fsim.exported_symbols())


def test_default_params_and_argument_checks(lib):
    from paper_2312_02999_gb300 import fsim
    p = fsim.default_params()
    assert p.max_iters == 500 and p.max_ls == 40 and abs(p.ccd_s - 0.1) < 1e-15
    assert abs(p.tol_abs - 1e-8) < 1e-20 and p.accd_max_iters == 2000
    assert lib.fsim_default_params(None) == fsim.FSIM_EINVAL
    assert lib.fsim_destroy(None) == fsim.FSIM_EINVAL
    assert lib.fsim_prefactor(None, 0, None) == fsim.FSIM_EINVAL
    assert lib.fsim_solve_frame(None, 0, None, 0, None) == fsim.FSIM_EINVAL
    h = C.c_void_p()
    assert lib.fsim_create(C.byref(h), -1) == fsim.FSIM_EINVAL


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2312_02999_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, re.M), f
