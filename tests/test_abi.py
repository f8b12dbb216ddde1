"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every function
that include/fehmm.h declares, and rejects invalid arguments without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fehmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fehmm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1908_08292_gb300 import build
    build.build()
    import paper_1908_08292_gb300 as fe
    return fe.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name


def test_default_options_and_argument_errors(L):
    import paper_1908_08292_gb300 as fe
    opt = fe.Options()
    assert L.fehmm_default_options(ctypes.byref(opt), 2, fe.PREC_MIXED) == 0
    assert opt.dim == 2 and opt.precision == 1 and opt.max_newton > 0 and 0 < opt.cg_rtol < 1
    assert opt.retry_stages == 4  # load-continuation retry of failed RVE solves, on by default
    assert L.fehmm_default_options(ctypes.byref(opt), 4, 0) == -1
    assert L.fehmm_default_options(None, 2, 0) == -1
    assert L.fehmm_create(None, None) == -1
    assert L.fehmm_destroy(None) == -1
    assert L.fehmm_rve_solve(None, None, None, None, None, None, None, 0, None) == -1
    assert L.fehmm_status_str(-5).decode() == "unsupported configuration"
    assert L.fehmm_launch_count(None) == -1
