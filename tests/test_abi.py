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


def test_surrogate_base_law_projection(L):
    """fehmm_surrogate_base_law (host code, no GPU): an isotropic tangent gives back its Lame
    constants and a zero remainder; a cubic one splits into its isotropic projection and a
    remainder that restores it, in Mandel form."""
    import numpy as np

    import paper_1908_08292_gb300 as fe  # noqa: F401  (loads the signatures)
    from paper_1908_08292_gb300.surrogate import SurrogateParams
    I = np.eye(3)
    II = np.einsum("ij,kl->ijkl", I, I)
    Isym = np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)
    sp = SurrogateParams()
    A = np.ascontiguousarray((1.7 * II + 0.9 * Isym).reshape(-1))
    assert L.fehmm_surrogate_base_law(A.ctypes.data, ctypes.byref(sp)) == 0
    assert abs(sp.lam0 - 1.7) < 1e-13 and abs(sp.mu0 - 0.9) < 1e-13
    assert np.abs(np.array(sp.Ca[:])).max() < 1e-13
    # cubic: extra stiffness c on the axial components only
    cub = np.zeros((3, 3, 3, 3))
    for i in range(3):
        cub[i, i, i, i] = 0.6
    A = 1.7 * II + 0.9 * Isym + cub
    assert L.fehmm_surrogate_base_law(np.ascontiguousarray(A.reshape(-1)).ctypes.data, ctypes.byref(sp)) == 0
    iso = sp.lam0 * II + sp.mu0 * Isym
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    w = [1.0, 1.0, 1.0] + [np.sqrt(2.0)] * 3
    M = np.array([[(A - iso)[i, j, k, l] * w[p] * w[q] for q, (k, l) in enumerate(pairs)]
                  for p, (i, j) in enumerate(pairs)])
    np.testing.assert_allclose(np.array(sp.Ca[:]).reshape(6, 6), M, atol=1e-13)
    # the projection removes the isotropic content: the remainder has no bulk or shear trace
    R = A - iso
    assert abs(np.einsum("iijj->", R)) < 1e-12 and abs(np.einsum("ijij->", R)) < 1e-12


def test_surrogate_polynomial_and_mlp_argument_errors(L):
    """Invalid arguments of the polynomial fit and the MLP status check are rejected on the host,
    before any device call; the parameter struct carries the 896 polynomial coefficients."""
    from paper_1908_08292_gb300.surrogate import POLY_TERMS, SurrogateParams
    sp = SurrogateParams()
    assert POLY_TERMS == 896 and len(sp.poly) == 896
    assert ctypes.sizeof(SurrogateParams) == 8 * (5 + 36 + 1 + 6 + 36 + 896)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the checks come first
    for deg in (2, 7):
        assert L.fehmm_surrogate_fit_poly(ctypes.byref(sp), dummy, dummy, dummy, 10, deg, None) == -1
    assert L.fehmm_surrogate_fit_poly(None, dummy, dummy, dummy, 10, 6, None) == -1
    assert L.fehmm_surrogate_fit_poly(ctypes.byref(sp), dummy, dummy, dummy, 0, 6, None) == -1
    flag = ctypes.c_int(0)
    assert L.fehmm_mlp_check(None, ctypes.byref(flag)) == -1
