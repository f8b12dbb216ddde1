"""Pins of the FP64 surrogate-MLP oracle by central finite differences: dy/dx, the input
Hessian, and the parameter gradient of the Sobolev loss (value + input-gradient targets)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import mlp


@pytest.fixture(scope="module")
def net():
    p = mlp.init_params(7, width=16)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * synth.random_field(8, 1, p[k].size, 1.0)[0]
    return p


def _small(monkeypatch):
    monkeypatch.setattr(mlp, "WIDTH", 16)


def test_input_grad_and_hessian_fd(net, monkeypatch):
    _small(monkeypatch)
    x = synth.random_field(9, 3, 6, 0.8)
    y, g, H = mlp.input_hessian(net, x)
    h = 1e-5
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        yp, gp, _, _ = mlp.input_grad(net, x + e)
        ym, gm, _, _ = mlp.input_grad(net, x - e)
        np.testing.assert_allclose((yp - ym) / (2 * h), g[:, k], atol=1e-8)
        np.testing.assert_allclose((gp - gm) / (2 * h), H[:, :, k], atol=1e-7)
    np.testing.assert_allclose(H, np.swapaxes(H, 1, 2), atol=1e-10)  # symmetric


def test_param_grad_fd(net, monkeypatch):
    _small(monkeypatch)
    x = synth.random_field(10, 4, 6, 0.8)
    ty = synth.random_field(11, 1, 4, 1.0)[0]
    tg = synth.random_field(12, 4, 6, 1.0)
    G = mlp.param_grad(net, x, ty, tg, 0.7, 1.3)
    h = 1e-6
    rng_idx = synth.uniform(13, np.arange(len(net)), 3)
    for j, (name, v) in enumerate(net.items()):
        for u in rng_idx[j]:
            i = int(u * v.size)
            pp = {k: a.copy() for k, a in net.items()}
            pm = {k: a.copy() for k, a in net.items()}
            pp[name].reshape(-1)[i] += h
            pm[name].reshape(-1)[i] -= h
            fd = (mlp.loss(pp, x, ty, tg, 0.7, 1.3) - mlp.loss(pm, x, ty, tg, 0.7, 1.3)) / (2 * h)
            assert abs(fd - G[name].reshape(-1)[i]) < 1e-6 * max(1.0, abs(fd)), (name, i, fd, G[name].reshape(-1)[i])


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to the even (1.0)
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3])
    r = mlp.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8


def test_surrogate_chain_rule_fd():
    from oracle import surrogate as sur
    p = mlp.init_params(21)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.05 * synth.random_field(22, 1, p[k].size, 1.0)[0]
    F = synth.random_F(23, 2, 3, 0.12)
    lam0, mu0, sx, sg = 1.2, 0.8, 0.35, 0.05
    M = synth.random_field(24, 6, 6, 0.1)
    Ca = M + M.T
    origin = (0.01, synth.random_field(25, 1, 6, 0.02)[0], np.zeros((6, 6)))
    poly = 0.05 * synth.random_field(26, 1, sur.poly_exponents().shape[0], 1.0)[0]
    kw = dict(Ca=Ca, origin=origin, poly=poly)
    W, P, A = sur.evaluate(p, F, lam0, mu0, sx, sg, **kw)
    h = 1e-6
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = h
            Wp, Pp, _ = sur.evaluate(p, F + E, lam0, mu0, sx, sg, **kw)
            Wm, Pm, _ = sur.evaluate(p, F - E, lam0, mu0, sx, sg, **kw)
            np.testing.assert_allclose((Wp - Wm) / (2 * h), P[:, k, l], atol=2e-8)
            np.testing.assert_allclose((Pp - Pm) / (2 * h), A[:, :, :, k, l], atol=2e-7)


def test_stretch_distance_closed_form():
    from oracle import surrogate as sur
    U = synth.stretch_ball(31, 5, 0.3)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    d = sur.stretch_distance(R @ U)  # rotation-invariant: |U - I|_F of the stretch
    np.testing.assert_allclose(d, np.linalg.norm(U - np.eye(3), axis=(1, 2)), atol=1e-12)
    assert np.all(d <= 0.3 + 1e-12)


def test_polynomial_part_monomials_and_derivatives():
    """The polynomial part: 56 + 126 + 252 + 462 monomials in the documented order, a single
    coefficient reproduces its monomial, and gradient / Hessian match central differences of the
    value."""
    from oracle import surrogate as sur
    N = sur.poly_exponents()
    assert N.shape == (896, 6)
    assert [int((N.sum(1) == d).sum()) for d in (3, 4, 5, 6)] == [56, 126, 252, 462]
    assert list(N[0]) == [3, 0, 0, 0, 0, 0] and list(N[1]) == [2, 1, 0, 0, 0, 0]
    assert list(N[55]) == [0, 0, 0, 0, 0, 3] and list(N[56]) == [4, 0, 0, 0, 0, 0]
    assert list(N[433]) == [0, 0, 0, 0, 0, 5] and list(N[434]) == [6, 0, 0, 0, 0, 0]
    assert list(N[895]) == [0, 0, 0, 0, 0, 6]
    x = synth.random_field(41, 3, 6, 0.8) - 0.4
    # the monomial x0 x1 x5^2 (index tuple (0, 1, 5, 5), degree 4)
    idx = 56 + list(itertools.combinations_with_replacement(range(6), 4)).index((0, 1, 5, 5))
    c = np.zeros(896)
    c[idx] = 1.0
    y, g, H = sur.poly_value_grad_hess(c, x)
    np.testing.assert_allclose(y, x[:, 0] * x[:, 1] * x[:, 5] ** 2, rtol=1e-14)
    np.testing.assert_allclose(g[:, 5], 2 * x[:, 0] * x[:, 1] * x[:, 5], rtol=1e-14)
    np.testing.assert_allclose(H[:, 5, 5], 2 * x[:, 0] * x[:, 1], rtol=1e-14)
    np.testing.assert_allclose(H[:, 0, 5], 2 * x[:, 1] * x[:, 5], rtol=1e-14)
    np.testing.assert_allclose(H[:, 0, 0], 0.0, atol=1e-15)
    # random coefficients: derivatives against central differences
    c = synth.random_field(42, 1, 896, 1.0)[0]
    y, g, H = sur.poly_value_grad_hess(c, x)
    h = 1e-5
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        yp, gp, _ = sur.poly_value_grad_hess(c, x + e)
        ym, gm, _ = sur.poly_value_grad_hess(c, x - e)
        np.testing.assert_allclose((yp - ym) / (2 * h), g[:, k], rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose((gp - gm) / (2 * h), H[:, :, k], rtol=1e-7, atol=1e-8)
    # no term below degree 3: value, gradient and Hessian vanish at x = 0
    y0, g0, H0 = sur.poly_value_grad_hess(c, np.zeros((1, 6)))
    assert y0[0] == 0.0 and not g0.any() and not H0.any()
