"""GPU parity of the BF16 tensor-core MLP and the surrogate evaluation with the FP64 oracles.

The oracle rounds the weights and every matrix-product operand to bfloat16 at the same points as
the kernels (oracle.mlp, bf16=True); what remains is FP32 accumulation order and the FP32 vs FP64
evaluation of silu before rounding, so the tolerances are a few bfloat16 units (2^-8) relative."""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp
from oracle import surrogate as osur

pytestmark = pytest.mark.gpu


def net(seed):
    p = omlp.init_params(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * synth.random_field(seed + 1, 1, p[k].size, 1.0)[0]
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [300, 1500, 2600])
def test_mlp_eval_forward_gradient_hessian(B):
    """B = 300: ragged tiles everywhere; the 6B-row tangent products of B = 1500 and 2600 run on the
    64- and 128-column tensor-core tiles (the forward products on the 32-column ones)."""
    import torch

    from paper_1908_08292_gb300.surrogate import MLP
    p = net(41)
    x = synth.random_field(43, B, 6, 0.9)
    dev = torch.device("cuda:0")
    m = MLP(max(512, B))
    m.set_params(p)
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    y = torch.zeros(B, dtype=torch.float32, device=dev)
    g = torch.zeros(B, 6, dtype=torch.float32, device=dev)
    H = torch.zeros(B, 6, 6, dtype=torch.float32, device=dev)
    m.eval(xt, y, g, H)
    m.check()  # no tensor-core product gave up waiting for its MMAs
    yr, gr, Hr = omlp.input_hessian(p, x, bf16=True)
    assert rel(y.cpu().numpy(), yr) < 4e-3
    assert rel(g.cpu().numpy(), gr) < 4e-3
    assert rel(H.cpu().numpy(), Hr) < 8e-3
    # per sample (row): a wrong row or a wrong ragged tail tile (the rows past the last full
    # 128-row tile) cannot hide in a batch norm; each row's error relative to the row's own size,
    # floored at 10 % of the batch RMS (rows near zero)
    yg, gg, Hg = y.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy().reshape(B, 36)
    for got, ref, tol in ((yg[:, None], yr[:, None], 3e-2), (gg, gr, 3e-2), (Hg, Hr.reshape(B, 36), 5e-2)):
        floor = 0.1 * np.sqrt((ref ** 2).sum(axis=1).mean())
        row = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), floor)
        assert row.max() < tol, (int(row.argmax()), float(row.max()))
        if B % 128:
            assert row[B - B % 128:].max() < tol  # the ragged tail tile
    # and close to the unquantised FP64 network (BF16 error budget)
    y64, g64, H64 = omlp.input_hessian(p, x)
    assert rel(y.cpu().numpy(), y64) < 3e-2 and rel(g.cpu().numpy(), g64) < 3e-2
    m.close()


def test_mlp_loss_parameter_gradient():
    import torch

    from paper_1908_08292_gb300.surrogate import MLP, unpack
    p = net(51)
    B = 257
    x = synth.random_field(52, B, 6, 0.9)
    ty = synth.random_field(53, 1, B, 1.0)[0]
    tg = synth.random_field(54, B, 6, 1.0)
    cy, cg = 0.7, 1.3
    dev = torch.device("cuda:0")
    m = MLP(512)
    m.set_params(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    m.loss_grad(torch.tensor(x, dtype=torch.float32, device=dev), torch.tensor(ty, dtype=torch.float32, device=dev),
                torch.tensor(tg, dtype=torch.float32, device=dev), cy, cg, loss)
    m.check()
    G = unpack(m.get_grad())
    Gr = omlp.param_grad(p, x, ty, tg, cy, cg, bf16=True)
    Lr = omlp.loss(p, x, ty, tg, cy, cg, bf16=True)
    assert abs(loss.item() - Lr) < 2e-3 * Lr
    for k in Gr:
        assert rel(G[k], Gr[k]) < 2e-2, (k, rel(G[k], Gr[k]))
        # element by element, against the tensor's largest entry: a wrong index or sign in one
        # bias row or one input column cannot hide under the tensor norm
        err = np.abs(np.asarray(G[k]) - np.asarray(Gr[k])).max() / np.abs(Gr[k]).max()
        assert err < 3e-2, (k, err)

    # central finite differences of the GPU loss itself.  The output bias b5 reaches the loss
    # through FP32 arithmetic only, so a small step is exact to O(h^2).  The hidden biases feed
    # bfloat16-rounded activations, whose rounding makes the loss piecewise constant on the
    # scale of a bfloat16 unit: a wide step (h = 0.25) averages that out, and the check is
    # against the same difference of the oracle's bfloat16-mirroring loss (and, loosely, the
    # analytic gradient), which catches a wrong sign or index, not a few percent.
    def gpu_loss(params):
        m.set_params(params)
        m.loss_grad(torch.tensor(x, dtype=torch.float32, device=dev),
                    torch.tensor(ty, dtype=torch.float32, device=dev),
                    torch.tensor(tg, dtype=torch.float32, device=dev), cy, cg, loss)
        torch.cuda.synchronize()
        return float(loss.item())

    def shifted(k, idx, h):
        q = {n: v.copy() for n, v in p.items()}
        q[k].reshape(-1)[idx] += h
        return q

    h = 1e-2
    fd = (gpu_loss(shifted("b5", 0, h)) - gpu_loss(shifted("b5", 0, -h))) / (2 * h)
    g5 = float(np.asarray(G["b5"]).reshape(-1)[0])
    assert abs(fd - g5) < 2e-3 * abs(g5), (fd, g5)
    h = 0.25
    for k in ("b1", "b2", "b4"):
        idx = int(np.argmax(np.abs(np.asarray(Gr[k]).reshape(-1))))  # an entry that matters
        fd_gpu = (gpu_loss(shifted(k, idx, h)) - gpu_loss(shifted(k, idx, -h))) / (2 * h)
        fd_ref = (omlp.loss(shifted(k, idx, h), x, ty, tg, cy, cg, bf16=True)
                  - omlp.loss(shifted(k, idx, -h), x, ty, tg, cy, cg, bf16=True)) / (2 * h)
        gk = float(np.asarray(G[k]).reshape(-1)[idx])
        assert abs(fd_gpu - fd_ref) < 2e-2 * abs(fd_ref), (k, idx, fd_gpu, fd_ref)
        assert abs(fd_gpu - gk) < 0.15 * abs(gk), (k, idx, fd_gpu, gk)
    m.close()


def test_surrogate_eval_and_trust_region():
    import torch

    from paper_1908_08292_gb300.surrogate import MLP, SurrogateParams, surrogate_eval, work_floats
    p = net(61)
    n = 200
    F = synth.random_F(62, n, 3, 0.25)
    lam0, mu0, sx, sg, radius = 1.5, 0.9, 0.35, 0.02, 0.3
    dev = torch.device("cuda:0")
    m = MLP(n)
    m.set_params(p)
    sp = SurrogateParams(lam0, mu0, sx, sg, radius)
    M = synth.random_field(63, 6, 6, 0.1)
    Ca = M + M.T
    sp.set_Ca(Ca)
    y0, g0 = 0.02, synth.random_field(64, 1, 6, 0.05)[0]
    sp.y0 = y0
    for k in range(6):
        sp.g0[k] = g0[k]
    Ft = torch.tensor(F.reshape(n, 9), device=dev)
    P = torch.zeros(n, 9, dtype=torch.float64, device=dev)
    A = torch.zeros(n, 81, dtype=torch.float64, device=dev)
    W = torch.zeros(n, dtype=torch.float64, device=dev)
    inside = torch.zeros(n, dtype=torch.int32, device=dev)
    work = torch.zeros(work_floats(n), dtype=torch.float32, device=dev)
    surrogate_eval(m, sp, Ft, P, A, W, inside, work)
    torch.cuda.synchronize()
    Wr, Pr, Ar = osur.evaluate(p, F, lam0, mu0, sx, sg, bf16=True, Ca=Ca, origin=(y0, g0, np.zeros((6, 6))))
    d = osur.stretch_distance(F)
    ins = inside.cpu().numpy()
    clear = np.abs(d - radius) > 1e-9
    assert np.array_equal(ins[clear], (d[clear] <= radius).astype(np.int32)[clear])
    assert 0 < ins.sum() < n  # both sides of the trust boundary are exercised
    # the base law is evaluated in FP64 on both sides; the network part (sg y and its derivatives)
    # carries the bfloat16 budget: a few 2^-8 units relative to its own size
    zero_net = {k: np.zeros_like(v) for k, v in p.items()}
    Wb, Pb, Ab = osur.evaluate(zero_net, F, lam0, mu0, sx, sg, Ca=Ca)  # base law only
    assert np.linalg.norm(W.cpu().numpy() - Wr) < 8e-3 * np.linalg.norm(Wr - Wb)
    assert np.linalg.norm(P.cpu().numpy() - Pr.reshape(n, 9)) < 8e-3 * np.linalg.norm((Pr - Pb).reshape(n, 9))
    assert np.linalg.norm(A.cpu().numpy() - Ar.reshape(n, 81)) < 1.6e-2 * np.linalg.norm((Ar - Ab).reshape(n, 81))
    # per point: each point's error against the size of its own network part (floored at 10 % of
    # the batch RMS), so that one wrong point cannot hide in the batch norm
    for got, ref, base, tol in ((W.cpu().numpy()[:, None], Wr[:, None], Wb[:, None], 2e-2),
                                (P.cpu().numpy(), Pr.reshape(n, 9), Pb.reshape(n, 9), 2e-2),
                                (A.cpu().numpy(), Ar.reshape(n, 81), Ab.reshape(n, 81), 4e-2)):
        netpart = np.linalg.norm(ref - base, axis=1)
        floor = 0.1 * np.sqrt((netpart ** 2).mean())
        row = np.linalg.norm(got - ref, axis=1) / np.maximum(netpart, floor)
        assert row.max() < tol, (int(row.argmax()), float(row.max()))
    # with a zero network (and no origin shift) the surrogate is exactly the base law
    sp.y0 = 0.0
    for k in range(6):
        sp.g0[k] = 0.0
    m.set_params(np.zeros_like(m.get_params()))
    surrogate_eval(m, sp, Ft, P, A, W, inside, work)
    torch.cuda.synchronize()
    assert rel(W.cpu().numpy(), Wb) < 1e-13
    assert rel(P.cpu().numpy(), Pb.reshape(n, 9)) < 1e-13
    assert rel(A.cpu().numpy(), Ab.reshape(n, 81)) < 1e-13
    # a polynomial part (FP64 on both sides): base law + polynomial, point by point
    c = 0.3 * synth.random_field(65, 1, 896, 1.0)[0]
    for k in range(896):
        sp.poly[k] = c[k]
    surrogate_eval(m, sp, Ft, P, A, W, inside, work)
    torch.cuda.synchronize()
    Wq, Pq, Aq = osur.evaluate(zero_net, F, lam0, mu0, sx, sg, Ca=Ca, poly=c)
    for got, ref in ((W.cpu().numpy()[:, None], Wq[:, None]), (P.cpu().numpy(), Pq.reshape(n, 9)),
                     (A.cpu().numpy(), Aq.reshape(n, 81))):
        part = np.linalg.norm(ref - (Wb[:, None] if ref.shape[1] == 1 else
                                     (Pb.reshape(n, 9) if ref.shape[1] == 9 else Ab.reshape(n, 81))), axis=1)
        assert np.all(np.linalg.norm(got - ref, axis=1) <= 1e-11 * np.maximum(np.linalg.norm(ref, axis=1), 1e-30))
        assert part.max() > 1e-3 * np.linalg.norm(ref, axis=1).max()  # the polynomial is not negligible
    m.close()


@pytest.mark.parametrize("max_degree", [5, 6])
def test_polynomial_fit_recovers_a_polynomial(max_degree):
    """fehmm_surrogate_fit_poly on targets made from a known polynomial of degree 3..max_degree
    (value and gradient by the oracle's power rule) recovers its coefficients, leaves the ones
    above max_degree zero and the remainders at FP32 rounding level; the coefficients agree with
    numpy's least squares of the same weighted system."""
    import torch

    from paper_1908_08292_gb300.surrogate import SurrogateParams, fit_poly
    n = 6000
    nt = {5: 434, 6: 896}[max_degree]
    x = (2.0 * synth.random_field(91, n, 6, 1.0) - 1.0).astype(np.float32)
    c_true = np.zeros(896)
    c_true[:nt] = synth.random_field(92, 1, nt, 1.0)[0] - 0.5
    y, g, _ = osur.poly_value_grad_hess(c_true, x.astype(np.float64))
    dev = torch.device("cuda:0")
    xt = torch.tensor(x, device=dev)
    tyt = torch.tensor(y, dtype=torch.float32, device=dev)
    tgt = torch.tensor(g, dtype=torch.float32, device=dev)
    sp = SurrogateParams(1.0, 1.0, 0.35, 0.01, 0.3)
    for k in range(896):
        sp.poly[k] = 1.0  # overwritten, above max_degree with zeros
    fit_poly(sp, xt, tyt, tgt, max_degree=max_degree)
    c = np.array(sp.poly[:])
    assert not c[nt:].any()
    assert np.abs(c - c_true).max() < 1e-4 * np.abs(c_true).max(), np.abs(c - c_true).max()
    # remainders: FP32 targets, so a few FP32 units of their size
    assert np.abs(tyt.cpu().numpy()).max() < 1e-4 * np.abs(y).max()
    assert np.abs(tgt.cpu().numpy()).max() < 1e-4 * np.abs(g).max()
    # numpy least squares of the same weighted system (rows scaled by the loss normalisation)
    yf, gf = y.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
    wy, wg = 1.0 / np.sqrt((yf ** 2).mean()), 1.0 / np.sqrt((gf ** 2).sum(1).mean())
    N = osur.poly_exponents()[:nt]
    xd = x.astype(np.float64)
    rows = [wy * np.prod(osur._pow(xd[:, None, :], N[None]), axis=-1)]
    for k in range(6):
        rows.append(wg * N[:, k] * np.prod(osur._pow(xd[:, None, :], (N - np.eye(6, dtype=int)[k])[None]), axis=-1))
    Phi = np.concatenate(rows, 0)
    rhs = np.concatenate([wy * yf] + [wg * gf[:, k] for k in range(6)])
    c_np = np.linalg.lstsq(Phi, rhs, rcond=None)[0]
    assert np.abs(c[:nt] - c_np).max() < 1e-6 * np.abs(c_np).max(), np.abs(c[:nt] - c_np).max()
