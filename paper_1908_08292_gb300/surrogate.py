"""Energy surrogate (the learned part of the workload; the paper has no counterpart): binding
of the BF16 tensor-core MLP and of the surrogate evaluation in libfehmm.so, plus the host
control flow of data generation and training.  Every numerical step runs in library kernels:
RVE solves for the training targets, the MLP forward/backward/Hessian and AdamW, the
surrogate's chain rule to P and dP/dF.

Model: W(F) = W_base(E) + sg * y(Mandel(E)/sx), E = (F^T F - I)/2, with W_base the paper's
compressible neo-Hookean law (Sec. 6) at Lame constants (lam0, mu0) taken as the isotropic
projection of the RVE's small-strain homogenised tangent, and y the MLP.  Training targets are
homogenised energies and second Piola-Kirchhoff stresses of full RVE solves at F = U, U sampled
uniformly in the ball |U - I|_F <= 0.3 (Sobolev loss on the value and the input gradient).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import Context, FehmmError, _check, _dev, _stream, lib

WIDTH, N_IN, N_INP = 128, 6, 8


def n_params() -> int:
    return int(lib().fehmm_mlp_num_params())


def _offsets():
    o, off = {}, 0
    for name, size in (("W1", WIDTH * N_INP), ("b1", WIDTH), ("W2", WIDTH * WIDTH), ("b2", WIDTH),
                       ("W3", WIDTH * WIDTH), ("b3", WIDTH), ("W4", WIDTH * WIDTH), ("b4", WIDTH),
                       ("w5", WIDTH), ("b5", 1)):
        o[name] = (off, size)
        off += size
    return o


def pack(params: dict) -> np.ndarray:
    """Packed float32 parameter vector in the library's layout (W1 padded to 8 input columns)."""
    v = np.zeros(n_params(), dtype=np.float32)
    for name, (off, size) in _offsets().items():
        a = np.asarray(params[name], dtype=np.float64)
        if name == "W1":
            w = np.zeros((WIDTH, N_INP))
            w[:, :N_IN] = a
            a = w
        v[off:off + size] = a.reshape(-1)
    return v


def unpack(v) -> dict:
    out = {}
    for name, (off, size) in _offsets().items():
        a = np.asarray(v[off:off + size], dtype=np.float64)
        if name == "W1":
            a = a.reshape(WIDTH, N_INP)[:, :N_IN]
        elif name.startswith("W"):
            a = a.reshape(WIDTH, WIDTH)
        out[name] = a.copy()
    return out


def init_params(seed: int, out_scale: float = 1.0) -> dict:
    """He-uniform weights from the SplitMix64 input generator, zero biases; the output weights
    scaled by out_scale (0: a zero output layer, so that training starts from y = 0, for targets
    far smaller than the initial network's output, e.g. what a fitted polynomial leaves)."""
    import synth
    p = {}
    fan = [N_IN, WIDTH, WIDTH, WIDTH]
    for l in range(4):
        b = math.sqrt(6.0 / fan[l])
        p[f"W{l + 1}"] = b * (2 * synth.uniform(seed, np.arange(WIDTH) + 1000 * l, fan[l]) - 1)
        p[f"b{l + 1}"] = np.zeros(WIDTH)
    p["w5"] = out_scale * math.sqrt(3.0 / WIDTH) * (2 * synth.uniform(seed, np.array([999999]), WIDTH)[0] - 1)
    p["b5"] = np.zeros(1)
    return p


class MLP:
    def __init__(self, max_batch: int):
        h = ctypes.c_void_p()
        _check(lib().fehmm_mlp_create(ctypes.byref(h), int(max_batch)), "mlp_create")
        self._h = h
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "_h", None):
            lib().fehmm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        v = pack(params) if isinstance(params, dict) else np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().fehmm_mlp_set_params(self._h, v.ctypes.data), "mlp_set_params")

    def get_params(self):
        v = np.zeros(n_params(), dtype=np.float32)
        _check(lib().fehmm_mlp_get_params(self._h, v.ctypes.data, None), "mlp_get_params")
        return v

    def grad_buffer(self):
        """Device view (torch float32, no copy) of the gradient of the last loss_grad call."""
        import torch

        from . import _DevArray
        ptr, n = ctypes.c_void_p(), ctypes.c_int()
        _check(lib().fehmm_mlp_grad_buffer(self._h, ctypes.byref(ptr), ctypes.byref(n)), "mlp_grad_buffer")
        return torch.as_tensor(_DevArray(ptr.value, n.value, "<f4"), device="cuda")

    def get_grad(self):
        v = np.zeros(n_params(), dtype=np.float32)
        _check(lib().fehmm_mlp_get_params(self._h, None, v.ctypes.data), "mlp_get_params")
        return v

    def eval(self, x, y=None, g=None, H=None, stream=None):
        import torch
        B = x.shape[0]
        _check(lib().fehmm_mlp_eval(self._h, _dev(x, torch.float32, "x", B * N_IN), B,
                                    _dev(y, torch.float32, "y"), _dev(g, torch.float32, "g"),
                                    _dev(H, torch.float32, "H"), _stream(stream)), "mlp_eval")

    def loss_grad(self, x, ty, tg, cy, cg, loss=None, stream=None):
        import torch
        B = x.shape[0]
        _check(lib().fehmm_mlp_loss_grad(self._h, _dev(x, torch.float32, "x", B * N_IN),
                                         _dev(ty, torch.float32, "ty", B), _dev(tg, torch.float32, "tg", B * N_IN),
                                         B, float(cy), float(cg), _dev(loss, torch.float32, "loss"),
                                         _stream(stream)), "mlp_loss_grad")

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(lib().fehmm_mlp_adamw(self._h, float(lr), float(beta1), float(beta2), float(eps),
                                     float(weight_decay), _stream(stream)), "mlp_adamw")

    def launches(self):
        """Kernels this MLP has launched so far."""
        return int(lib().fehmm_mlp_launch_count(self._h))

    def check(self):
        """Synchronise; raise if a tensor-core product gave up waiting for its MMAs since the
        last check (its outputs are then invalid)."""
        flag = ctypes.c_int(0)
        _check(lib().fehmm_mlp_check(self._h, ctypes.byref(flag)), "mlp_check")
        if flag.value:
            raise RuntimeError("fehmm: a tensor-core matrix product timed out waiting for its MMAs")


POLY_TERMS = 896  # monomials of degree 3..6 in the 6 features (FEHMM_POLY_TERMS)


class SurrogateParams(ctypes.Structure):
    _fields_ = [("lam0", ctypes.c_double), ("mu0", ctypes.c_double), ("sx", ctypes.c_double),
                ("sg", ctypes.c_double), ("radius", ctypes.c_double), ("Ca", ctypes.c_double * 36),
                ("y0", ctypes.c_double), ("g0", ctypes.c_double * 6), ("H0", ctypes.c_double * 36),
                ("poly", ctypes.c_double * POLY_TERMS)]

    def set_Ca(self, M):
        M = np.asarray(M, dtype=np.float64).reshape(36)
        for k in range(36):
            self.Ca[k] = M[k]

    def set_origin(self, mlp, hessian=False):
        """Store the network's value and gradient (and optionally Hessian) at x = 0, evaluated by
        the library, to be subtracted from the learned correction."""
        import torch
        dev = torch.device("cuda")
        x = torch.zeros(1, 6, dtype=torch.float32, device=dev)
        y = torch.zeros(1, dtype=torch.float32, device=dev)
        g = torch.zeros(1, 6, dtype=torch.float32, device=dev)
        H = torch.zeros(1, 6, 6, dtype=torch.float32, device=dev)
        mlp.eval(x, y, g, H)
        self.y0 = float(y.item())
        gh, Hh = g.cpu().numpy().reshape(6), H.cpu().numpy().reshape(36)
        for k in range(6):
            self.g0[k] = float(gh[k])
        for k in range(36):
            self.H0[k] = float(0.5 * (Hh[k] + Hh[6 * (k % 6) + k // 6])) if hessian else 0.0


def save(mlp: MLP, sp: SurrogateParams, path: str):
    """Write the trained network and its surrogate parameters to a file."""
    _check(lib().fehmm_surrogate_save(mlp._h, ctypes.byref(sp), str(path).encode()), "surrogate_save")


def load(mlp: MLP, path: str) -> SurrogateParams:
    """Read a surrogate file into `mlp`; returns its surrogate parameters."""
    sp = SurrogateParams()
    _check(lib().fehmm_surrogate_load(mlp._h, ctypes.byref(sp), str(path).encode()), "surrogate_load")
    return sp


def surrogate_eval(mlp: MLP, sp: SurrogateParams, F, P, A, W, inside, work, stream=None):
    import torch
    n = F.shape[0]
    _check(lib().fehmm_surrogate_eval(mlp._h, ctypes.byref(sp), _dev(F, torch.float64, "F", 9 * n), n,
                                      _dev(P, torch.float64, "P", 9 * n), _dev(A, torch.float64, "A"),
                                      _dev(W, torch.float64, "W"), _dev(inside, torch.int32, "inside", n),
                                      _dev(work, torch.float32, "work", work_floats(n)), _stream(stream)),
           "surrogate_eval")


def fit_poly(sp: SurrogateParams, x, ty, tg, max_degree=6, stream=None):
    """Fit the polynomial part of the correction (monomials of degree 3..max_degree) to the
    training targets (device x, ty, tg from surrogate_targets) by the library
    (fehmm_surrogate_fit_poly): sets sp.poly and replaces ty, tg in place by what the polynomial
    leaves for the network."""
    import torch
    n = x.shape[0]
    _check(lib().fehmm_surrogate_fit_poly(ctypes.byref(sp), _dev(x, torch.float32, "x", 6 * n),
                                          _dev(ty, torch.float32, "ty", n), _dev(tg, torch.float32, "tg", 6 * n), n,
                                          int(max_degree), _stream(stream)), "surrogate_fit_poly")


def work_floats(n: int) -> int:
    return int(lib().fehmm_surrogate_work_floats(int(n)))


def surrogate_targets(sp: SurrogateParams, F, P, W, x, ty, tg, stream=None):
    import torch
    n = F.shape[0]
    _check(lib().fehmm_surrogate_targets(ctypes.byref(sp), _dev(F, torch.float64, "F", 9 * n),
                                         _dev(P, torch.float64, "P", 9 * n), _dev(W, torch.float64, "W", n), n,
                                         _dev(x, torch.float32, "x", 6 * n), _dev(ty, torch.float32, "ty", n),
                                         _dev(tg, torch.float32, "tg", 6 * n), _stream(stream)), "surrogate_targets")


# ----------------------------------------------------------------------------- pipeline
def fixed_rve_context(n_qp, precision="mixed", grid=12, **options):
    """A 3D context whose n_qp points all use the fixed two-inclusion microstructure (grid^3)."""
    import synth
    phase, _ = synth.fixed_rve12(n=grid)
    ctx = Context(3, precision, **options)
    ctx.add_rves([grid], [phase], [[1.0, 10.0]], [[0.3, 0.3]])
    ctx.bind_qps(np.zeros(n_qp, dtype=np.int32))
    return ctx


def rve_solve_batch(ctx, F, with_tangent=False, with_energy=True, stages=1):
    """Full RVE solves at the deformation gradients F (device [n][9], n = ctx.n_qp) from zero
    fluctuations, reached in `stages` equal increments of F - I (load continuation; each
    stage warm-starts from the previous one).  Returns device tensors P, A (or None), W, status."""
    import torch

    from . import SOLVE_ENERGY, SOLVE_FROM_COMMITTED, SOLVE_NO_TANGENT
    n = ctx.n_qp
    dev = F.device
    P = torch.zeros(n, 9, dtype=torch.float64, device=dev)
    A = torch.zeros(n, 81, dtype=torch.float64, device=dev) if with_tangent else None
    W = torch.zeros(n, dtype=torch.float64, device=dev)
    st = torch.zeros(n, dtype=torch.int32, device=dev)
    it = torch.zeros(n, 4, dtype=torch.int32, device=dev)
    eye = torch.eye(3, dtype=torch.float64, device=dev).reshape(1, 9)
    for k in range(1, stages + 1):
        last = k == stages
        Fk = F if last else (eye + (k / stages) * (F - eye)).contiguous()
        flags = (SOLVE_FROM_COMMITTED if k == 1 else 0) | (SOLVE_ENERGY if (with_energy and last) else 0)
        flags |= 0 if (with_tangent and last) else SOLVE_NO_TANGENT
        ctx.rve_solve(Fk, P, A if last else None, st, it, W=W if last else None, flags=flags)
    return P, A, W, st


def base_law(ctx_one):
    """Base energy of the surrogate from the small-strain homogenised tangent A0 (an RVE solve at
    F = I): (lam0, mu0) its isotropic projection and Ca the Mandel form of the remainder, both by
    the library (fehmm_surrogate_base_law)."""
    import torch
    F = torch.eye(3, dtype=torch.float64, device="cuda").reshape(1, 9).repeat(ctx_one.n_qp, 1).contiguous()
    P, A, W, st = rve_solve_batch(ctx_one, F, with_tangent=True, with_energy=False)
    A0 = np.ascontiguousarray(A[0].cpu().numpy(), dtype=np.float64)
    sp = SurrogateParams()
    _check(lib().fehmm_surrogate_base_law(A0.ctypes.data, ctypes.byref(sp)), "surrogate_base_law")
    return sp.lam0, sp.mu0, np.array(sp.Ca[:]).reshape(6, 6)


def generate(ctx, sp, U, chunk=None, stages=3, drop_failed=True):
    """Training data from full GPU RVE solves at F = U (host array (N, 3, 3)): device float32
    features x (N, 6), targets ty (N,), tg (N, 6), plus the FP64 P, W of the solves and the
    number of samples dropped because their RVE solve failed (status > 1, reported)."""
    import torch
    N = U.shape[0]
    chunk = ctx.n_qp if chunk is None else chunk
    dev = torch.device("cuda")
    x = torch.zeros(N, 6, dtype=torch.float32, device=dev)
    ty = torch.zeros(N, dtype=torch.float32, device=dev)
    tg = torch.zeros(N, 6, dtype=torch.float32, device=dev)
    Ps = torch.zeros(N, 9, dtype=torch.float64, device=dev)
    Ws = torch.zeros(N, dtype=torch.float64, device=dev)
    bad = 0
    hist = np.zeros(8, dtype=np.int64)
    ok = torch.ones(N, dtype=torch.bool, device=dev)
    for s0 in range(0, N, chunk):
        m = min(chunk, N - s0)
        Fh = np.zeros((ctx.n_qp, 9))
        Fh[:, [0, 4, 8]] = 1.0
        Fh[:m] = U[s0:s0 + m].reshape(m, 9)
        F = torch.tensor(Fh, device=dev)
        P, _, W, st = rve_solve_batch(ctx, F, stages=stages)
        ok[s0:s0 + m] = st[:m] <= 1
        sts = st[:m].cpu().numpy()
        bad += int((sts > 1).sum())
        hist += np.bincount(np.clip(sts, 0, 7), minlength=8)
        surrogate_targets(sp, F[:m].contiguous(), P[:m].contiguous(), W[:m].contiguous(), x[s0:s0 + m],
                          ty[s0:s0 + m], tg[s0:s0 + m])
        Ps[s0:s0 + m] = P[:m]
        Ws[s0:s0 + m] = W[:m]
    if bad and not drop_failed:
        raise FehmmError(f"{bad} training RVE solves failed (status counts {hist.tolist()})")
    if bad:
        x, ty, tg, Ps, Ws = (t[ok].contiguous() for t in (x, ty, tg, Ps, Ws))
    return x, ty, tg, Ps, Ws, bad


def train(mlp, x, ty, tg, epochs, batch=4096, lr=2e-3, lr_end=2e-5, weight_decay=0.0, cg_weight=1.0, log=None,
          rank=0, world=1):
    """AdamW over contiguous batches of i.i.d. samples; cosine learning-rate decay.  Loss weights
    normalise each term by its target's mean square.  With world > 1 (one process per GPU, the
    same x, ty, tg on every rank) each rank trains on its slice of every global batch and the
    gradient is summed over the ranks before each AdamW step (dist.allreduce_gradient)."""
    import torch

    from .dist import allreduce_gradient, batch_slice
    N = x.shape[0]
    cy = 1.0 / max(float((ty.double() ** 2).mean().item()), 1e-30) / batch
    cgw = cg_weight / max(float((tg.double() ** 2).sum(1).mean().item()), 1e-30) / batch
    steps = epochs * max(1, N // batch)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    hist = []
    k = 0
    for ep in range(epochs):
        for s0 in range(0, N - batch + 1, batch):
            t = k / max(1, steps - 1)
            rate = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * t))
            a, b = batch_slice(s0, batch, rank, world)
            mlp.loss_grad(x[a:b], ty[a:b], tg[a:b], cy, cgw, loss)
            allreduce_gradient(mlp.grad_buffer() if world > 1 else None, world)
            mlp.adamw(rate, weight_decay=weight_decay)
            k += 1
        hist.append(float(loss.item()))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.3e}")
    mlp.check()
    return hist


def stress_errors(P_s, P_ref, floor):
    """Relative Frobenius stress errors |P_s - P_ref| / max(|P_ref|, floor) per point (host)."""
    P_s = np.asarray(P_s).reshape(-1, 9)
    P_ref = np.asarray(P_ref).reshape(-1, 9)
    return np.linalg.norm(P_s - P_ref, axis=1) / np.maximum(np.linalg.norm(P_ref, axis=1), floor)


class SurrogateDriver:
    """Load steps of a macro problem whose constitutive step is the surrogate with fallback:
    the surrogate gives Pbar, Abar at every point; points outside the trust region are replaced
    by full RVE solves (fehmm_select + fehmm_rve_solve_list), and every `audit_stride`-th point
    inside is also solved fully into separate arrays so that the surrogate's error is measured
    online.  All steps are library kernels."""

    def __init__(self, problem, mlp, sp, audit_stride=0, **options):
        import torch

        from . import select
        from .driver import LoadStepDriver
        self._select = select
        drv = LoadStepDriver(problem, **options)
        self.drv = drv
        self.mlp, self.sp = mlp, sp
        n = problem.n_qp
        dev = drv.u.device
        self.inside = torch.zeros(n, dtype=torch.int32, device=dev)
        self.work = torch.zeros(work_floats(n), dtype=torch.float32, device=dev)
        self.lst = torch.zeros(n, dtype=torch.int32, device=dev)
        self.cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        self.audit_stride = audit_stride
        if audit_stride:
            self.alst = torch.zeros(n, dtype=torch.int32, device=dev)
            self.acnt = torch.zeros(1, dtype=torch.int32, device=dev)
            self.Pa = torch.zeros_like(drv.P)
            self.Aa = torch.zeros_like(drv.A)
            self.sta = torch.zeros_like(drv.st)
            self.ita = torch.zeros_like(drv.it)
        drv._constitutive = self._constitutive
        self.fallback = []
        self.audit = []

    def _constitutive(self, first):
        from . import SOLVE_FROM_COMMITTED
        d = self.drv
        flags = SOLVE_FROM_COMMITTED if first else 0
        surrogate_eval(self.mlp, self.sp, d.F, d.P, d.A, None, self.inside, self.work)
        d.st.zero_()
        self._select(self.inside, 0, self.lst, self.cnt)
        d.ctx.rve_solve_list(d.F, d.P, d.A, d.st, d.it, flags, self.lst, self.cnt)
        if self.audit_stride:
            self._select(self.inside, 1, self.alst, self.acnt, stride=self.audit_stride)
            d.ctx.rve_solve_list(d.F, self.Pa, self.Aa, self.sta, self.ita, flags, self.alst, self.acnt)

    def audit_errors(self, floor):
        """Stress errors of the surrogate at the audited points of the last constitutive step."""
        k = int(self.acnt.item())
        idx = self.alst[:k].long()
        return stress_errors(self.drv.P[idx].cpu().numpy(), self.Pa[idx].cpu().numpy(), floor)

    def fallback_count(self):
        return int(self.cnt.item())
