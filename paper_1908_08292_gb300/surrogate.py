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
SQ2 = math.sqrt(2.0)
MANDEL = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


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


def init_params(seed: int) -> dict:
    """He-uniform weights from the SplitMix64 input generator, zero biases."""
    import synth
    p = {}
    fan = [N_IN, WIDTH, WIDTH, WIDTH]
    for l in range(4):
        b = math.sqrt(6.0 / fan[l])
        p[f"W{l + 1}"] = b * (2 * synth.uniform(seed, np.arange(WIDTH) + 1000 * l, fan[l]) - 1)
        p[f"b{l + 1}"] = np.zeros(WIDTH)
    p["w5"] = math.sqrt(3.0 / WIDTH) * (2 * synth.uniform(seed, np.array([999999]), WIDTH)[0] - 1)
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


class SurrogateParams(ctypes.Structure):
    _fields_ = [("lam0", ctypes.c_double), ("mu0", ctypes.c_double), ("sx", ctypes.c_double),
                ("sg", ctypes.c_double), ("radius", ctypes.c_double)]


def surrogate_eval(mlp: MLP, sp: SurrogateParams, F, P, A, W, inside, work, stream=None):
    import torch
    n = F.shape[0]
    _check(lib().fehmm_surrogate_eval(mlp._h, ctypes.byref(sp), _dev(F, torch.float64, "F", 9 * n), n,
                                      _dev(P, torch.float64, "P", 9 * n), _dev(A, torch.float64, "A"),
                                      _dev(W, torch.float64, "W"), _dev(inside, torch.int32, "inside", n),
                                      _dev(work, torch.float32, "work", work_floats(n)), _stream(stream)),
           "surrogate_eval")


def work_floats(n: int) -> int:
    return int(lib().fehmm_surrogate_work_floats(int(n)))


def isotropic_projection(A):
    """(lam, mu) of the isotropic part of a fourth-order tangent A[3,3,3,3]:
    3K = A_iijj / 3, mu = (A_ijij - A_iijj / 3) / 10, lam = K - 2 mu / 3."""
    A = np.asarray(A).reshape(3, 3, 3, 3)
    iijj = np.einsum("iijj->", A)
    ijij = np.einsum("ijij->", A)
    K = iijj / 9.0
    mu = (ijij - iijj / 3.0) / 10.0
    return K - 2.0 * mu / 3.0, mu


def surrogate_targets(sp: SurrogateParams, F, P, W, x, ty, tg, stream=None):
    import torch
    n = F.shape[0]
    _check(lib().fehmm_surrogate_targets(ctypes.byref(sp), _dev(F, torch.float64, "F", 9 * n),
                                         _dev(P, torch.float64, "P", 9 * n), _dev(W, torch.float64, "W", n), n,
                                         _dev(x, torch.float32, "x", 6 * n), _dev(ty, torch.float32, "ty", n),
                                         _dev(tg, torch.float32, "tg", 6 * n), _stream(stream)), "surrogate_targets")
