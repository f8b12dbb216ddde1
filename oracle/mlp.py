"""FP64 reference of the energy-surrogate MLP (oracle; test infrastructure only).

Network (the learned part of the workload, not in the paper): x in R^6 -> 4 hidden layers of 128
SiLU units -> scalar,
    z1 = W1 x + b1, a_l = silu(z_l), z_{l+1} = W_{l+1} a_l + b_{l+1} (l = 1..3), y = w5 . a4 + b5.
Provided here, all in float64 and written out layer by layer:
  * forward y(x);
  * input gradient dy/dx (reverse mode): d4 = w5 * silu'(z4), d_l = (W_{l+1}^T d_{l+1}) * silu'(z_l),
    dy/dx = W1^T d1;
  * input Hessian d2y/dx2 (forward mode over the reverse pass, one input direction at a time);
  * the training loss L = 1/2 sum_b [cy (y_b - ty_b)^2 + cg |dy/dx_b - tg_b|^2] and its exact
    gradient with respect to every parameter (reverse mode through both the forward pass and
    the input-gradient pass: the "double backward").
Option `bf16=True` rounds the weights and both operands of every matrix product (x, a_1..a_4,
the backward and double-backward vectors) to bfloat16 (round to nearest even), the points where
the CUDA kernels store bfloat16 for their tensor-core products; sums over the batch for the
bias and output-weight gradients stay in full precision.
Pins (tests/test_oracle_mlp.py): central finite differences of y -> dy/dx, of dy/dx -> Hessian,
of L -> parameter gradient.
"""
from __future__ import annotations

import numpy as np

WIDTH, DEPTH, N_IN = 128, 4, 6


def to_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_d(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def silu_dd(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


def init_params(seed, width=WIDTH, depth=DEPTH, n_in=N_IN):
    """He-style uniform initialisation from the SplitMix64 generator (deterministic)."""
    import synth
    sizes = [n_in] + [width] * depth
    params = {}
    for l in range(depth):
        fan_in = sizes[l]
        bound = np.sqrt(6.0 / fan_in)
        params[f"W{l + 1}"] = bound * (2 * synth.uniform(seed, np.arange(width) + 1000 * l, fan_in) - 1)
        params[f"b{l + 1}"] = np.zeros(width)
    params["w5"] = np.sqrt(3.0 / width) * (2 * synth.uniform(seed, np.array([999999]), width)[0] - 1)
    params["b5"] = np.zeros(1)
    return params


def _q(a, bf16):
    return to_bf16(a) if bf16 else np.asarray(a, dtype=np.float64)


def forward(params, x, bf16=False):
    """y (B,) and the cache of pre-activations z_l (B, 128) and activations a_l."""
    zs, As = [], []
    a = _q(x, bf16)
    for l in range(DEPTH):
        W = _q(params[f"W{l + 1}"], bf16)
        z = a @ W.T + params[f"b{l + 1}"]
        zs.append(z)
        a = _q(silu(z), bf16)
        As.append(a)
    y = a @ _q(params["w5"], bf16) + params["b5"][0]
    return y, {"x": _q(x, bf16), "z": zs, "a": As}


def input_grad(params, x, bf16=False):
    y, c = forward(params, x, bf16)
    d = _q(params["w5"], bf16)[None, :] * silu_d(c["z"][-1])
    ds = [d]
    for l in range(DEPTH - 1, 0, -1):
        W = _q(params[f"W{l + 1}"], bf16)
        d = (_q(d, bf16) @ W) * silu_d(c["z"][l - 1])
        ds.append(d)
    ds = ds[::-1]  # d_1 .. d_4
    g = _q(ds[0], bf16) @ _q(params["W1"], bf16)
    return y, g, c, ds


def input_hessian(params, x, bf16=False):
    """(B, 6, 6) Hessian by forward-mode differentiation of the input-gradient pass."""
    y, g, c, ds = input_grad(params, x, bf16)
    B = x.shape[0]
    H = np.zeros((B, N_IN, N_IN))
    Ws = [_q(params[f"W{l + 1}"], bf16) for l in range(DEPTH)]
    w5 = _q(params["w5"], bf16)
    for k in range(N_IN):
        # tangents of z_l along e_k
        zd = [np.broadcast_to(Ws[0][:, k], (B, WIDTH)).copy()]
        for l in range(1, DEPTH):
            ad = silu_d(c["z"][l - 1]) * zd[l - 1]
            zd.append(_q(ad, bf16) @ Ws[l].T)
        # tangent of the backward pass
        dd = w5[None, :] * silu_dd(c["z"][-1]) * zd[-1]
        for l in range(DEPTH - 1, 0, -1):
            back = _q(ds[l], bf16) @ Ws[l]
            dd = (_q(dd, bf16) @ Ws[l]) * silu_d(c["z"][l - 1]) + back * silu_dd(c["z"][l - 1]) * zd[l - 1]
        H[:, :, k] = _q(dd, bf16) @ Ws[0]
    return y, g, H


def loss(params, x, ty, tg, cy, cg, bf16=False):
    y, g, _, _ = input_grad(params, x, bf16)
    return 0.5 * (cy * ((y - ty) ** 2).sum() + cg * ((g - tg) ** 2).sum())


def param_grad(params, x, ty, tg, cy, cg, bf16=False):
    """Exact gradient of `loss` with respect to all parameters (reverse mode through the forward
    pass and the input-gradient pass)."""
    y, g, c, ds = input_grad(params, x, bf16)
    Ws = [_q(params[f"W{l + 1}"], bf16) for l in range(DEPTH)]
    w5 = _q(params["w5"], bf16)
    z, A, xq = c["z"], c["a"], c["x"]
    grads = {k: np.zeros_like(v) for k, v in params.items()}
    ry = cy * (y - ty)          # dL/dy            (B,)
    rg = cg * (g - tg)          # dL/d(dy/dx)      (B, 6)
    # ---- reverse through the input-gradient pass: g = W1^T d1, d_l = (W_{l+1}^T d_{l+1}) s'(z_l)
    e = _q(rg, bf16) @ Ws[0].T  # dL/dd_1          (B, 128)
    grads["W1"] += _q(ds[0], bf16).T @ _q(rg, bf16)
    qz = [None] * DEPTH         # direct adjoints of z_l through s'(z_l)
    for l in range(1, DEPTH):   # d_l = c_l * s'(z_l), c_l = W_{l+1}^T d_{l+1}
        cvec = _q(ds[l], bf16) @ Ws[l]
        qz[l - 1] = e * cvec * silu_dd(z[l - 1])
        es = e * silu_d(z[l - 1])            # dL/dc_l
        grads[f"W{l + 1}"] += _q(ds[l], bf16).T @ _q(es, bf16)   # c_l = W^T d: dc/dW
        e = _q(es, bf16) @ Ws[l].T                             # dL/dd_{l+1}
    # d_4 = w5 * s'(z_4)
    grads["w5"] += (e * silu_d(z[-1])).sum(0)
    qz[DEPTH - 1] = e * w5[None, :] * silu_dd(z[-1])
    # ---- reverse through the forward pass, adding the direct adjoints qz
    grads["w5"] += A[-1].T @ ry
    grads["b5"][0] += ry.sum()
    dz = ry[:, None] * w5[None, :] * silu_d(z[-1]) + qz[-1]
    for l in range(DEPTH - 1, -1, -1):
        a_prev = xq if l == 0 else A[l - 1]
        grads[f"W{l + 1}"] += _q(dz, bf16).T @ a_prev
        grads[f"b{l + 1}"] += dz.sum(0)
        if l > 0:
            dz = (_q(dz, bf16) @ Ws[l]) * silu_d(z[l - 1]) + qz[l - 1]
    return grads
