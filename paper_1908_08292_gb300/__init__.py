"""Python binding of the GB300 batched FE-HMM / FE^2 RVE engine (libfehmm.so, include/fehmm.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  The binding fails loudly when the compiled
library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Context", "FehmmError", "lib", "library_path", "PREC_FP64", "PREC_MIXED", "PRECOND_JACOBI", "PRECOND_MG",
           "SOLVE_NO_TANGENT", "SOLVE_FROM_COMMITTED", "SOLVE_ENERGY", "RVE_STATUS"]

PREC_FP64, PREC_MIXED = 0, 1
PRECOND_JACOBI, PRECOND_MG = 0, 1
SOLVE_NO_TANGENT, SOLVE_FROM_COMMITTED, SOLVE_ENERGY = 1, 2, 4
RVE_STATUS = {0: "ok", 1: "newton_cap", 2: "J<=0", 3: "pcg_breakdown", 4: "nonfinite", 5: "pcg_cap"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def library_path() -> str:
    return os.path.join(_HERE, "libfehmm.so")


class FehmmError(RuntimeError):
    pass


class Options(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("precision", ctypes.c_int),
                ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("max_cg", ctypes.c_int),
                ("cond_rtol", ctypes.c_double), ("max_cond_cg", ctypes.c_int),
                ("retry_stages", ctypes.c_int), ("precond", ctypes.c_int),
                ("bc", ctypes.c_int), ("law", ctypes.c_int), ("mg_omega", ctypes.c_double),
                ("mg_reuse", ctypes.c_int), ("transfer_warm", ctypes.c_int)]


class TuneResult(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int), ("mg_omega", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("mg_reuse", ctypes.c_int), ("seconds_per_solve", ctypes.c_double), ("from_cache", ctypes.c_int),
                ("candidates", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "fehmm_default_options": (_I, [ctypes.POINTER(Options), _I, _I]),
    "fehmm_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Options)]),
    "fehmm_destroy": (_I, [_P]),
    "fehmm_get_options": (_I, [_P, ctypes.POINTER(Options)]),
    "fehmm_set_options": (_I, [_P, ctypes.POINTER(Options)]),
    "fehmm_add_rves": (_I, [_P, _I, _P, _P, _P, _P, _I, ctypes.POINTER(_I)]),
    "fehmm_bind_qps": (_I, [_P, _I, _P]),
    "fehmm_rve_solve": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "fehmm_commit": (_I, [_P, _P]),
    "fehmm_rollback": (_I, [_P, _P]),
    "fehmm_fluctuation": (_I, [_P, _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_I)]),
    "fehmm_fluctuation_all": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_longlong)]),
    "fehmm_transfer_state_all": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_longlong)]),
    "fehmm_macro_create": (_I, [_P, _P]),
    "fehmm_macro_qp_F": (_I, [_P, _P, _P, _P]),
    "fehmm_macro_assemble": (_I, [_P, _P, _P, _P, _P, _P]),
    "fehmm_macro_set_dirichlet": (_I, [_P, _I, _P, _P]),
    "fehmm_macro_apply_dirichlet": (_I, [_P, _P, _P, ctypes.c_double, _P]),
    "fehmm_macro_update": (_I, [_P, _P, _P, _P]),
    "fehmm_macro_dirichlet_load": (_I, [_P, _P, ctypes.c_double, _P, _P]),
    "fehmm_macro_solve": (_I, [_P, _P, _P, _P, _P, ctypes.c_double, _I, _P]),
    "fehmm_macro_csr": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "fehmm_launch_count": (ctypes.c_longlong, [_P]),
    "fehmm_autotune": (_I, [_P, _P, _I, ctypes.c_char_p, ctypes.POINTER(TuneResult), _P]),
    "fehmm_status_str": (ctypes.c_char_p, [_I]),
    "fehmm_rve_solve_list": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P]),
    "fehmm_select": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "fehmm_mlp_num_params": (_I, []),
    "fehmm_mlp_create": (_I, [ctypes.POINTER(_P), _I]),
    "fehmm_mlp_destroy": (_I, [_P]),
    "fehmm_mlp_set_params": (_I, [_P, _P]),
    "fehmm_mlp_get_params": (_I, [_P, _P, _P]),
    "fehmm_mlp_eval": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "fehmm_mlp_loss_grad": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, ctypes.c_float, _P, _P]),
    "fehmm_mlp_adamw": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "fehmm_mlp_launch_count": (ctypes.c_longlong, [_P]),
    "fehmm_mlp_check": (_I, [_P, ctypes.POINTER(_I)]),
    "fehmm_mlp_grad_buffer": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I)]),
    "fehmm_surrogate_save": (_I, [_P, _P, ctypes.c_char_p]),
    "fehmm_surrogate_base_law": (_I, [_P, _P]),
    "fehmm_surrogate_load": (_I, [_P, _P, ctypes.c_char_p]),
    "fehmm_surrogate_eval": (_I, [_P, _P, _P, _I, _P, _P, _P, _P, _P, _P]),
    "fehmm_surrogate_work_floats": (ctypes.c_size_t, [_I]),
    "fehmm_surrogate_targets": (_I, [_P, _P, _P, _P, _I, _P, _P, _P, _P]),
    "fehmm_surrogate_fit_poly": (_I, [_P, _P, _P, _P, _I, _I, _P]),
    "fehmm_rve2d_solve_fp64_noalloc": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Options), _P]),
}


def lib():
    """Load libfehmm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise FehmmError(f"{path} is missing: build it with `python -m paper_1908_08292_gb300.build`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def status_str(code: int) -> str:
    return lib().fehmm_status_str(int(code)).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise FehmmError(f"{what}: {status_str(rc)} ({rc})")
    return rc


def _dev(t, dtype, name, numel=None):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FehmmError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise FehmmError(f"{name} must be a contiguous {dtype} tensor")
    if numel is not None and t.numel() < numel:
        raise FehmmError(f"{name} has {t.numel()} elements, need {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def select(mask, value, out_list, out_count, stride=1, stream=None):
    """out_list[:out_count[0]] <- indices q with mask == value and q % stride == 0 (device, ascending)."""
    import torch
    _check(lib().fehmm_select(_dev(mask, torch.int32, "mask"), int(mask.numel()), int(value), int(stride),
                              _dev(out_list, torch.int32, "list", mask.numel()), _dev(out_count, torch.int32, "count", 1),
                              _stream(stream)), "select")


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


class Context:
    """One fehmm context: microstructures, per-qp fluctuation state and the macro mesh."""

    def __init__(self, dim: int, precision: str = "mixed", **options):
        L = lib()
        prec = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision]
        opt = Options()
        _check(L.fehmm_default_options(ctypes.byref(opt), dim, prec), "default_options")
        for k, v in options.items():
            if not hasattr(opt, k):
                raise FehmmError(f"unknown option {k}")
            setattr(opt, k, v)
        h = _P()
        _check(L.fehmm_create(ctypes.byref(h), ctypes.byref(opt)), "create")
        self._h = h
        self.dim = dim
        self.precision = precision
        self.n_qp = 0

    # -------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().fehmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- options
    @property
    def options(self) -> Options:
        opt = Options()
        _check(lib().fehmm_get_options(self._h, ctypes.byref(opt)), "get_options")
        return opt

    def set_options(self, **kw):
        opt = self.options
        for k, v in kw.items():
            setattr(opt, k, v)
        _check(lib().fehmm_set_options(self._h, ctypes.byref(opt)), "set_options")

    # -------------------------------------------------------- microstructure
    def add_rves(self, grid_n, phases, E, nu) -> int:
        grid_n = np.ascontiguousarray(grid_n, dtype=np.int32)
        phase = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.uint8).reshape(-1) for p in phases]))
        E = np.ascontiguousarray(E, dtype=np.float64)
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        if E.ndim != 2 or E.shape != nu.shape or E.shape[0] != grid_n.size:
            raise FehmmError("E and nu must have shape (n_rve, n_phase)")
        first = _I()
        _check(lib().fehmm_add_rves(self._h, int(grid_n.size), grid_n.ctypes.data, phase.ctypes.data,
                                    E.ctypes.data, nu.ctypes.data, int(E.shape[1]), ctypes.byref(first)),
               "add_rves")
        return first.value

    def bind_qps(self, rve_of_qp):
        r = np.ascontiguousarray(rve_of_qp, dtype=np.int32)
        _check(lib().fehmm_bind_qps(self._h, int(r.size), r.ctypes.data), "bind_qps")
        self.n_qp = int(r.size)

    # ------------------------------------------------------------ RVE solves
    def rve_solve(self, F, P, A=None, status=None, iters=None, W=None, flags=0, stream=None):
        import torch
        d, n = self.dim, self.n_qp
        _check(lib().fehmm_rve_solve(self._h, _dev(F, torch.float64, "F", n * d * d),
                                     _dev(P, torch.float64, "P", n * d * d),
                                     _dev(A, torch.float64, "A", n * d ** 4),
                                     _dev(W, torch.float64, "W", n),
                                     _dev(status, torch.int32, "status", n),
                                     _dev(iters, torch.int32, "iters", 4 * n), int(flags), _stream(stream)),
               "rve_solve")

    def rve_solve_list(self, F, P, A, status, iters, flags, qp_list, count, W=None, stream=None):
        """RVE solves for the quadrature points qp_list[:count[0]] (device int32 arrays)."""
        import torch
        d, n = self.dim, self.n_qp
        _check(lib().fehmm_rve_solve_list(self._h, _dev(F, torch.float64, "F", n * d * d),
                                          _dev(P, torch.float64, "P", n * d * d), _dev(A, torch.float64, "A"),
                                          _dev(W, torch.float64, "W"), _dev(status, torch.int32, "status", n),
                                          _dev(iters, torch.int32, "iters"), int(flags),
                                          _dev(qp_list, torch.int32, "qp_list"), _dev(count, torch.int32, "count", 1),
                                          _stream(stream)), "rve_solve_list")

    def commit(self, stream=None):
        _check(lib().fehmm_commit(self._h, _stream(stream)), "commit")

    def rollback(self, stream=None):
        _check(lib().fehmm_rollback(self._h, _stream(stream)), "rollback")

    def fluctuation(self, q: int, committed: bool = False):
        """Device view (torch float64, no copy) of quadrature point q's fluctuation field."""
        import torch
        ptr, n = _P(), _I()
        _check(lib().fehmm_fluctuation(self._h, int(q), int(committed), ctypes.byref(ptr), ctypes.byref(n)),
               "fluctuation")
        return torch.as_tensor(_DevArray(ptr.value, n.value, "<f8"), device="cuda")

    def autotune(self, F, n_sample=0, cache_path=None, stream=None) -> dict:
        """Time candidate solver settings on a sample of the bound points at Fbar = F and keep the
        fastest that converges (fehmm_autotune); returns the choice."""
        import torch
        r = TuneResult()
        _check(lib().fehmm_autotune(self._h, _dev(F, torch.float64, "F"), int(n_sample),
                                    cache_path.encode() if cache_path else None, ctypes.byref(r), _stream(stream)),
               "autotune")
        return r.as_dict()

    def fluctuations(self, committed: bool = False):
        """Device view (torch float64, no copy) of every point's fluctuation, concatenated."""
        import torch
        ptr, n = _P(), ctypes.c_longlong()
        _check(lib().fehmm_fluctuation_all(self._h, int(committed), ctypes.byref(ptr), ctypes.byref(n)),
               "fluctuation_all")
        return torch.as_tensor(_DevArray(ptr.value, n.value, "<f8"), device="cuda")

    def transfer_state(self, committed: bool = False):
        """Device view (torch uint8, no copy) of the kept tangent-transfer solutions, or None."""
        import torch
        ptr, n = _P(), ctypes.c_longlong()
        _check(lib().fehmm_transfer_state_all(self._h, int(committed), ctypes.byref(ptr), ctypes.byref(n)),
               "transfer_state_all")
        if not ptr.value or n.value == 0:
            return None
        return torch.as_tensor(_DevArray(ptr.value, n.value, "|u1"), device="cuda")

    # ------------------------------------------------------------------ macro
    def macro_create(self, n_el):
        arr = np.ascontiguousarray(n_el, dtype=np.int32)
        _check(lib().fehmm_macro_create(self._h, arr.ctypes.data), "macro_create")

    def macro_qp_F(self, u, F, stream=None):
        import torch
        _check(lib().fehmm_macro_qp_F(self._h, _dev(u, torch.float64, "u"), _dev(F, torch.float64, "F"),
                                      _stream(stream)), "macro_qp_F")

    def macro_assemble(self, P, A, f, K_vals, stream=None):
        import torch
        _check(lib().fehmm_macro_assemble(self._h, _dev(P, torch.float64, "P"), _dev(A, torch.float64, "A"),
                                          _dev(f, torch.float64, "f"), _dev(K_vals, torch.float64, "K_vals"),
                                          _stream(stream)), "macro_assemble")

    def macro_set_dirichlet(self, dofs, values):
        d = np.ascontiguousarray(dofs, dtype=np.int32)
        v = np.ascontiguousarray(values, dtype=np.float64)
        if v.shape != d.shape:
            raise FehmmError("dofs and values must have the same length")
        _check(lib().fehmm_macro_set_dirichlet(self._h, int(d.size), d.ctypes.data if d.size else None,
                                               v.ctypes.data if v.size else None), "macro_set_dirichlet")

    def macro_apply_dirichlet(self, u, du, scale, stream=None):
        import torch
        _check(lib().fehmm_macro_apply_dirichlet(self._h, _dev(u, torch.float64, "u"), _dev(du, torch.float64, "du"),
                                                 float(scale), _stream(stream)), "macro_apply_dirichlet")

    def macro_dirichlet_load(self, K_vals, dscale, g, stream=None):
        import torch
        _check(lib().fehmm_macro_dirichlet_load(self._h, _dev(K_vals, torch.float64, "K"), float(dscale),
                                                _dev(g, torch.float64, "g"), _stream(stream)), "macro_dirichlet_load")

    def macro_update(self, u, du, stream=None):
        import torch
        _check(lib().fehmm_macro_update(self._h, _dev(u, torch.float64, "u"), _dev(du, torch.float64, "du"),
                                        _stream(stream)), "macro_update")

    def macro_solve(self, K_vals, f, du, info, rtol=1e-12, max_it=20000, stream=None):
        """du = -K_ff^-1 f_f (du = 0 on Dirichlet dofs); info <- (|f_free|, iterations, status)."""
        import torch
        _check(lib().fehmm_macro_solve(self._h, _dev(K_vals, torch.float64, "K_vals"), _dev(f, torch.float64, "f"),
                                       _dev(du, torch.float64, "du"), _dev(info, torch.float64, "info", 3),
                                       float(rtol), int(max_it), _stream(stream)), "macro_solve")

    def macro_csr(self):
        """(rowptr, col, n_rows, nnz); rowptr/col are int32 device views owned by the context."""
        import torch
        rp, cl, nr, nz = _P(), _P(), _I(), _I()
        _check(lib().fehmm_macro_csr(self._h, ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(nr), ctypes.byref(nz)),
               "macro_csr")
        rowptr = torch.as_tensor(_DevArray(rp.value, nr.value + 1, "<i4"), device="cuda")
        col = torch.as_tensor(_DevArray(cl.value, nz.value, "<i4"), device="cuda")
        return rowptr, col, nr.value, nz.value

    @property
    def launches(self) -> int:
        return int(lib().fehmm_launch_count(self._h))
