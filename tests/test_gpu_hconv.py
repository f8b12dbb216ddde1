"""Micro mesh convergence on the GPU (Sec. 4 a-priori estimates; the micro-convergence studies of
Sec. 6) for a microstructure every grid resolves exactly (a box inclusion [0.25, 0.75)^d): the
homogenised tangent of grids n = 4, 8, 16 approaches the finest grid's monotonically, periodic and
KUBC; the coarse grids match the FP64 oracle; and the KUBC-periodic gap (the modelling error of
Eq. ModelingError) shrinks on k x k tilings of one cell while the periodic result does not
depend on the tiling."""
import numpy as np
import pytest

import synth
from gpu_harness import gpu_batch, rel_err
from oracle.kubc import DirichletRVE
from oracle.rve import PeriodicRVE

pytestmark = pytest.mark.gpu

STRICT = dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-12)
F2 = np.array([[1.12, 0.06], [0.03, 0.95]])
F3 = np.array([[1.10, 0.05, 0.0], [0.02, 0.96, 0.03], [0.0, 0.01, 0.97]])


@pytest.mark.parametrize("dim,bc", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_h_convergence_of_the_tangent(dim, bc):
    ns = [4, 8, 16, 32] if dim == 2 else [4, 8, 16]
    F = F2 if dim == 2 else F3
    phases = [synth.box_inclusion(n, dim) for n in ns]
    out = gpu_batch(dim, "fp64", ns, phases, [[1.0, 10.0]] * len(ns), [[0.3, 0.3]] * len(ns),
                    np.arange(len(ns)), np.stack([F] * len(ns)), bc=bc, **STRICT)
    assert (out["status"] == 0).all()
    eA = [rel_err(out["A"][k], out["A"][-1], 1e-3) for k in range(len(ns) - 1)]
    assert all(eA[k + 1] < eA[k] for k in range(len(eA) - 1)), eA
    # the coarsest two grids against the oracle
    cls = DirichletRVE if bc else PeriodicRVE
    for k in (0, 1):
        ref = cls(ns[k], dim, phases[k], [1.0, 10.0], [0.3, 0.3]).solve(F, rtol=1e-14, atol=1e-16)
        assert rel_err(out["P"][k], ref["P"], 1e-3) < 1e-10 and rel_err(out["A"][k], ref["A"], 1e-3) < 1e-10


def test_kubc_modelling_error_shrinks_with_the_tiling():
    ks = [1, 2, 4]
    cell = synth.box_inclusion(8, 2).reshape(8, 8)
    tiles = [np.tile(cell, (k, k)).reshape(-1) for k in ks]
    args = ([8 * k for k in ks], tiles, [[1.0, 10.0]] * 3, [[0.3, 0.3]] * 3, np.arange(3), np.stack([F2] * 3))
    per = gpu_batch(2, "fp64", *args, **STRICT)
    kub = gpu_batch(2, "fp64", *args, bc=1, **STRICT)
    gap = [rel_err(kub["A"][j], per["A"][j], 1e-3) for j in range(3)]
    assert gap[0] > gap[1] > gap[2] > 0, gap
    for j in (1, 2):  # periodic coupling: the k x k tiling is the same problem
        assert rel_err(per["A"][j], per["A"][0], 1e-3) < 1e-9
