"""Seeded synthetic inputs for the batched FE-HMM / FE^2 RVE problems.

This module produces INPUT DATA ONLY: microstructures (a phase id per micro
element), per-phase material constants (E, nu), macro mesh sizes, Dirichlet
data and load schedules, and random fields used by tests.  It contains none of
the method's arithmetic (no kinematics, constitutive law, assembly or solver)
and is shared, as data, by the FP64 oracle and by the CUDA path.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based hash:
draw j of stream `key` under seed `s` is splitmix64((s << 40) ^ (key << 12) ^ j).

Conventions shared with both sides:
  * RVE: periodic unit cell [0,1]^d split into n^d square/cube elements; element
    (i, j[, k]) has lexicographic index i + n*j (+ n*n*k) and centroid
    ((i+1/2)/n, ...).  A phase map is a uint8 array of length n^d in that order.
  * Phase assignment follows the pixel/voxel rule of the paper's image-based
    meshes (Sec. 6.3): an element belongs to an inclusion when its centroid lies
    inside it, measured with the periodic minimum-image distance; a centroid
    exactly on the surface counts as inside.
  * Macro mesh: [0,1]^d split into nx x ny (x nz) Q1/Hex8 elements; node
    (i, j[, k]) has index i + (nx+1)*j (+ (nx+1)*(ny+1)*k); dof = node*d + comp.
    Macro quadrature points are numbered element-major, Gauss-point-minor with
    the Gauss points in lexicographic order (xi fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 counters."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
    with np.errstate(over="ignore"):
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, key, count: int) -> np.ndarray:
    """`count` uniforms in [0,1) for each key (array of stream ids) -> shape (len(key), count)."""
    key = np.atleast_1d(np.asarray(key, dtype=np.uint64))
    j = np.arange(count, dtype=np.uint64)
    ctr = (np.uint64(seed) << np.uint64(40)) ^ (key[:, None] << np.uint64(12)) ^ j[None, :]
    return (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, key, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms (shape (len(key), count))."""
    m = (count + 1) // 2
    u = uniform(seed, key, 2 * m)
    u1 = 1.0 - u[:, 0::2]  # (0,1]
    u2 = u[:, 1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)], axis=1)
    return z[:, :count]


def phase_from_inclusions(n: int, dim: int, centers, radii) -> np.ndarray:
    """uint8 phase map (0 = matrix, 1 = inclusion) of an n^dim periodic grid.

    centers: (m, dim) inclusion centres in [0,1)^dim; radii: (m,) radii.
    """
    centers = np.atleast_2d(np.asarray(centers, dtype=np.float64))
    radii = np.atleast_1d(np.asarray(radii, dtype=np.float64))
    c1 = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([c1] * dim), indexing="ij")  # grids[0] varies with axis 0
    # lexicographic order: x fastest -> flatten with x as the last-varying axis
    pts = np.stack([g.transpose().reshape(-1) for g in grids], axis=1)  # (n^d, dim)
    inside = np.zeros(pts.shape[0], dtype=bool)
    for c, r in zip(centers, radii):
        d = pts - c[None, :]
        d -= np.round(d)  # periodic minimum image
        inside |= (d * d).sum(axis=1) <= r * r
    return inside.astype(np.uint8)


@dataclass
class Problem:
    """One synthetic FE-HMM workload (all arrays are host numpy)."""
    name: str
    dim: int
    macro_n: tuple            # elements per axis of the macro mesh on [0,1]^d
    rve_n: np.ndarray         # (n_rve,) micro grid size per microstructure
    rve_phase: list           # n_rve uint8 arrays of length rve_n^dim
    rve_E: np.ndarray         # (n_rve, n_phase) Young's moduli
    rve_nu: np.ndarray        # (n_rve, n_phase) Poisson ratios
    qp_rve: np.ndarray        # (n_qp,) microstructure used at each macro quadrature point
    dirichlet_dofs: np.ndarray    # macro dofs with prescribed displacement
    dirichlet_end: np.ndarray     # their values at the end of loading (scaled by k/n_steps)
    n_steps: int
    precision: str            # "fp64" or "mixed"
    newton_tol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def n_qp(self) -> int:
        return int(self.qp_rve.shape[0])


def _macro_nodes(macro_n):
    dim = len(macro_n)
    axes = [np.arange(m + 1) / m for m in macro_n]
    g = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.transpose().reshape(-1) for a in g], axis=1)  # node index: x fastest


def _affine_bc(macro_n, F_end, on_node):
    X = _macro_nodes(macro_n)
    dim = len(macro_n)
    sel = np.nonzero(on_node(X))[0]
    H = np.asarray(F_end, dtype=np.float64) - np.eye(dim)
    vals = X[sel] @ H.T  # u = (F - I) X
    dofs = (sel[:, None] * dim + np.arange(dim)[None, :]).reshape(-1)
    return dofs.astype(np.int64), vals.reshape(-1)


def _uniaxial_rollers(macro_n, stretch):
    """Symmetry rollers u_a = 0 on X_a = 0 for every axis a; u_x = stretch on X_x = 1."""
    X = _macro_nodes(macro_n)
    dim = len(macro_n)
    dofs, vals = [], []
    for a in range(dim):
        nodes = np.nonzero(np.isclose(X[:, a], 0.0))[0]
        dofs.append(nodes * dim + a)
        vals.append(np.zeros(nodes.size))
    nodes = np.nonzero(np.isclose(X[:, 0], 1.0))[0]
    dofs.append(nodes * dim + 0)
    vals.append(np.full(nodes.size, stretch))
    dofs = np.concatenate(dofs)
    vals = np.concatenate(vals)
    order = np.argsort(dofs, kind="stable")
    return dofs[order].astype(np.int64), vals[order]


def uniaxial_2d_small() -> Problem:
    """2D plane strain, 4x4 Q1 macro (64 qps), one 8x8 RVE with a centred circle r = 0.25."""
    phase = phase_from_inclusions(8, 2, [[0.5, 0.5]], [0.25])
    dofs, vals = _uniaxial_rollers((4, 4), 0.1)
    return Problem("c1_2d_fp64_4x4_rve8", 2, (4, 4), np.array([8]), [phase],
                   np.array([[1.0, 10.0]]), np.array([[0.3, 0.3]]),
                   np.zeros(64, dtype=np.int64), dofs, vals, 10, "fp64", 1e-10)


def biaxial_shear_2d(macro: int = 32, rve: int = 32, seed: int = 1002, n_rve: int | None = None,
            macro_y: int | None = None) -> Problem:
    """2D batch: macro macro x macro_y (default square) Q1 on the unit square (4 qps/element, one
    RVE each) of rve x rve RVEs, random circle (centre uniform, r ~ U(0.15, 0.35)), stiffness
    ratio log-uniform in [5, 50].  A taller mesh (macro_y = k macro) keeps the first RVEs of the
    square workload and adds k - 1 times as many (weak scaling over k ranks)."""
    macro_y = macro if macro_y is None else macro_y
    n_qp = macro * macro_y * 4
    n_rve = n_qp if n_rve is None else n_rve
    u = uniform(seed, np.arange(n_rve), 4)
    centers = u[:, 0:2]
    radii = 0.15 + 0.20 * u[:, 2]
    ratio = np.exp(np.log(5.0) + (np.log(50.0) - np.log(5.0)) * u[:, 3])
    phases = [phase_from_inclusions(rve, 2, centers[i:i + 1], radii[i:i + 1]) for i in range(n_rve)]
    E = np.stack([np.ones(n_rve), ratio], axis=1)
    nu = np.full((n_rve, 2), 0.3)
    F_end = [[1.3, 0.3], [0.0, 1.3]]
    dofs, vals = _affine_bc((macro, macro_y), F_end,
                            lambda X: np.isclose(X, 0.0).any(1) | np.isclose(X, 1.0).any(1))
    qp_rve = np.arange(n_qp) % n_rve
    return Problem(f"c2_2d_mixed_{macro}x{macro_y}_rve{rve}", 2, (macro, macro_y),
                   np.full(n_rve, rve), phases, E, nu, qp_rve, dofs, vals, 20, "mixed", 1e-10,
                   extra={"centers": centers, "radii": radii, "ratio": ratio, "F_end": np.array(F_end)})


def sphere_rve(n: int, n_incl: int, phi: float, centers) -> np.ndarray:
    r = (3.0 * phi / (4.0 * np.pi * n_incl)) ** (1.0 / 3.0)
    return phase_from_inclusions(n, 3, centers, np.full(n_incl, r))


def uniaxial_3d_uneven(macro: int = 8, seed: int = 1003, sizes=(8, 12, 16), n_rve: int | None = None) -> Problem:
    """3D uneven batch: macro macro^3 Hex8 (8 qps/element, one RVE each); RVE n drawn from
    `sizes`, 1-4 spherical inclusions, volume fraction U(0.1, 0.3), stiffness ratio 10."""
    n_qp = macro ** 3 * 8
    n_rve = n_qp if n_rve is None else n_rve
    u = uniform(seed, np.arange(n_rve), 3 + 12)
    ns = np.array(sizes)[np.minimum((u[:, 0] * len(sizes)).astype(int), len(sizes) - 1)]
    n_incl = 1 + np.minimum((u[:, 1] * 4).astype(int), 3)
    phi = 0.1 + 0.2 * u[:, 2]
    phases = []
    for i in range(n_rve):
        c = u[i, 3:3 + 3 * n_incl[i]].reshape(n_incl[i], 3)
        phases.append(sphere_rve(int(ns[i]), int(n_incl[i]), float(phi[i]), c))
    E = np.tile([1.0, 10.0], (n_rve, 1))
    nu = np.full((n_rve, 2), 0.3)
    dofs, vals = _uniaxial_rollers((macro, macro, macro), 0.2)
    qp_rve = np.arange(n_qp) % n_rve
    return Problem(f"c3_3d_mixed_{macro}^3_rve8-12-16", 3, (macro,) * 3, ns, phases, E, nu,
                   qp_rve, dofs, vals, 10, "mixed", 1e-10,
                   extra={"n_incl": n_incl, "phi_target": phi})


def fixed_rve12(seed: int = 1004, n: int = 12) -> tuple:
    """The fixed two-inclusion microstructure (the 3D workload generator, n_incl = 2) on an n^3 grid
    (12^3 in the workloads; smaller grids of the same geometry serve quick tests)."""
    u = uniform(seed, np.array([0]), 7)[0]
    phi = 0.1 + 0.2 * u[0]
    return sphere_rve(n, 2, phi, u[1:7].reshape(2, 3)), phi


def cantilever_3d_fixed_rve(macro: int = 16) -> Problem:
    """3D large macro: macro^3 Hex8 (8 qps/element), all with the fixed 12^3 RVE; clamped at
    x = 0, u = (F - I) X at x = 1 with F_end - I = 0.35 (e1 x e1 + e1 x e2)/sqrt(2)."""
    phase, phi = fixed_rve12()
    H = np.zeros((3, 3))
    H[0, 0] = H[0, 1] = 0.35 / math.sqrt(2.0)
    F_end = np.eye(3) + H
    X = _macro_nodes((macro,) * 3)
    left = np.nonzero(np.isclose(X[:, 0], 0.0))[0]
    dl = (left[:, None] * 3 + np.arange(3)[None, :]).reshape(-1)
    dr, vr = _affine_bc((macro,) * 3, F_end, lambda X: np.isclose(X[:, 0], 1.0))
    dofs = np.concatenate([dl, dr])
    vals = np.concatenate([np.zeros(dl.size), vr])
    order = np.argsort(dofs, kind="stable")
    n_qp = macro ** 3 * 8
    return Problem(f"c5_3d_{macro}^3_rve12", 3, (macro,) * 3, np.array([12]), [phase],
                   np.array([[1.0, 10.0]]), np.array([[0.3, 0.3]]),
                   np.zeros(n_qp, dtype=np.int64), dofs[order].astype(np.int64), vals[order],
                   20, "mixed", 1e-10, extra={"phi": phi, "F_end": F_end})


def box_inclusion(n: int, dim: int, lo: float = 0.25, hi: float = 0.75) -> np.ndarray:
    """uint8 phase map of an axis-aligned box inclusion [lo, hi)^dim on an n^dim grid (element
    centroid rule).  With lo, hi multiples of 1/n the pixelised geometry is exact, so a sequence
    of grids n = 4, 8, 16, ... refines one and the same microstructure (mesh-convergence studies)."""
    c1 = (np.arange(n) + 0.5) / n
    inside1 = (c1 >= lo) & (c1 < hi)
    grids = np.meshgrid(*([inside1] * dim), indexing="ij")
    inside = np.logical_and.reduce([g.transpose().reshape(-1) for g in grids])
    return inside.astype(np.uint8)


def stretch_ball(seed: int, count: int, radius: float = 0.3, first: int = 0) -> np.ndarray:
    """`count` symmetric right stretch tensors U (count, 3, 3) uniform in the 6-D ball
    ||U - I||_F <= radius (off-diagonal components carry the sqrt(2) weight)."""
    keys = np.arange(first, first + count)
    z = normal(seed, keys, 6)
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    rad = radius * uniform(seed + 7919, keys, 1)[:, 0] ** (1.0 / 6.0)
    v = z * rad[:, None]
    U = np.repeat(np.eye(3)[None], count, axis=0)
    U[:, 0, 0] += v[:, 0]
    U[:, 1, 1] += v[:, 1]
    U[:, 2, 2] += v[:, 2]
    s = 1.0 / math.sqrt(2.0)
    for (a, b), c in zip(((0, 1), (0, 2), (1, 2)), (3, 4, 5)):
        U[:, a, b] += s * v[:, c]
        U[:, b, a] += s * v[:, c]
    return U


def random_F(seed: int, count: int, dim: int, scale: float = 0.1, key0: int = 0) -> np.ndarray:
    """Deformation gradients I + scale * (uniform(-1, 1) matrix), shape (count, dim, dim)."""
    u = uniform(seed, np.arange(key0, key0 + count), dim * dim)
    return np.eye(dim)[None] + scale * (2.0 * u - 1.0).reshape(count, dim, dim)


def random_field(seed: int, count: int, length: int, scale: float = 1.0, key0: int = 0) -> np.ndarray:
    """Uniform(-scale, scale) arrays of shape (count, length)."""
    return scale * (2.0 * uniform(seed, np.arange(key0, key0 + count), length) - 1.0)
