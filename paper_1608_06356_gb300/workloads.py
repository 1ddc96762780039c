"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code shared by the CUDA path and the CPU oracle in
the tests: it draws particle ensembles and fields with numpy and holds none
of the method's arithmetic.  Every generator takes a seed and returns host
(numpy, float64) arrays; callers cast to the precision they run in.

Recipes (units: momentum m_e c, fields m_e c omega0 / e, a_S = 412148.45):
  single      n electrons, gamma0 along x, uniform B along z, E = 0
              (the paper's single-particle-type test: gamma0 = 1000, B = 410,
              so chi_e ~ 1)
  ensemble    gamma log-uniform in [g_lo, g_hi], isotropic directions;
              per-particle E and B with independent isotropic directions and
              |E|, |B| log-uniform in [f_lo, f_hi] (chi ~ 0.01 .. 10)
  chi_target  gamma log-uniform, isotropic p; B perpendicular to p with
              |B| = chi a_S / |p| for chi log-uniform in [chi_lo, chi_hi]; E = 0
  cascade     electrons at rest, uniform in the central block of a periodic
              grid (the 3D PIC-like cascade seed)
  batched     run sizes log-uniform in [1e3, 1e6]; per-run chi ranges from
              two sorted log-uniform draws in [0.01, 10]
"""
from __future__ import annotations

import numpy as np

A_S_1UM = 412148.45


def _iso(rng, n):
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2 * np.pi, n)
    s = np.sqrt(1.0 - mu * mu)
    return np.stack([s * np.cos(phi), s * np.sin(phi), mu])


def _loguniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def single(n=10_000, gamma0=1000.0, B=410.0):
    p = np.sqrt(gamma0**2 - 1.0)
    z = np.zeros(n)
    return dict(x=z.copy(), y=z.copy(), z=z.copy(), px=np.full(n, p), py=z.copy(), pz=z.copy(),
                w=np.ones(n), id=np.arange(n, dtype=np.uint64)), dict(E=(0.0, 0.0, 0.0), B=(0.0, 0.0, B))


def ensemble(n, seed=0, g_lo=1e2, g_hi=1e4, f_lo=10.0, f_hi=2000.0, photons=False, id0=0):
    """Leptons (photons=False: |p| = sqrt(gamma^2-1)) or photons (|p| = gamma)."""
    rng = np.random.default_rng(seed)
    g = _loguniform(rng, g_lo, g_hi, n)
    d = _iso(rng, n)
    pm = g if photons else np.sqrt(g * g - 1.0)
    Ed = _iso(rng, n) * _loguniform(rng, f_lo, f_hi, n)
    Bd = _iso(rng, n) * _loguniform(rng, f_lo, f_hi, n)
    pos = rng.uniform(-1.0, 1.0, (3, n))
    return dict(x=pos[0], y=pos[1], z=pos[2], px=pm * d[0], py=pm * d[1], pz=pm * d[2],
                w=np.ones(n), id=np.arange(id0, id0 + n, dtype=np.uint64),
                ex=Ed[0], ey=Ed[1], ez=Ed[2], bx=Bd[0], by=Bd[1], bz=Bd[2])


def chi_target(n, seed=0, chi_lo=1e-3, chi_hi=1e2, g_lo=1e2, g_hi=1e4, a_S=A_S_1UM, id0=0):
    rng = np.random.default_rng(seed)
    chi = _loguniform(rng, chi_lo, chi_hi, n)
    g = _loguniform(rng, g_lo, g_hi, n)
    d = _iso(rng, n)
    pm = np.sqrt(g * g - 1.0)
    r = _iso(rng, n)
    b = r - d * (r * d).sum(0)  # component of a random direction perpendicular to p
    b /= np.linalg.norm(b, axis=0)
    Bm = chi * a_S / pm
    z = np.zeros(n)
    return dict(x=z.copy(), y=z.copy(), z=z.copy(), px=pm * d[0], py=pm * d[1], pz=pm * d[2],
                w=np.ones(n), id=np.arange(id0, id0 + n, dtype=np.uint64),
                ex=z.copy(), ey=z.copy(), ez=z.copy(), bx=Bm * b[0], by=Bm * b[1], bz=Bm * b[2]), chi, g


def cascade_seed(n, seed=0, nx=256, dx=2 * np.pi / 32, block=64):
    """n electrons at rest, uniform in the central block^3 cells of an nx^3 grid."""
    rng = np.random.default_rng(seed)
    lo = (nx - block) / 2 * dx
    pos = rng.uniform(lo, lo + block * dx, (3, n))
    z = np.zeros(n)
    return dict(x=pos[0], y=pos[1], z=pos[2], px=z.copy(), py=z.copy(), pz=z.copy(), w=np.ones(n),
                id=np.arange(n, dtype=np.uint64))


def batched_runs(n_runs=256, seed=0, lo=1e3, hi=1e6, chi_lo=0.01, chi_hi=10.0):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n_runs))).astype(np.int64)
    ranges = np.sort(_loguniform(rng, chi_lo, chi_hi, (n_runs, 2)), axis=1)
    return sizes, ranges


def uniform_words(n, seed=0):
    """Uniform 32-bit words (inputs to the inverse-CDF parity checks)."""
    return np.random.default_rng(seed).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


def plasma(nx, ny, nz, dx, ppc=1, density=0.01, p_th=0.0, drift=(0.0, 0.0, 0.0), seed=0,
           lattice=False, id0=0, cell_order=False):
    """Electrons filling a periodic box of nx*ny*nz cubic cells of side dx at
    `density` (units of the critical density) with weights density dx^3 / ppc:
    ppc per cell, at uniform random positions (lattice=True: one at each cell
    centre), momenta normal with deviation p_th per axis plus `drift`.
    cell_order=True stores them by cell (z, then y, then x), the order a PIC
    code's periodic particle sort keeps; ids follow the storage order."""
    rng = np.random.default_rng(seed)
    cells = nx * ny * nz
    if lattice:
        assert ppc == 1
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        pos = [((a + 0.5) * dx).ravel() for a in (i, j, k)]
    else:
        box = (nx * dx, ny * dx, nz * dx)
        pos = [rng.uniform(0.0, L, cells * ppc) for L in box]
    n = cells * ppc
    if cell_order and not lattice:
        cell = [np.floor(pos[a] / dx).astype(np.int64) for a in range(3)]
        o = np.argsort((cell[2] * ny + cell[1]) * nx + cell[0], kind="stable")
        pos = [q[o] for q in pos]
    p = rng.normal(0.0, 1.0, (3, n)) * p_th + np.asarray(drift, dtype=np.float64)[:, None]
    return dict(x=pos[0], y=pos[1], z=pos[2], px=p[0], py=p[1], pz=p[2],
                w=np.full(n, density * dx ** 3 / ppc), id=np.arange(id0, id0 + n, dtype=np.uint64))
