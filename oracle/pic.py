"""FP64 numpy oracle of the particle-in-cell loop around the QED step.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code allowed to import this module.
It shares no code with the CUDA path.

The paper adds its QED module to a PIC code (introduction) without describing
that code's field solver or current deposition.  What this module computes is
the textbook explicit scheme the library implements for that loop, written
out plainly with whole-array numpy operations:

  * Maxwell's equations in the paper's units (time 1/omega0, length c/omega0,
    fields m_e c omega0/e, current e n_c c with n_c the critical density):
        dB/dt = -curl E,        dE/dt = curl B - J,
    on Yee's staggered grid (K. S. Yee, IEEE Trans. Antennas Propag. 14, 302
    (1966)), periodic, node (i, j, k) at (x0 + i dx, y0 + j dy, z0 + k dz):
        Ex, Jx at (i+1/2, j, k)     Bx at (i, j+1/2, k+1/2)
        Ey, Jy at (i, j+1/2, k)     By at (i+1/2, j, k+1/2)
        Ez, Jz at (i, j, k+1/2)     Bz at (i+1/2, j+1/2, k)
    arrays indexed [k, j, i];
  * the leapfrog step from time n to n+1 with J at n+1/2:
        B -= dt/2 curl E;   E += dt (curl B - J);   B -= dt/2 curl E;
  * the node values the particle gather reads: each E component the mean of
    its two staggered neighbours along its own axis, each B component the
    mean of its four neighbours in the plane normal to it;
  * the current of a particle of charge q and weight w: q w weight_unit v /
    (dx dy dz) with v = p/gamma, at the mid-step position x - v dt/2, spread
    over the 2 x 2 x 2 staggered J positions around it with the linear (CIC)
    weights.

Pins (tests/test_oracle_pic.py): the exact discrete plane wave of the Yee
scheme (dispersion sin(w dt/2) = (dt/d) sin(k d/2)) along each axis and
polarisation, nodes of that wave in closed form, a uniform current draining
E linearly, the deposit against a direct evaluation of the CIC hat function
at every staggered position, and the cold-plasma oscillation of the whole
loop (with the oracle's QED step) against its closed-form frequency.
"""
from __future__ import annotations

import numpy as np

# staggered offset (in cells) of each array along (x, y, z)
OFFSETS = {
    "ex": (0.5, 0.0, 0.0), "ey": (0.0, 0.5, 0.0), "ez": (0.0, 0.0, 0.5),
    "bx": (0.0, 0.5, 0.5), "by": (0.5, 0.0, 0.5), "bz": (0.5, 0.5, 0.0),
    "jx": (0.5, 0.0, 0.0), "jy": (0.0, 0.5, 0.0), "jz": (0.0, 0.0, 0.5),
}
AXIS = {"x": 2, "y": 1, "z": 0}  # array axis of each coordinate ([k, j, i] indexing)


class Grid:
    """Yee grid state in FP64: ex..bz and jx..jz, each [nz, ny, nx]."""

    def __init__(self, nx, ny, nz, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz = float(dx), float(dy), float(dz)
        self.x0, self.y0, self.z0 = float(x0), float(y0), float(z0)
        for nm in OFFSETS:
            setattr(self, nm, np.zeros((self.nz, self.ny, self.nx)))

    def positions(self, name):
        """Coordinates (x, y, z) of every entry of array `name`, each [nz, ny, nx]."""
        ox, oy, oz = OFFSETS[name]
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        return (self.x0 + (i + ox) * self.dx, self.y0 + (j + oy) * self.dy, self.z0 + (k + oz) * self.dz)


def _fwd(a, axis, d):
    """(a[index + 1] - a[index]) / d along `axis`, periodic."""
    return (np.roll(a, -1, axis=axis) - a) / d


def _bwd(a, axis, d):
    """(a[index] - a[index - 1]) / d along `axis`, periodic."""
    return (a - np.roll(a, 1, axis=axis)) / d


def b_half(g: Grid, dt: float) -> None:
    """B -= (dt/2) curl E, each component at its own staggered position:
    curl E at the B positions takes forward differences of E."""
    h = 0.5 * dt
    cx = _fwd(g.ez, AXIS["y"], g.dy) - _fwd(g.ey, AXIS["z"], g.dz)
    cy = _fwd(g.ex, AXIS["z"], g.dz) - _fwd(g.ez, AXIS["x"], g.dx)
    cz = _fwd(g.ey, AXIS["x"], g.dx) - _fwd(g.ex, AXIS["y"], g.dy)
    g.bx = g.bx - h * cx
    g.by = g.by - h * cy
    g.bz = g.bz - h * cz


def e_full(g: Grid, dt: float) -> None:
    """E += dt (curl B - J); curl B at the E positions takes backward
    differences of B."""
    cx = _bwd(g.bz, AXIS["y"], g.dy) - _bwd(g.by, AXIS["z"], g.dz)
    cy = _bwd(g.bx, AXIS["z"], g.dz) - _bwd(g.bz, AXIS["x"], g.dx)
    cz = _bwd(g.by, AXIS["x"], g.dx) - _bwd(g.bx, AXIS["y"], g.dy)
    g.ex = g.ex + dt * (cx - g.jx)
    g.ey = g.ey + dt * (cy - g.jy)
    g.ez = g.ez + dt * (cz - g.jz)


def field_step(g: Grid, dt: float) -> None:
    """Fields from time n to n+1 with the current at n+1/2; J is then zeroed."""
    b_half(g, dt)
    e_full(g, dt)
    b_half(g, dt)
    for nm in ("jx", "jy", "jz"):
        setattr(g, nm, np.zeros_like(getattr(g, nm)))


def nodes(g: Grid) -> np.ndarray:
    """E and B at the nodes, [nz, ny, nx, 8] FP64 (Ex Ey Ez Bx By Bz 0 0)."""
    out = np.zeros((g.nz, g.ny, g.nx, 8))
    back = lambda a, ax: np.roll(a, 1, axis=ax)  # value at index - 1
    out[..., 0] = 0.5 * (g.ex + back(g.ex, AXIS["x"]))
    out[..., 1] = 0.5 * (g.ey + back(g.ey, AXIS["y"]))
    out[..., 2] = 0.5 * (g.ez + back(g.ez, AXIS["z"]))
    for c, (a, b) in ((3, ("y", "z")), (4, ("x", "z")), (5, ("x", "y"))):
        f = (g.bx, g.by, g.bz)[c - 3]
        fa = back(f, AXIS[a])
        out[..., c] = 0.25 * (f + fa + back(f, AXIS[b]) + back(fa, AXIS[b]))
    return out


def deposit(g: Grid, x, y, z, px, py, pz, w, q: float, dt: float, weight_unit: float = 1.0) -> None:
    """Add the current of the particles (FP64 arrays) to jx, jy, jz."""
    x, y, z, px, py, pz, w = (np.asarray(a, dtype=np.float64) for a in (x, y, z, px, py, pz, w))
    gam = np.sqrt(1.0 + px * px + py * py + pz * pz)
    v = (px / gam, py / gam, pz / gam)
    pos = (x - 0.5 * dt * v[0], y - 0.5 * dt * v[1], z - 0.5 * dt * v[2])
    amount = q * w * weight_unit / (g.dx * g.dy * g.dz)
    origin = (g.x0, g.y0, g.z0)
    step = (g.dx, g.dy, g.dz)
    size = (g.nx, g.ny, g.nz)
    for c, name in enumerate(("jx", "jy", "jz")):
        off = OFFSETS[name]
        lo, frac = [], []
        for a in range(3):
            f = (pos[a] - origin[a]) / step[a] - off[a]
            fl = np.floor(f)
            lo.append(fl.astype(np.int64))
            frac.append(f - fl)
        J = getattr(g, name)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    wgt = ((frac[0] if di else 1 - frac[0]) * (frac[1] if dj else 1 - frac[1])
                           * (frac[2] if dk else 1 - frac[2]))
                    i = (lo[0] + di) % size[0]
                    j = (lo[1] + dj) % size[1]
                    k = (lo[2] + dk) % size[2]
                    np.add.at(J, (k, j, i), amount * v[c] * wgt)


def courant_ok(g: Grid, dt: float) -> bool:
    """dt below the Yee stability limit (axes with one cell do not count)."""
    s = sum(1.0 / d ** 2 for d, n in ((g.dx, g.nx), (g.dy, g.ny), (g.dz, g.nz)) if n > 1)
    return dt * np.sqrt(s) < 1.0


def loop_step(cfg, g: Grid, electrons, positrons, photons, step_index: int,
              weight_unit: float = 1.0):
    """One cycle of the loop: the oracle's QED step (``oracle.step``) gathering
    from the node grid stored in float (the layout the library's gather
    reads), the current of the leptons that existed when the cycle began,
    then the field step.  Returns the step's counters."""
    from . import grid_fields, step
    F = grid_fields(nodes(g).astype(np.float32), g.dx, g.dy, g.dz, g.x0, g.y0, g.z0)
    n0 = [s.n if s is not None else 0 for s in (electrons, positrons)]
    counters = step(cfg, F, electrons, positrons, photons, step_index)
    for s, n in zip((electrons, positrons), n0):
        if s is not None and n > 0:
            deposit(g, s.x[:n], s.y[:n], s.z[:n], s.px[:n], s.py[:n], s.pz[:n], s.w[:n], s.q,
                    cfg.dt, weight_unit)
    field_step(g, cfg.dt)
    return counters
