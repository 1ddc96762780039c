"""Pins of the particle-in-cell loop oracle (oracle/pic.py) against facts
that do not come from it: the exact discrete plane wave of Yee's scheme along
every axis and polarisation (and its node values in closed form), a uniform
current draining E linearly, the deposit against a direct evaluation of the
CIC hat function at every staggered position (and its sum rule), and the
cold-plasma oscillation of the whole loop -- the oracle's QED step included --
against its closed-form frequency and amplitude."""
import math

import numpy as np
import pytest

from oracle import pic

# n x e for each (propagation axis, polarisation): the B component and its sign
CROSS = {("x", "y"): ("z", 1), ("x", "z"): ("y", -1), ("y", "z"): ("x", 1),
         ("y", "x"): ("z", -1), ("z", "x"): ("y", 1), ("z", "y"): ("x", -1)}


def _grid():
    return pic.Grid(16, 12, 10, 0.3, 0.25, 0.4, x0=-1.0, y0=0.5, z0=2.0)


@pytest.mark.parametrize("axis,pol", sorted(CROSS))
def test_discrete_plane_wave_is_exact(axis, pol):
    """E_pol = cos(k s - w t), B_{n x e} = cos(w dt/2) cos(k s - w t) at integer
    times, with sin(w dt/2) = (dt/d) sin(k d/2), solves the leapfrog exactly
    (s the coordinate along the axis, d the spacing)."""
    g = _grid()
    a = "xyz".index(axis)
    n_ax, d = (g.nx, g.ny, g.nz)[a], (g.dx, g.dy, g.dz)[a]
    origin = (g.x0, g.y0, g.z0)[a]
    k = 2 * math.pi * 3 / (n_ax * d)
    dt = 0.1
    assert pic.courant_ok(g, dt)
    w = 2 / dt * math.asin(dt / d * math.sin(k * d / 2))
    bc, sign = CROSS[(axis, pol)]

    def wave(name, t, factor=1.0):
        s = g.positions(name)[a] - origin
        return factor * np.cos(k * s - w * t)

    setattr(g, "e" + pol, wave("e" + pol, 0.0))
    setattr(g, "b" + bc, wave("b" + bc, 0.0, sign * math.cos(w * dt / 2)))
    steps = 25
    for _ in range(steps):
        pic.field_step(g, dt)
    t = steps * dt
    for nm in ("ex", "ey", "ez", "bx", "by", "bz"):
        if nm == "e" + pol:
            ref = wave(nm, t)
        elif nm == "b" + bc:
            ref = wave(nm, t, sign * math.cos(w * dt / 2))
        else:
            ref = np.zeros_like(getattr(g, nm))
        np.testing.assert_allclose(getattr(g, nm), ref, rtol=0, atol=1e-12, err_msg=nm)
    # nodes: E averages along its own axis (normal to the propagation), B over
    # a plane that contains the propagation axis: a factor cos(k d/2)
    N = pic.nodes(g)
    k_, j_, i_ = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    s_node = ((i_ * g.dx, j_ * g.dy, k_ * g.dz)[a])
    base = np.cos(k * s_node - w * t)
    ref = np.zeros(N.shape)
    ref[..., "xyz".index(pol)] = base
    ref[..., 3 + "xyz".index(bc)] = sign * math.cos(w * dt / 2) * math.cos(k * d / 2) * base
    np.testing.assert_allclose(N, ref, rtol=0, atol=1e-12)


def test_uniform_current_drains_e_and_is_zeroed():
    g = _grid()
    rng = np.random.default_rng(1)
    E0, B0, J = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
    for c, nm in enumerate("xyz"):
        getattr(g, "e" + nm)[...] = E0[c]
        getattr(g, "b" + nm)[...] = B0[c]
        getattr(g, "j" + nm)[...] = J[c]
    dt = 0.07
    pic.field_step(g, dt)
    for c, nm in enumerate("xyz"):
        np.testing.assert_allclose(getattr(g, "e" + nm), E0[c] - dt * J[c], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(getattr(g, "b" + nm), B0[c], rtol=1e-14, atol=1e-14)
        assert not getattr(g, "j" + nm).any()
    N = pic.nodes(g)
    np.testing.assert_allclose(N[..., :3], np.broadcast_to(E0 - dt * J, N[..., :3].shape), rtol=1e-13)
    np.testing.assert_allclose(N[..., 3:6], np.broadcast_to(B0, N[..., 3:6].shape), rtol=1e-13)
    assert not N[..., 6:].any()


def test_deposit_equals_hat_function_everywhere():
    """J at every staggered position = sum over particles of q w v / V times the
    product of hat functions max(0, 1 - |periodic distance| / d)."""
    g = pic.Grid(7, 5, 6, 0.5, 0.3, 0.45, x0=0.2, y0=-0.4, z0=1.0)
    rng = np.random.default_rng(4)
    n = 40
    x = rng.uniform(-3, 8, n)
    y = rng.uniform(-2, 2, n)
    z = rng.uniform(0, 5, n)
    p = rng.normal(scale=2.0, size=(3, n))
    w = rng.uniform(0.5, 2, n)
    q, dt, wu = -1.0, 0.2, 1.7
    pic.deposit(g, x, y, z, *p, w, q, dt, wu)
    gam = np.sqrt(1 + (p * p).sum(0))
    v = p / gam
    pos = (x - dt / 2 * v[0], y - dt / 2 * v[1], z - dt / 2 * v[2])
    L = (g.nx * g.dx, g.ny * g.dy, g.nz * g.dz)
    d = (g.dx, g.dy, g.dz)
    V = g.dx * g.dy * g.dz
    for c, nm in enumerate(("jx", "jy", "jz")):
        R = g.positions(nm)
        ref = np.zeros_like(R[0])
        for m in range(n):
            S = np.ones_like(R[0])
            for a in range(3):
                delta = (R[a] - pos[a][m]) % L[a]
                delta = np.minimum(delta, L[a] - delta)  # periodic distance
                S *= np.maximum(0.0, 1.0 - delta / d[a])
            ref += q * w[m] * wu * v[c][m] / V * S
        np.testing.assert_allclose(getattr(g, nm), ref, rtol=1e-10, atol=1e-12, err_msg=nm)
        # sum rule: the integral of J is the total q w v
        np.testing.assert_allclose(getattr(g, nm).sum() * V, (q * w * wu * v[c]).sum(), rtol=1e-12)


def test_courant_limit():
    g = pic.Grid(8, 8, 8, 0.2, 0.2, 0.2)
    lim = 0.2 / math.sqrt(3)
    assert pic.courant_ok(g, 0.99 * lim) and not pic.courant_ok(g, 1.01 * lim)
    g1 = pic.Grid(8, 1, 1, 0.2, 0.01, 0.01)  # one-cell axes do not count
    assert pic.courant_ok(g1, 0.19)


def cold_plasma(orc, p0=1e-3, density=0.04, dt=0.1, cells=(4, 3, 2), dx=0.5):
    """A uniform cold electron plasma, one electron per cell at the cell
    centres moving with p0 along x, E = B = 0: the oracle loop's E_x series."""
    nx, ny, nz = cells
    g = pic.Grid(nx, ny, nz, dx, dx, dx)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    n = nx * ny * nz
    st = dict(x=((i + 0.5) * dx).ravel(), y=((j + 0.5) * dx).ravel(), z=((k + 0.5) * dx).ravel(),
              px=np.full(n, p0), py=np.zeros(n), pz=np.zeros(n), w=np.full(n, density * dx ** 3),
              id=np.arange(n, dtype=np.uint64))
    cfg = orc.make_config(dt=dt, seed=3)
    e = orc.Species(n, -1.0).load(**st)
    ph = orc.Species(16, 0.0, with_alive=True)
    return cfg, g, e, ph


def test_cold_plasma_oscillation_closed_form(orc):
    """E_x^n = C sin(w n dt), p^{n+1/2} = p0 cos(w (n+1/2) dt) / cos(w dt/2) with
    4 sin^2(w dt/2) = n dt^2 / gamma0 and C = dt n p0 / (gamma0 sin(w dt)): the
    leapfrog of dp/dt = -E, dE/dt = -J = n v for a uniform electron plasma."""
    p0, dens, dt = 1e-3, 0.04, 0.1
    cfg, g, e, ph = cold_plasma(orc, p0, dens, dt)
    g0 = math.sqrt(1 + p0 * p0)
    w = 2 / dt * math.asin(dt / 2 * math.sqrt(dens / g0))
    C = dt * dens * p0 / (g0 * math.sin(w * dt))
    steps = 160  # about half a plasma period
    for s in range(steps):
        pic.loop_step(cfg, g, e, None, ph, s)
        n = s + 1
        np.testing.assert_allclose(g.ex, C * math.sin(w * n * dt), rtol=0, atol=2e-4 * C)
        np.testing.assert_allclose(e.px[:e.n], p0 * math.cos(w * (n - 0.5) * dt) / math.cos(w * dt / 2),
                                   rtol=0, atol=2e-4 * p0)
    for nm in ("ey", "ez", "bx", "by", "bz"):
        assert np.abs(getattr(g, nm)).max() < 1e-6 * C, nm
    assert ph.n == 0  # gamma < 2: no photon above the infrared cut
