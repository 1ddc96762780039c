"""The particle-in-cell loop around the step (qed_pic_fields, qed_pic_deposit,
qed_pic_step) against the FP64 oracle of oracle/pic.py, on identical seeded
inputs.

Tolerances, from the arithmetic: the field kernels run in float, so one step
of E, B (values of order 1, curl terms dt/d of order 1) is within a few float
ulps of the largest term: 2e-6 of the largest field.  The deposit adds each
particle's 24 float contributions by atomics in an order that varies, so a
cell's J is within about (contributions per cell) ulps: 1e-5 of the largest J.
Over a multi-step loop those errors feed the push and grow with the
plasma's response: 2e-4 of the amplitude over half a plasma period."""
import math

import numpy as np
import pytest
import torch

from _parity import ambiguous, by_id, oracle_host, oracle_species, to32

pytestmark = pytest.mark.gpu

YEE = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def pic():
    from oracle import pic as P
    return P


@pytest.fixture(scope="module")
def W():
    from paper_1608_06356_gb300 import workloads
    return workloads


def _pair(api, pic, nx, ny, nz, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0):
    return (api.Yee(nx, ny, nz, dx, dy, dz, x0, y0, z0), pic.Grid(nx, ny, nz, dx, dy, dz, x0, y0, z0))


def _load(y, g, arrays):
    """Same float32 values on both sides."""
    for nm, a in arrays.items():
        a32 = np.asarray(a, dtype=np.float32)
        getattr(y, nm).copy_(torch.from_numpy(a32))
        setattr(g, nm, a32.astype(np.float64))


def _close(gpu, ref, rel, what):
    scale = max(float(np.abs(ref).max()), 1e-30)
    np.testing.assert_allclose(gpu, ref, rtol=0, atol=rel * scale, err_msg=what)


@pytest.mark.parametrize("shape", [(300, 7, 5), (16, 1, 1), (5, 9, 130)])
def test_field_step_and_nodes_match_oracle(api, pic, shape):
    """One leapfrog step with a random current, then the nodes; a grid
    spanning several 128-cell runs with a ragged tail, a 1-D grid, and one
    thin along x."""
    nx, ny, nz = shape
    ctx = api.qed_init_tables(api.config(dt=0.05))
    y, g = _pair(api, pic, nx, ny, nz, 0.31, 0.27, 0.4, x0=-2.0, y0=1.0, z0=0.5)
    rng = np.random.default_rng(nx + ny + nz)
    _load(y, g, {nm: rng.normal(size=(nz, ny, nx)) for nm in YEE})
    api.qed_pic_fields(ctx, y, advance=False)
    torch.cuda.synchronize()
    _close(y.nodes.cpu().numpy(), pic.nodes(g), 5e-7, "nodes before the step")
    api.qed_pic_fields(ctx, y, advance=True)
    pic.field_step(g, 0.05)
    torch.cuda.synchronize()
    for nm in YEE:
        got = getattr(y, nm).cpu().numpy().astype(np.float64)
        if nm.startswith("j"):
            assert not got.any(), nm
        else:
            _close(got, getattr(g, nm), 2e-6, nm)
    _close(y.nodes.cpu().numpy(), pic.nodes(g), 2e-6, "nodes")


@pytest.mark.parametrize("precision", [0, 1])
def test_deposit_matches_oracle(api, pic, precision):
    """Random particles inside and outside the periodic box; the count
    limit d_count; both element types."""
    ctx = api.qed_init_tables(api.config(dt=0.1, precision=precision))
    dt_ = torch.float64 if precision else torch.float32
    y, g = _pair(api, pic, 19, 7, 5, 0.5, 0.3, 0.45, x0=0.2, y0=-0.4, z0=1.0)
    rng = np.random.default_rng(11 + precision)
    n = 20_000
    st = dict(x=rng.uniform(-4, 14, n), y=rng.uniform(-3, 3, n), z=rng.uniform(0, 5, n),
              px=rng.normal(scale=3.0, size=n), py=rng.normal(scale=3.0, size=n),
              pz=rng.normal(scale=3.0, size=n), w=rng.uniform(0.5, 2.0, n),
              id=np.arange(n, dtype=np.uint64))
    if not precision:
        st = to32(st)
    e = api.Species.empty(n, -1, dtype=dt_).load(**st)
    lim = torch.tensor([n // 2 + 17], dtype=torch.int64, device="cuda")
    api.qed_pic_deposit(ctx, e, y, 1.7, d_count=lim)
    m = n // 2 + 17
    pic.deposit(g, *(st[k][:m] for k in ("x", "y", "z", "px", "py", "pz", "w")), -1.0, 0.1, 1.7)
    torch.cuda.synchronize()
    for nm in ("jx", "jy", "jz"):
        _close(getattr(y, nm).cpu().numpy().astype(np.float64), getattr(g, nm), 1e-5, nm)
    # all particles: the second half added on top
    api.qed_pic_deposit(ctx, e, y, 1.7)
    pic.deposit(g, *(st[k] for k in ("x", "y", "z", "px", "py", "pz", "w")), -1.0, 0.1, 1.7)
    torch.cuda.synchronize()
    for nm in ("jx", "jy", "jz"):
        _close(getattr(y, nm).cpu().numpy().astype(np.float64), getattr(g, nm), 1e-5, nm + " (all)")
    assert (api.qed_read_counters(ctx)["status"] & 4) == 0


def test_cold_plasma_oscillation(api, pic, orc, W):
    """The whole loop on a uniform cold plasma: E_x follows the closed form
    C sin(w n dt) (the oracle's pin) and the oracle loop, step by step."""
    p0, dens, dt, dx = 1e-3, 0.04, 0.1, 0.5
    nx, ny, nz = 16, 8, 8
    st = W.plasma(nx, ny, nz, dx, density=dens, drift=(p0, 0, 0), lattice=True)
    n = len(st["x"])
    ctx = api.qed_init_tables(api.config(dt=dt, seed=3, max_particles=1 << 16))
    y, g = _pair(api, pic, nx, ny, nz, dx, dx, dx)
    e = api.Species.empty(n, -1).load(**to32(st))
    ph = api.Species.empty(1024, 0)
    api.qed_pic_fields(ctx, y, advance=False)
    cfg = orc.make_config(dt=dt, seed=3)
    oe = oracle_species(orc, n, -1.0, to32(st))
    oph = orc.Species(1024, 0.0, with_alive=True)
    g0 = math.sqrt(1 + p0 * p0)
    w = 2 / dt * math.asin(dt / 2 * math.sqrt(dens / g0))
    C = dt * dens * p0 / (g0 * math.sin(w * dt))
    for s in range(160):
        api.qed_pic_step(ctx, e, None, ph, y, 1.0, s)
        pic.loop_step(cfg, g, oe, None, oph, s)
        if s % 20 == 19 or s == 0:
            ex = y.ex.cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(ex, C * math.sin(w * (s + 1) * dt), rtol=0, atol=2e-4 * C)
            _close(ex, g.ex, 2e-4, f"ex at step {s}")
    h = e.host()
    np.testing.assert_allclose(h["px"], oe.px[:n], rtol=0, atol=2e-4 * p0)
    assert ph.count() == 0 and (api.qed_read_counters(ctx)["status"] & ~2) == 0


def test_warm_plasma_matches_oracle(api, pic, orc, W):
    """Random positions and thermal momenta (gamma < 2: no emission), both
    lepton species, ten cycles: fields and particles against the oracle loop."""
    nx, ny, nz, dx, dt = 12, 10, 6, 0.4, 0.1
    st_e = W.plasma(nx, ny, nz, dx, ppc=4, density=0.05, p_th=0.1, seed=5)
    st_p = W.plasma(nx, ny, nz, dx, ppc=2, density=0.02, p_th=0.05, seed=6, id0=1 << 20)
    ne, np_ = len(st_e["x"]), len(st_p["x"])
    ctx = api.qed_init_tables(api.config(dt=dt, seed=9, max_particles=1 << 16))
    y, g = _pair(api, pic, nx, ny, nz, dx, dx, dx)
    e = api.Species.empty(ne, -1).load(**to32(st_e))
    p = api.Species.empty(np_, 1).load(**to32(st_p))
    ph = api.Species.empty(1024, 0)
    api.qed_pic_fields(ctx, y, advance=False)
    cfg = orc.make_config(dt=dt, seed=9)
    oe = oracle_species(orc, ne, -1.0, to32(st_e))
    op = oracle_species(orc, np_, 1.0, to32(st_p))
    oph = orc.Species(1024, 0.0, with_alive=True)
    for s in range(10):
        api.qed_pic_step(ctx, e, p, ph, y, 1.0, s)
        pic.loop_step(cfg, g, oe, op, oph, s)
    torch.cuda.synchronize()
    for nm in ("ex", "ey", "ez", "bx", "by", "bz"):
        _close(getattr(y, nm).cpu().numpy().astype(np.float64), getattr(g, nm), 1e-4, nm)
    for sp, o, what in ((e, oe, "electrons"), (p, op, "positrons")):
        h = sp.host()
        for k in ("px", "py", "pz"):
            _close(h[k], getattr(o, k)[:o.n], 1e-5, what + " " + k)
        for k in ("x", "y", "z"):
            np.testing.assert_allclose(h[k], getattr(o, k)[:o.n], rtol=0, atol=2e-5, err_msg=what + k)
    assert ph.count() == 0 and oph.n == 0


def test_loop_step_with_emission_matches_oracle(api, pic, orc, W):
    """Energetic electrons in a strong uniform B held on the Yee grid: one
    cycle emits photons (gathered from the nodes) and deposits the recoiled
    leptons' current, against the oracle's cycle.  The seeded input has no
    Method I decision within tolerance of its threshold (checked first)."""
    nx, ny, nz, dx, dt, B0 = 10, 8, 6, 0.5, 0.02, 1.0e3
    n = 2000
    st = W.ensemble(n, seed=77)
    st = {k: v for k, v in st.items() if k not in ("ex", "ey", "ez", "bx", "by", "bz")}
    rng = np.random.default_rng(78)
    st["x"], st["y"], st["z"] = (rng.uniform(0, m * dx, n) for m in (nx, ny, nz))
    st["w"] = np.full(n, 0.01)
    st = to32(st)
    cfg = orc.make_config(dt=dt, seed=21)
    amb = ambiguous(orc, cfg, st, lambda i: (np.zeros(3), np.array([0.0, 0.0, B0])), -1.0, 0)
    assert not amb.any()
    ctx = api.qed_init_tables(api.config(dt=dt, seed=21))
    y, g = _pair(api, pic, nx, ny, nz, dx, dx, dx)
    y.bz.fill_(B0)
    g.bz[...] = B0
    e = api.Species.empty(n, -1).load(**st)
    ph = api.Species.empty(8 * n, 0)
    api.qed_pic_fields(ctx, y, advance=False)
    api.qed_pic_step(ctx, e, None, ph, y, 1.0, 0)
    oe = oracle_species(orc, n, -1.0, st)
    oph = orc.Species(8 * n, 0.0, with_alive=True)
    lc, _ = pic.loop_step(cfg, g, oe, None, oph, 0)
    torch.cuda.synchronize()
    assert lc.events > 100
    eh, oh = e.host(), oracle_host(oe)
    # a later sub-step's decision may still sit within the rate tolerance of
    # its threshold: allow a couple of leptons (and their photons) to differ
    pm = np.sqrt(oh["px"] ** 2 + oh["py"] ** 2 + oh["pz"] ** 2)
    dev = np.sqrt(sum((eh[k] - oh[k]) ** 2 for k in ("px", "py", "pz"))) / pm
    assert (dev > 2e-5).sum() <= 2, np.sort(dev)[-5:]
    for k in ("x", "y", "z"):
        np.testing.assert_allclose(eh[k], oh[k], rtol=0, atol=2e-5, err_msg=k)
    gi, gg = by_id(ph.host())
    oi, oo = by_id(oracle_host(oph))
    common, ig, io = np.intersect1d(gi, oi, return_indices=True)
    assert len(gi) + len(oi) - 2 * len(common) <= 4 and len(common) > 100
    pg = np.sqrt(sum(gg[k][ig].astype(np.float64) ** 2 for k in ("px", "py", "pz")))
    po = np.sqrt(sum(oo[k][io] ** 2 for k in ("px", "py", "pz")))
    np.testing.assert_allclose(pg, po, rtol=2e-5, err_msg="photon energies")
    for nm in ("ex", "ey", "ez", "bx", "by", "bz"):
        got = getattr(y, nm).cpu().numpy().astype(np.float64)
        ref = getattr(g, nm)
        if nm == "bz":  # B0 plus a response finer than a float step of B0
            np.testing.assert_allclose(got, ref, rtol=0, atol=2 * float(np.spacing(np.float32(B0))))
        else:
            _close(got, ref, 1e-4, nm)


def test_pic_rejects_bad_arguments(api):
    ctx = api.qed_init_tables(api.config(dt=0.5))
    y = api.Yee(8, 8, 8, 0.5, 0.5, 0.5)
    with pytest.raises(RuntimeError):  # dt = 0.5 > 0.5 / sqrt(3): beyond the Courant limit
        api.qed_pic_fields(ctx, y, advance=True)
    api.qed_pic_fields(ctx, y, advance=False)  # nodes only: no time step, accepted
    y1 = api.Yee(8, 1, 1, 0.6, 0.01, 0.01)  # one-cell axes do not count
    api.qed_pic_fields(ctx, y1, advance=True)
    g = api.Species.empty(16, 0)
    with pytest.raises(RuntimeError):  # photons carry no current
        api.qed_pic_deposit(ctx, api.Species.empty(16, 0, alive=True).load(
            x=np.zeros(1), y=np.zeros(1), z=np.zeros(1), px=np.ones(1), py=np.zeros(1), pz=np.zeros(1),
            w=np.ones(1), id=np.zeros(1, dtype=np.uint64)), y1)
    bad = api.Yee(8, 8, 8, 0.5, 0.5, 0.5)
    bad.ex = bad.ex.view(-1)[1:]  # not 16-byte aligned
    with pytest.raises(RuntimeError):
        api.qed_pic_fields(ctx, bad, advance=False)
    torch.cuda.synchronize()
    assert g.count() == 0
