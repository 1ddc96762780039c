"""chi where the vector sum of Eqs. (2) and (3) cancels: leptons and photons
moving along (or close to) the propagation direction of a plane wave.  In an
FP32 context the kernels evaluate chi_e a_S = sqrt(E_par^2 + |gamma E_perp +
p x B|^2) in FP32 and redo the vector sum in FP64 when it cancels by more than
2^7; these inputs take that branch (checked here), in the step kernels as well
as through the qed_chi hook.

Stated errors (FP32 context, inputs rounded to FP32):
- chi against Eq. (2)/(3) evaluated on the same inputs in 50-digit
  arithmetic: <= 1e-6 relative for gamma up to 1e5 and photon angles down to
  3e-4 (FP32 rounding of the result, 6e-8, dominates);
- chi against the oracle: <= 1e-6 relative plus the oracle's own error
  bound (the printed formula in FP64, which loses precision to the same
  cancellation);
- the FP32 formula alone would be off by more than 1e-3 on these inputs.
FP64 context: <= 1e-9 + 4 gamma^2 eps_64 relative against the 50-digit
evaluation (exact plane waves, whose inputs carry no rounding, to ~1e-16; a
rotated one keeps an O(eps_64 |E|) remainder of E_perp + n x B, which |p|
multiplies against a chi of O(|E| / gamma)).
The emission and pair steps on co-moving ensembles then match the oracle
element-wise with the usual tolerances."""
import numpy as np
import pytest
import torch

from _parity import ambiguous, by_id, oracle_host, oracle_species, to32
from test_oracle_chi_precision import A_S, chi_exact, lepton_case, literal_bound

pytestmark = pytest.mark.gpu

FIELD_NAMES = ("ex", "ey", "ez", "bx", "by", "bz")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


def _rotations(rng, k):
    return [np.eye(3)] + [np.linalg.qr(rng.normal(size=(3, 3)))[0] for _ in range(k)]


def _species(api, q, p, E, B, dtype):
    n = len(p)
    sp = api.Species.empty(n, q, dtype=dtype, fields=True)
    z = np.zeros(n)
    arr = dict(x=z, y=z, z=z, px=p[:, 0], py=p[:, 1], pz=p[:, 2], w=np.ones(n),
               id=np.arange(n, dtype=np.uint64), ex=E[:, 0], ey=E[:, 1], ez=E[:, 2],
               bx=B[:, 0], by=B[:, 1], bz=B[:, 2])
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    return sp.load(**{k: (v.astype(np_dt) if v.dtype.kind == "f" else v) for k, v in arr.items()})


def _fp32_lepton_chi(p, E, B):
    """The FP32 sum-of-squares evaluation without the FP64 fallback (numpy
    float32), and its cancellation test."""
    f = np.float32
    p, E, B = p.astype(f), E.astype(f), B.astype(f)
    g = np.sqrt(f(1) + (p * p).sum(1))
    n = p / np.sqrt((p * p).sum(1))[:, None]
    epar = (n * E).sum(1)
    eq = E - epar[:, None] * n
    c = np.cross(p, B)
    d = g[:, None] * eq + c
    d2 = (d * d).sum(1)
    scale = g * np.abs(eq).sum(1) + np.abs(c).sum(1)
    return np.sqrt(epar * epar + d2) / f(A_S), d2 * f(16384) < scale * scale


def _lepton_inputs(rng, gammas, thetas, rots):
    P, Es, Bs, tags = [], [], [], []
    for g in gammas:
        for th in thetas:
            p, E, B, _ = lepton_case(g, th)
            for q in rots:
                P.append(q @ p), Es.append(q @ E), Bs.append(q @ B)
                tags.append((g, th))
    return np.array(P), np.array(Es), np.array(Bs), tags


def test_chi_lepton_comoving_fp32(api, orc):
    rng = np.random.default_rng(11)
    p, E, B, tags = _lepton_inputs(rng, [1e3, 1e4, 1e5], [0.0, 1e-5, 1e-4, 1e-3], _rotations(rng, 6))
    p, E, B = (a.astype(np.float32).astype(np.float64) for a in (p, E, B))
    ctx = api.qed_init_tables(api.config())
    chi = api.qed_chi(ctx, _species(api, -1, p, E, B, torch.float32)).cpu().numpy()
    exact = np.array([chi_exact(p[i], E[i], B[i], A_S, False) for i in range(len(p))])
    f32, cancels = _fp32_lepton_chi(p, E, B)
    assert cancels.all()  # every input takes the FP64 branch
    # the FP32 formula alone fails on the exact plane waves (unrotated inputs)
    plain = np.array([i for i, (g, th) in enumerate(tags) if i % 7 == 0 and th == 0.0])
    assert (np.abs(f32[plain] - exact[plain]) / exact[plain]).min() > 1e-3
    rel = np.abs(chi - exact) / exact
    assert rel.max() <= 1e-6, (rel.max(), tags[int(rel.argmax())])
    # against the oracle: within 1e-6 plus the oracle's own stated bound
    bounds = np.array([literal_bound(p[i], E[i], B[i], False) for i in range(len(p))])
    ochi = np.array([orc.chi_lepton(p[i], E[i], B[i], A_S) for i in range(len(p))])
    assert (np.abs(chi - ochi) <= (1e-6 + bounds) * exact).all()
    assert (bounds <= 1e-7).sum() >= 5  # cases where the oracle alone decides at 1e-6


def test_chi_photon_comoving_fp32(api, orc):
    rng = np.random.default_rng(12)
    P, Es, Bs, ths = [], [], [], []
    for k in (1e3, 1e5):
        for th in (3e-4, 1e-3, 1e-2, 0.1):
            E0 = 1.0 * A_S / (k * 2.0 * np.sin(th / 2) ** 2)  # chi_ph ~ 1
            p = np.array([k * np.cos(th), k * np.sin(th), 0.0])
            E, B = np.array([0.0, E0, 0.0]), np.array([0.0, 0.0, E0])
            for q in _rotations(rng, 6):
                P.append(q @ p), Es.append(q @ E), Bs.append(q @ B), ths.append(th)
    p, E, B = (np.array(a).astype(np.float32).astype(np.float64) for a in (P, Es, Bs))
    ctx = api.qed_init_tables(api.config())
    chi = api.qed_chi(ctx, _species(api, 0, p, E, B, torch.float32)).cpu().numpy()
    exact = np.array([chi_exact(p[i], E[i], B[i], A_S, True) for i in range(len(p))])
    rel = np.abs(chi - exact) / exact
    assert rel.max() <= 1e-6, (rel.max(), ths[int(rel.argmax())])
    bounds = np.array([literal_bound(p[i], E[i], B[i], True) for i in range(len(p))])
    ochi = np.array([orc.chi_photon(p[i], E[i], B[i], A_S) for i in range(len(p))])
    assert (np.abs(chi - ochi) <= (1e-6 + bounds) * exact).all()
    assert (bounds <= 1e-7).sum() >= 5


def test_chi_lepton_comoving_fp64(api):
    rng = np.random.default_rng(13)
    p, E, B, tags = _lepton_inputs(rng, [1e3, 1e4, 1e5], [0.0, 1e-5, 1e-3], _rotations(rng, 4))
    ctx = api.qed_init_tables(api.config(precision=1))
    chi = api.qed_chi(ctx, _species(api, -1, p, E, B, torch.float64)).cpu().numpy()
    exact = np.array([chi_exact(p[i], E[i], B[i], A_S, False) for i in range(len(p))])
    rel = np.abs(chi - exact) / exact
    bound = np.array([1e-9 + 4 * g * g * 2.0 ** -52 for g, _ in tags])
    assert (rel <= bound).all(), (rel.max(), tags[int(np.argmax(rel / bound))])
    # exact plane waves along x (identity first in each group of rotations,
    # theta = 0): inputs without rounding, chi to the last bits
    exact_wave = np.array([i % 5 == 0 and th == 0.0 for i, (g, th) in enumerate(tags)])
    assert rel[exact_wave].max() <= 1e-12


def _comoving_leptons(rng, n):
    """Leptons at angle theta (0 for a third, else log-uniform in [1e-5,
    1e-2]) to a plane wave of random direction and polarisation, gamma
    log-uniform in [1e2, 1e4], the amplitude set for chi log-uniform in [0.05, 5]."""
    g = np.exp(rng.uniform(np.log(1e2), np.log(1e4), n))
    th = np.where(rng.uniform(size=n) < 1 / 3, 0.0, np.exp(rng.uniform(np.log(1e-5), np.log(1e-2), n)))
    chi = np.exp(rng.uniform(np.log(0.05), np.log(5.0), n))
    P, Es, Bs = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    for i in range(n):
        p, E, B, _ = lepton_case(g[i], th[i], chi[i])
        q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        P[i], Es[i], Bs[i] = q @ p, q @ E, q @ B
    z = np.zeros(n)
    st = dict(x=z, y=z, z=z, px=P[:, 0], py=P[:, 1], pz=P[:, 2], w=np.ones(n),
              id=np.arange(n, dtype=np.uint64), ex=Es[:, 0], ey=Es[:, 1], ez=Es[:, 2],
              bx=Bs[:, 0], by=Bs[:, 1], bz=Bs[:, 2])
    return to32(st)


def _ff(st):
    return lambda i: (np.array([st["ex"][i], st["ey"][i], st["ez"][i]]),
                      np.array([st["bx"][i], st["by"][i], st["bz"][i]]))


def _gamma(h, photon=False):
    p2 = sum(np.asarray(h[c], dtype=np.float64) ** 2 for c in ("px", "py", "pz"))
    return np.sqrt(p2) if photon else np.sqrt(1 + p2)


def test_emission_of_comoving_leptons_matches_oracle(api, orc):
    """qed_emit (no push: the FP32 push itself loses the co-moving force to
    rounding) on 4000 co-moving leptons against the oracle's emission pass."""
    rng = np.random.default_rng(21)
    n, step, dt, seed = 4000, 3, 0.01, 77
    st = _comoving_leptons(rng, n)
    ctx = api.qed_init_tables(api.config(dt=dt, seed=seed))
    e = api.Species.empty(n, -1, fields=True).load(**st)
    g = api.Species.empty(40 * n, 0, fields=True)
    F = api.Fields.per_particle()
    api.qed_emit(ctx, e, g, F, step)
    torch.cuda.synchronize()
    cnt = api.qed_read_counters(ctx)
    cfg = orc.make_config(dt=dt, seed=seed)
    oe = oracle_species(orc, n, -1.0, st, fields=True)
    og = orc.Species(40 * n, 0.0, per_particle_fields=True, with_alive=True)
    lc = orc.emit(cfg, orc.per_particle_fields(), oe, og, step)
    amb = ambiguous(orc, cfg, st, _ff(st), -1.0, step, push=False)
    assert amb.sum() <= 4
    assert lc.events > 100  # the ensemble emits, some particles more than once
    ge, o = e.host(), oracle_host(oe)
    ok = ~amb
    np.testing.assert_allclose(_gamma({k: ge[k][ok] for k in ("px", "py", "pz")}),
                               _gamma({k: o[k][ok] for k in ("px", "py", "pz")}), rtol=2e-5)
    gi, gh = by_id(g.host())
    oi, oh = by_id(oracle_host(og))
    common, ig, io = np.intersect1d(gi, oi, return_indices=True)
    assert len(gi) + len(oi) - 2 * len(common) <= 40 * int(amb.sum())
    np.testing.assert_allclose(_gamma({k: gh[k][ig] for k in ("px", "py", "pz")}, True),
                               _gamma({k: oh[k][io] for k in ("px", "py", "pz")}, True), rtol=2e-5)
    assert abs(cnt["emit_events"] - lc.events) <= 40 * int(amb.sum())
    assert cnt["dropped"] == 0 and (cnt["status"] & ~2) == 0


def test_pairs_of_comoving_photons_match_oracle(api, orc):
    """The fused step's photon stage (ballistic push, chi_ph, Breit-Wheeler)
    on 4000 photons at angles 1e-3 .. 3e-2 to a plane wave, chi_ph in [2, 20]."""
    rng = np.random.default_rng(22)
    n, step, dt, seed = 4000, 2, 0.05, 91
    k = np.exp(rng.uniform(np.log(1e3), np.log(1e4), n))
    th = np.exp(rng.uniform(np.log(1e-3), np.log(3e-2), n))
    chi = np.exp(rng.uniform(np.log(2.0), np.log(20.0), n))
    P, Es, Bs = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    for i in range(n):
        E0 = chi[i] * A_S / (k[i] * 2.0 * np.sin(th[i] / 2) ** 2)
        q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        P[i] = q @ np.array([k[i] * np.cos(th[i]), k[i] * np.sin(th[i]), 0.0])
        Es[i], Bs[i] = q @ np.array([0.0, E0, 0.0]), q @ np.array([0.0, 0.0, E0])
    z = np.zeros(n)
    st = to32(dict(x=z, y=z, z=z, px=P[:, 0], py=P[:, 1], pz=P[:, 2], w=np.ones(n),
                   id=np.arange(n, dtype=np.uint64), ex=Es[:, 0], ey=Es[:, 1], ez=Es[:, 2],
                   bx=Bs[:, 0], by=Bs[:, 1], bz=Bs[:, 2]))
    ctx = api.qed_init_tables(api.config(dt=dt, seed=seed))
    e = api.Species.empty(2 * n, -1, fields=True)
    p = api.Species.empty(2 * n, +1, fields=True)
    g = api.Species.empty(n, 0, fields=True).load(**st)
    api.qed_step_fused(ctx, e, p, g, api.Fields.per_particle(), step)
    torch.cuda.synchronize()
    cnt = api.qed_read_counters(ctx)
    cfg = orc.make_config(dt=dt, seed=seed)
    oe = orc.Species(2 * n, -1.0, per_particle_fields=True)
    op = orc.Species(2 * n, 1.0, per_particle_fields=True)
    og = oracle_species(orc, n, 0.0, st, fields=True, alive=True)
    _, pc = orc.step(cfg, orc.per_particle_fields(), oe, op, og, step)
    amb = ambiguous(orc, cfg, st, _ff(st), 0.0, step, photon=True)
    assert amb.sum() <= 4
    assert pc.events > 100
    gg, o = g.host(), oracle_host(og)
    np.testing.assert_array_equal(gg["alive"][~amb], o["alive"][~amb])
    for name, gs, os_ in (("electrons", e, oe), ("positrons", p, op)):
        gi, gh = by_id(gs.host())
        oi, oh = by_id(oracle_host(os_))
        common, ig, io = np.intersect1d(gi, oi, return_indices=True)
        assert len(gi) + len(oi) - 2 * len(common) <= int(amb.sum()), name
        np.testing.assert_allclose(_gamma({c: gh[c][ig] for c in ("px", "py", "pz")}),
                                   _gamma({c: oh[c][io] for c in ("px", "py", "pz")}), rtol=2e-5,
                                   err_msg=name)
    assert abs(cnt["pair_events"] - pc.events) <= int(amb.sum())
    assert cnt["dropped"] == 0 and (cnt["status"] & ~2) == 0
