"""Parity at the benchmark's full size: the 2^26-electron chi-target ensemble
(chi log-uniform in [1e-3, 1e2], gamma log-uniform in [1e2, 1e4], per-particle
fields, FP32 state, Dt = 0.01, table sampler) in the context the benchmark
times -- its max_particles (which sizes the scratch of the deferred-particle
passes), its persistent grids and its lepton capacities; the photon buffer is
twice the benchmark's, which empties it every step.  Step 0 is the
benchmark's step.

Two fused steps and a stable compaction run on the whole ensemble.  Then:
- the oracle recomputes seeded samples one by one: a particle's step depends
  only on its own state, id and fields (partition invariance), so a
  sub-ensemble of sampled particles, with the GPU's inputs for that step,
  gives the same particles and children;
- properties that hold at any size are checked on every particle: energy
  conservation of the emissions (E = 0 here, so the push keeps gamma),
  appended counts against the event counters, no drops, and the order and
  content of the compacted photons.

Tolerances: lepton energies 1e-4 relative (several emissions compound the
1e-5 xi tolerance), positions 1e-6 relative + 1e-5 absolute, children matched
by id.  Particles whose first Method I decision lies within the rate
tolerance of its threshold are excluded and counted.  A later sub-step of a
heavy particle can also flip within that tolerance; up to one such particle
per thousand sampled is accepted, each one excusing the children of its
chain."""
import numpy as np
import pytest
import torch

from _parity import ambiguous, by_id, oracle_host, oracle_species, to32

pytestmark = pytest.mark.gpu

SAMPLE = 3000     # electrons (and photons) recomputed by the oracle
HOT_PHOTONS = 1000  # the most energetic photons, added to the photon sample for pair events
STATE = ("x", "y", "z", "px", "py", "pz", "w")
FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


def _take(sp, idx, names):
    """Host copies of the given fields at device indices idx."""
    it = torch.as_tensor(idx, dtype=torch.int64, device=sp.x.device)
    out = {}
    for k in names:
        a = getattr(sp, k).index_select(0, it).cpu().numpy()
        out[k] = a.view(np.uint64) if k == "id" else a
    return out


def _gamma(h, photon=False):
    p2 = sum(np.asarray(h[c], dtype=np.float64) ** 2 for c in ("px", "py", "pz"))
    return np.sqrt(p2) if photon else np.sqrt(1.0 + p2)


def _energy_sum(sp, photon=False, chunk=1 << 24):
    """Sum over a species of gamma (leptons) or |p| (photons), on the device in FP64."""
    n = sp.count()
    tot = 0.0
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        p2 = sum(getattr(sp, c)[c0:c1].double() ** 2 for c in ("px", "py", "pz"))
        if photon and sp.alive is not None:
            p2 = p2 * sp.alive[c0:c1].double()
        tot += float((p2.sqrt() if photon else (1.0 + p2).sqrt()).sum())
    return tot


def _ff(st):
    return lambda i: (np.array([st["ex"][i], st["ey"][i], st["ez"][i]]),
                      np.array([st["bx"][i], st["by"][i], st["bz"][i]]))


def _lepton_mismatch(g, o, ok):
    """Sampled leptons (ok: not excluded) whose energy or position disagree."""
    eg, eo = _gamma(g), _gamma(o)
    bad = ~np.isclose(eg, eo, rtol=1e-4, atol=0.0)
    for c in ("x", "y", "z"):
        bad |= ~np.isclose(g[c], o[c], rtol=1e-6, atol=1e-5)
    return bad & ok


def _children(gpu_ids, gpu_take, orc_h, what, allowed):
    """Every oracle child id must be on the GPU (up to `allowed` missing), and
    the children found must agree in energy, position and weight."""
    oi, o = by_id(orc_h)
    pos = np.searchsorted(gpu_ids[0], oi)
    pos = np.minimum(pos, len(gpu_ids[0]) - 1)
    found = gpu_ids[0][pos] == oi
    assert (~found).sum() <= allowed, (what, int((~found).sum()), allowed, len(oi))
    g = gpu_take(gpu_ids[1][pos[found]])
    assert np.array_equal(g["id"], oi[found])
    sub = {k: v[found] for k, v in o.items()}
    photon = what == "photons"
    np.testing.assert_allclose(_gamma(g, photon), _gamma(sub, photon), rtol=1e-4, err_msg=what)
    for c in ("x", "y", "z"):
        np.testing.assert_allclose(g[c], sub[c], rtol=1e-6, atol=1e-5, err_msg=what + " " + c)
    np.testing.assert_array_equal(g["w"], sub["w"])
    return int(found.sum())


def _sorted_ids(sp, lo):
    ids = sp.id[lo:sp.count()].cpu().numpy().view(np.uint64)
    order = np.argsort(ids, kind="stable")
    return ids[order], order + lo


def test_full_size_steps_and_compaction(api, orc):
    import bench
    n = bench.N_PART
    cap_e, cap_p, cap_g, maxp = bench.capacities(n)
    cap_g *= 2  # the benchmark empties the photons every step; here two steps' photons stay
    assert cap_g <= maxp  # so the context (scratch sizes, grids) is the benchmark's
    host = bench.host_workload(n, seed=0)
    ctx = api.qed_init_tables(api.config(dt=bench.DT, seed=1, max_particles=maxp,
                                         append_order=bench.APPEND_ORDER))
    cfg = orc.make_config(dt=bench.DT, seed=1)
    e = api.Species.empty(cap_e, -1, fields=True).load(**host)
    p = api.Species.empty(cap_p, +1, fields=True)
    g = api.Species.empty(cap_g, 0, fields=True)
    F = api.Fields.per_particle()
    rng = np.random.default_rng(20240607)
    iS = np.sort(rng.choice(n, SAMPLE, replace=False))
    st0 = to32({k: v[iS] for k, v in host.items()})
    del host
    all_names = STATE + ("id",) + FIELDS
    E_before = _energy_sum(e)

    # ---- step 0: electrons only (no photons yet) --------------------------
    api.qed_step_fused(ctx, e, p, g, F, 0)
    torch.cuda.synchronize()
    c0 = api.qed_read_counters(ctx)
    ng0 = g.count()
    assert c0["dropped"] == 0 and (c0["status"] & ~2) == 0, c0
    assert e.count() == n and p.count() == 0 and ng0 == c0["emit_events"]
    # energy: what the electrons lost is in the photons (E = 0: the push keeps gamma)
    E_e, E_g = _energy_sum(e), _energy_sum(g, photon=True)
    assert abs(E_before - (E_e + E_g)) <= 1e-6 * E_before, (E_before, E_e, E_g)

    oe = oracle_species(orc, 2 * SAMPLE, -1.0, st0, fields=True)
    op = orc.Species(SAMPLE, 1.0, per_particle_fields=True)
    og = orc.Species(60 * SAMPLE, 0.0, per_particle_fields=True, with_alive=True)
    lc, _ = orc.step(cfg, orc.per_particle_fields(), oe, op, og, 0)
    o_e, o_g = oracle_host(oe), oracle_host(og)
    amb = ambiguous(orc, cfg, st0, _ff(st0), -1.0, 0)
    ge = _take(e, iS, all_names)
    np.testing.assert_array_equal(ge["id"], o_e["id"][:SAMPLE])
    bad = _lepton_mismatch(ge, {k: v[:SAMPLE] for k, v in o_e.items()}, ~amb)
    assert bad.sum() <= SAMPLE // 1000, (int(bad.sum()), iS[bad])
    assert lc.events > 200  # the sample emits (and its heavy particles run several sub-steps)
    ids_g0 = _sorted_ids(g, 0)
    found = _children(ids_g0, lambda idx: _take(g, idx, all_names), o_g, "photons",
                      allowed=60 * int(amb.sum() + bad.sum()))
    assert found >= lc.events - 60 * int(amb.sum() + bad.sum())

    # ---- step 1: sampled electrons and photons from the GPU's state --------
    st1e = to32(_take(e, iS, all_names))
    hot = np.argsort(_gamma(_take(g, np.arange(ng0), ("px", "py", "pz")), photon=True))[-HOT_PHOTONS:]
    jS = np.unique(np.concatenate([rng.choice(ng0, SAMPLE, replace=False), hot]))
    st1g = to32(_take(g, jS, all_names))
    api.qed_reset_counters(ctx)
    E_before = _energy_sum(e) + _energy_sum(g, photon=True)
    api.qed_step_fused(ctx, e, p, g, F, 1)
    torch.cuda.synchronize()
    c1 = api.qed_read_counters(ctx)
    ne1, np1, ng1 = e.count(), p.count(), g.count()
    assert c1["dropped"] == 0 and (c1["status"] & ~2) == 0, c1
    assert ne1 - n == c1["pair_events"] and np1 == c1["pair_events"] and c1["pair_events"] > 0
    assert ng1 - ng0 == c1["emit_events"]
    E_after = _energy_sum(e) + _energy_sum(p) + _energy_sum(g, photon=True)
    assert abs(E_before - E_after) <= 1e-6 * E_before, (E_before, E_after)

    m = len(jS)
    oe = oracle_species(orc, 2 * SAMPLE + 2 * m, -1.0, st1e, fields=True)
    op = orc.Species(2 * m, 1.0, per_particle_fields=True)
    og = oracle_species(orc, m + 60 * SAMPLE, 0.0, st1g, fields=True, alive=True)
    lc, pc = orc.step(cfg, orc.per_particle_fields(), oe, op, og, 1)
    o_e, o_p, o_g = oracle_host(oe), oracle_host(op), oracle_host(og)
    amb_e = ambiguous(orc, cfg, st1e, _ff(st1e), -1.0, 1)
    amb_g = ambiguous(orc, cfg, st1g, _ff(st1g), 0.0, 1, photon=True)
    ge = _take(e, iS, all_names)
    bad = _lepton_mismatch(ge, {k: v[:SAMPLE] for k, v in o_e.items()}, ~amb_e)
    assert bad.sum() <= SAMPLE // 1000, (int(bad.sum()), iS[bad])
    # sampled photons keep their slots within the step: alive flags and pushed positions
    gg = _take(g, jS, all_names + ("alive",))
    ok = ~amb_g
    np.testing.assert_array_equal(gg["alive"][ok], o_g["alive"][:m][ok])
    for c in ("x", "y", "z"):
        np.testing.assert_allclose(gg[c][ok], o_g[c][:m][ok], rtol=1e-6, atol=1e-5)
    assert pc.events > 0  # the hot photons convert
    # children: photons of the sampled electrons, pairs of the sampled photons
    ids_g1 = _sorted_ids(g, ng0)
    _children(ids_g1, lambda idx: _take(g, idx, all_names), {k: v[m:] for k, v in o_g.items()},
              "photons", allowed=60 * int(amb_e.sum() + bad.sum()))
    _children(_sorted_ids(e, n), lambda idx: _take(e, idx, all_names),
              {k: v[SAMPLE:] for k, v in o_e.items()}, "pair electrons", allowed=int(amb_g.sum()))
    _children(_sorted_ids(p, 0), lambda idx: _take(p, idx, all_names), o_p, "pair positrons",
              allowed=int(amb_g.sum()))

    # ---- stable compaction of the converted photons, at full size ---------
    alive = g.alive[:ng1].cpu().numpy().astype(bool)
    keep_ids = g.id[:ng1].cpu().numpy().view(np.uint64)[alive]
    probe = np.sort(rng.choice(ng1, SAMPLE, replace=False))
    probe = probe[alive[probe]]
    before = _take(g, probe, all_names)
    api.qed_compact(ctx, g)
    torch.cuda.synchronize()
    assert g.count() == int(alive.sum())
    np.testing.assert_array_equal(g.id[:g.count()].cpu().numpy().view(np.uint64), keep_ids)
    assert bool(g.alive[:g.count()].all())
    # the probed photons moved with all their fields, to their rank among the survivors
    dest = np.cumsum(alive)[probe] - 1
    after = _take(g, dest, all_names)
    for k in all_names:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
    del e, p, g
    torch.cuda.empty_cache()
