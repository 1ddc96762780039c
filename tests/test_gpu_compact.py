"""qed_compact_fill (removal of dead particles by moving live particles from
the end into the holes) against its definition and against the oracle's
compaction.

Definition checked element by element: with a live particles left, live
particles below a keep their slot and the k-th dead slot below a (in index
order) holds the k-th live particle at or above a.  The set of particles
(all fields, by id) equals the oracle's stable compaction of the same input.
Sizes span several 2048-slot chunks with ragged tails; dead fractions from
none to all."""
import numpy as np
import pytest
import torch

from _parity import oracle_species, to32

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "px", "py", "pz", "w", "ex", "ey", "ez", "bx", "by", "bz")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


def _expected(st, alive):
    """The definition, written out with numpy."""
    n = len(alive)
    a = int(alive.sum())
    order = np.arange(n)
    holes = np.flatnonzero(alive[:a] == 0)
    tails = a + np.flatnonzero(alive[a:] == 1)
    assert len(holes) == len(tails)
    src = order[:a].copy()
    src[holes] = tails
    return {k: v[src] for k, v in st.items()}, a


@pytest.mark.parametrize("n,dead", [(0, 0.0), (1, 0.0), (1, 1.0), (2047, 0.3), (2048, 0.3),
                                    (2049, 0.5), (10000, 0.0), (10000, 1.0), (300001, 0.1),
                                    (300001, 0.9)])
def test_fill_compaction_definition(api, orc, n, dead):
    from paper_1608_06356_gb300 import workloads as W
    st = to32(W.ensemble(max(n, 1), seed=61, photons=True, id0=7))
    st = {k: v[:n] for k, v in st.items()}
    st["tag"] = (np.arange(n) % 13).astype(np.uint32)
    rng = np.random.default_rng(n)
    alive = (rng.uniform(size=n) >= dead).astype(np.uint8)
    ctx = api.qed_init_tables(api.config())
    g = api.Species.empty(max(n, 1), 0, fields=True, tag=True).load(**st)
    g.alive[:n].copy_(torch.tensor(alive))
    api.qed_compact_fill(ctx, g)
    torch.cuda.synchronize()
    exp, a = _expected(st, alive)
    assert g.count() == a
    h = g.host()
    for k in FIELDS + ("id", "tag"):
        np.testing.assert_array_equal(h[k], exp[k], err_msg=k)
    assert np.all(h["alive"] == 1)
    # the oracle's stable compaction keeps the same particles
    og = oracle_species(orc, max(n, 1), 0.0, {k: v for k, v in st.items() if k != "tag"},
                        fields=True, alive=True)
    og.alive[:n] = alive
    orc.compact(og)
    oid = og.view("id")
    assert len(oid) == a
    o_order, h_order = np.argsort(oid), np.argsort(h["id"])
    np.testing.assert_array_equal(oid[o_order], h["id"][h_order])
    for k in ("x", "pz", "w", "bx"):
        np.testing.assert_array_equal(og.view(k)[o_order].astype(np.float32), h[k][h_order])


def test_fill_compaction_after_steps_matches_stable(api):
    """A few fused steps with hole filling and with stable compaction end with
    the same particles (by id, all fields)."""
    from paper_1608_06356_gb300 import workloads as W
    n = 20000
    st = to32(W.ensemble(n, seed=5, photons=True, id0=1, g_lo=1e3, g_hi=1e5, f_lo=100, f_hi=3000))
    F = api.Fields.per_particle()
    out = []
    for fill in (False, True):
        ctx = api.qed_init_tables(api.config(dt=0.05, seed=3))
        e = api.Species.empty(4 * n, -1, fields=True)
        p = api.Species.empty(4 * n, 1, fields=True)
        g = api.Species.empty(4 * n, 0, fields=True).load(**st)
        for k in range(4):
            api.qed_step_fused(ctx, e, p, g, F, k)
            (api.qed_compact_fill if fill else api.qed_compact)(ctx, g)
        torch.cuda.synchronize()
        out.append((g.host(), api.qed_read_counters(ctx)))
    (h0, c0), (h1, c1) = out
    assert c0["pair_events"] > 100
    assert len(h0["id"]) == len(h1["id"])
    i0, i1 = np.argsort(h0["id"]), np.argsort(h1["id"])
    for k in ("id",) + FIELDS:
        np.testing.assert_array_equal(h0[k][i0], h1[k][i1], err_msg=k)


@pytest.mark.parametrize("n", [0, 1, 2049, 100003])
def test_count_alive(api, n):
    from paper_1608_06356_gb300 import workloads as W
    st = to32(W.ensemble(max(n, 1), seed=9, photons=True))
    st = {k: v[:n] for k, v in st.items()}
    alive = (np.random.default_rng(n).uniform(size=n) > 0.4).astype(np.uint8)
    ctx = api.qed_init_tables(api.config())
    g = api.Species.empty(max(n, 1) + 100, 0, fields=True).load(**st)
    g.alive[:n].copy_(torch.tensor(alive))
    g.alive[n:].fill_(1)  # stale flags past the count are not counted
    out = torch.full((3,), -5, dtype=torch.int64, device="cuda")
    api.qed_count_alive(ctx, g, out[1:2])
    torch.cuda.synchronize()
    assert out.tolist() == [-5, int(alive.sum()), -5]
