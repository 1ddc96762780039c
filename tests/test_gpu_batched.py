"""Batched independent runs under a captured CUDA graph (qed_run_batched),
inherited run tags, and the launch autotuner."""
import numpy as np
import pytest
import torch

from _parity import by_id, oracle_host, oracle_species, to32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


def _runs(W, sizes, seed=0):
    """Concatenated runs: run r has sizes[r] electrons with its own chi range."""
    rng = np.random.default_rng(seed)
    parts = []
    off = 0
    for r, n in enumerate(sizes):
        lo, hi = np.sort(np.exp(rng.uniform(np.log(0.01), np.log(10.0), 2)))
        st, _, _ = W.chi_target(int(n), seed=1000 + r, chi_lo=lo, chi_hi=hi, id0=off)
        st["tag"] = np.full(int(n), r, dtype=np.uint32)
        parts.append(st)
        off += int(n)
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def _species(api, st, n, cap_factor=3):
    e = api.Species.empty(cap_factor * n, -1, fields=True, tag=True).load(**to32(st))
    p = api.Species.empty(cap_factor * n, 1, fields=True, tag=True)
    g = api.Species.empty(cap_factor * n, 0, fields=True, tag=True)
    return e, p, g


def test_graph_replay_equals_eager_steps(api):
    from paper_1608_06356_gb300 import workloads as W
    sizes = [3000, 17, 900, 40000, 1, 5555, 256, 12000]
    st = _runs(W, sizes)
    n = len(st["x"])
    F = api.Fields.per_particle()
    ctx_a = api.qed_init_tables(api.config(dt=0.02, seed=9))
    ctx_b = api.qed_init_tables(api.config(dt=0.02, seed=9))
    ea, pa, ga = _species(api, st, n)
    eb, pb, gb = _species(api, st, n)
    for k in range(6):  # eager: fused step + photon compaction by hole filling
        api.qed_step_fused(ctx_a, ea, pa, ga, F, 10 + k)
        api.qed_compact_fill(ctx_a, ga)
    counts = api.qed_run_batched(ctx_b, eb, pb, gb, F, 10, 3, n_runs=len(sizes))
    api.qed_run_batched(ctx_b, eb, pb, gb, F, 13, 3)  # replays the cached graph
    torch.cuda.synchronize()
    for sa, sb in ((ea, eb), (pa, pb), (ga, gb)):
        assert sa.count() == sb.count()
        ha, hb = sa.host(), sb.host()
        for k in ha:
            np.testing.assert_array_equal(ha[k], hb[k], err_msg=k)
    assert ga.count() > 1000
    # per-run alive photon counts after the first three steps were returned; check
    # the final ones against the tags
    final = api.qed_run_batched(ctx_b, eb, pb, gb, F, 16, 3, n_runs=len(sizes))
    torch.cuda.synchronize()
    h = gb.host()
    ref = np.bincount(h["tag"][h["alive"] == 1], minlength=len(sizes))
    np.testing.assert_array_equal(final.cpu().numpy(), ref)
    assert counts is not None


def test_children_inherit_tags_like_the_oracle(api, orc):
    from paper_1608_06356_gb300 import workloads as W
    n = 2000
    st, _, _ = W.chi_target(n, seed=77, chi_lo=0.5, chi_hi=20)
    st = to32(st)
    st["tag"] = (np.arange(n) % 7).astype(np.uint32)
    ctx = api.qed_init_tables(api.config(dt=0.05, seed=4))
    e = api.Species.empty(n, -1, fields=True, tag=True).load(**st)
    g = api.Species.empty(20 * n, 0, fields=True, tag=True)
    api.qed_step_fused(ctx, e, api.Species.empty(0, 1, fields=True, tag=True), g, api.Fields.per_particle(), 1)
    torch.cuda.synchronize()
    cfg = orc.make_config(dt=0.05, seed=4)
    oe = orc.Species(n, -1.0, per_particle_fields=True, with_tag=True).load(**st)
    og = orc.Species(20 * n, 0.0, per_particle_fields=True, with_alive=True, with_tag=True)
    orc.step(cfg, orc.per_particle_fields(), oe, orc.Species(1, 1.0), og, 1)
    gi, gh = by_id(g.host())
    oh = {"id": og.view("id"), "tag": og.view("tag")}
    oi, oh = by_id(oh)
    common, ig, io = np.intersect1d(gi, oi, return_indices=True)
    assert len(common) > 0.99 * max(len(gi), len(oi)) and len(common) > 100
    np.testing.assert_array_equal(gh["tag"][ig], oh["tag"][io])


def test_autotuner_picks_a_factor(api):
    from paper_1608_06356_gb300 import workloads as W
    st = _runs(W, [50000, 20000])
    n = len(st["x"])
    ctx = api.qed_init_tables(api.config(dt=0.01, seed=2))
    e, p, g = _species(api, st, n, cap_factor=8)
    best, ms = api.qed_autotune(ctx, e, p, g, api.Fields.per_particle(), reps=2)
    assert 1 <= best <= 8
    assert all(m > 0 for m in ms)
    assert ms[best - 1] == min(ms)


@pytest.mark.parametrize("order", [0, 1])
def test_group_autotuner_picks_a_factor_per_kernel_group(api, order):
    """qed_autotune_groups: one factor per kernel group, each the fastest of
    the factors it timed; the chosen configuration is the one the context
    keeps, and the steps it runs afterwards give the same particles as an
    untuned context (launch sizes change no result)."""
    from paper_1608_06356_gb300 import workloads as W
    st = _runs(W, [50000, 20000])
    n = len(st["x"])
    ctx = api.qed_init_tables(api.config(dt=0.01, seed=2, append_order=order))
    e, p, g = _species(api, st, n, cap_factor=8)
    t = api.qed_autotune_groups(ctx, e, p, g, api.Fields.per_particle(), reps=2)
    for name, f in t["grid_factor"].items():
        ms = t["ms"][name]
        assert 1 <= f <= 8 and all(m > 0 for m in ms), name
        assert ms[f - 1] == min(ms), name
    for name, v in t["sched"].items():
        tried = t["sched_ms"][name]
        assert len(tried) >= 3 and all(m > 0 for m in tried.values()), name
        assert tried[v] == min(tried.values()), name
    assert t["ms_per_step"] == min([min(t["ms"]["compact"])] +
                                   [min(v.values()) for v in t["sched_ms"].values()])
    out = []
    for c in (ctx, api.qed_init_tables(api.config(dt=0.01, seed=2, append_order=order))):
        e2, p2, g2 = _species(api, st, n, cap_factor=8)
        api.qed_step_fused(c, e2, p2, g2, api.Fields.per_particle(), 5)
        torch.cuda.synchronize()
        out.append((e2.host(), g2.host()))
    np.testing.assert_array_equal(out[0][0]["px"], out[1][0]["px"])
    np.testing.assert_array_equal(np.sort(out[0][1]["id"]), np.sort(out[1][1]["id"]))


@pytest.mark.parametrize("order", [0, 1])
def test_chain_scheduling_changes_no_result(api, order):
    """The Method I chain-scheduling parameters (lanes per round, draws per
    round, queue trigger) at their extremes give the same particles, photons
    and counters as the defaults."""
    from paper_1608_06356_gb300 import workloads as W
    st = _runs(W, [40000, 30000])
    n = len(st["x"])
    out = []
    for sched in ({}, {"emit_lanes": 1, "round_lanes": 1, "scan_draws": 2, "scan_left": 1,
                       "queue_trigger": 1},
                  {"emit_lanes": 32, "round_lanes": 32, "scan_draws": 16, "scan_left": 32,
                   "queue_trigger": 33}):
        ctx = api.qed_init_tables(api.config(dt=0.02, seed=4, append_order=order))
        api.qed_set_tuning(ctx, {}, sched)
        e, p, g = _species(api, st, n, cap_factor=8)
        for s in range(2):
            api.qed_step_fused(ctx, e, p, g, api.Fields.per_particle(), 7 + s)
        torch.cuda.synchronize()
        c = api.qed_read_counters(ctx)
        assert c["status"] & ~2 == 0
        out.append((e.host(), p.host(), g.host(), c))
    for o in out[1:]:
        for a, b in zip(out[0][:3], o[:3]):
            ia, ib = np.argsort(a["id"], kind="stable"), np.argsort(b["id"], kind="stable")
            for k in a:
                np.testing.assert_array_equal(a[k][ia], b[k][ib], err_msg=k)
        for k in ("emit_events", "pair_events", "substeps", "dropped", "hist"):
            assert out[0][3][k] == o[3][k], k
    assert out[0][3]["emit_events"] > 1000


def test_set_tuning_rejects_out_of_range_values(api):
    ctx = api.qed_init_tables(api.config())
    for bad in ({"emit_lanes": 33}, {"scan_draws": 3}, {"scan_draws": 18}, {"queue_trigger": 34},
                {"round_lanes": -1}):
        with pytest.raises(RuntimeError):
            api.qed_set_tuning(ctx, {}, bad)
    api.qed_set_tuning(ctx, {"stream": 2}, {"scan_draws": 8})
