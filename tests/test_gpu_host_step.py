"""qed_lepton_step_host: the lepton stage for leptons in page-locked host
memory, streamed through the GPU in chunks (three staging buffers, copies
overlapping the steps).  Particle ids key the random draws, so the result
must be that of one qed_step_fused call on the same ensemble held on the
device (no photons at the start, so its photon stage does nothing): every
lepton equal bit for bit, the same photons (as a set: chunks append in chunk
order), the same counters; and the host mirror of the photon species equal to
the device species it mirrors.  Ragged chunks, a chunk larger than the
ensemble, both append orders, FP64, the Method II event generator (its
per-particle state copied in and out) and a mirror in pageable memory (which
the device may not map: then the host reads each chunk's photon count) are
covered."""
import numpy as np
import pytest
import torch

from _parity import to32

pytestmark = pytest.mark.gpu

LEPTON_KEYS = ("x", "y", "z", "px", "py", "pz", "w", "id")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


def _ensemble(n, seed, f64):
    from paper_1608_06356_gb300 import workloads as W
    st, _, _ = W.chi_target(n, seed=seed, chi_lo=1e-2, chi_hi=30.0)
    return st if f64 else to32(st)


def _by_id(h):
    o = np.argsort(h["id"], kind="stable")
    return {k: v[o] for k, v in h.items()}


@pytest.mark.parametrize("order,precision,generator,chunk,mirror_pinned", [
    (1, 0, 0, 7_001, True), (1, 0, 0, 1 << 20, True), (0, 0, 0, 977, True), (0, 1, 0, 12_345, True),
    (0, 0, 1, 9_000, True), (1, 0, 0, 6_000, False)])
def test_host_step_equals_device_step(api, order, precision, generator, chunk, mirror_pinned):
    n = 50_001
    f64 = precision == 1
    dt = torch.float64 if f64 else torch.float32
    st = _ensemble(n, 90 + order + 2 * precision + 4 * generator, f64)
    od = generator != 0
    cfg = dict(dt=0.02, seed=5, append_order=order, precision=precision, generator=generator)
    F = api.Fields.per_particle()
    cap_g = 6 * n
    # on the device, one call
    ctx_d = api.qed_init_tables(api.config(**cfg))
    e = api.Species.empty(n, -1, dtype=dt, fields=True, od=od).load(**st)
    g = api.Species.empty(cap_g, 0, dtype=dt, fields=True)
    api.qed_step_fused(ctx_d, e, api.Species.empty(0, 1, dtype=dt, fields=True, od=od), g, F, 4)
    torch.cuda.synchronize()
    ref_e, ref_g, ref_c = e.host(), g.host(), api.qed_read_counters(ctx_d)
    # in host memory, streamed in chunks
    ctx_h = api.qed_init_tables(api.config(**cfg))
    eh = api.Species.empty(n, -1, dtype=dt, fields=True, od=od, pinned=True).load(**st)
    g2 = api.Species.empty(cap_g, 0, dtype=dt, fields=True)
    gh = (api.Species.empty(cap_g, 0, dtype=dt, fields=True, pinned=True) if mirror_pinned
          else api.Species.empty(cap_g, 0, dtype=dt, fields=True, device="cpu"))
    api.qed_lepton_step_host(ctx_h, eh, g2, gh, F, 4, chunk)
    c = api.qed_read_counters(ctx_h)
    assert eh.n.is_pinned() and int(eh.n[0]) == n
    for k in LEPTON_KEYS + (("od_p", "od_r") if od else ()):
        np.testing.assert_array_equal(getattr(eh, k)[:n].numpy(), ref_e[k].view(getattr(eh, k).numpy().dtype)
                                      if k == "id" else ref_e[k], err_msg=k)
    m = g2.count()
    assert int(gh.n[0]) == m == len(ref_g["id"]) > 500
    hg = {k: getattr(gh, k)[:m].numpy() for k in ref_g}
    hg["id"] = hg["id"].view(np.uint64)
    dg = g2.host()
    for k in dg:  # the mirror is a copy of the device species, index by index
        np.testing.assert_array_equal(hg[k], dg[k], err_msg=k)
    a, b = _by_id(ref_g), _by_id(dg)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    for k in ("emit_events", "substeps", "dropped", "hist"):
        assert c[k] == ref_c[k], k
    assert (c["status"] & ~2) == 0


def test_host_step_rejects_bad_arguments(api):
    ctx = api.qed_init_tables(api.config(max_particles=1 << 16))
    eh = api.Species.empty(100, -1, fields=True, pinned=True)
    g = api.Species.empty(100, 0, fields=True)
    F = api.Fields.per_particle()
    with pytest.raises(RuntimeError):
        api.qed_lepton_step_host(ctx, eh, g, None, F, 0, 0)  # chunk 0
    with pytest.raises(RuntimeError):
        api.qed_lepton_step_host(ctx, eh, g, None, F, 0, (1 << 16) + 1)  # beyond max_particles
    small = api.Species.empty(10, 0, fields=True, pinned=True)
    with pytest.raises(RuntimeError):
        api.qed_lepton_step_host(ctx, eh, g, small, F, 0, 64)  # mirror smaller than g
    api.qed_lepton_step_host(ctx, eh, g, None, F, 0, 64)  # empty ensemble: nothing to do
    assert g.count() == 0
