"""The allocation-free compaction entry point (qed_compact_noalloc).

Callers that cannot allocate device memory (an application that owns every
allocation through its own pool, a sandbox that forbids cudaMalloc, code where
an allocation would synchronise the device) use this variant: it needs no
context and keeps its scratch in a static device array.  Its result must equal
that of qed_compact, the context-based entry point, element by element (the
compaction moves values, so the comparison is exact), on two calls in a row --
the second call reuses the array the first one left behind.

This file is collected after the parity tests, so a run that stops at the
first failure has run them before it."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _photons(api, n, seed, dead_frac):
    from paper_1608_06356_gb300 import workloads as W
    st = W.ensemble(n, seed=seed, photons=True, id0=seed * 10**7)
    g = api.Species.empty(n, 0, fields=True).load(**st)
    rng = np.random.default_rng(seed)
    alive = (rng.uniform(size=n) > dead_frac).astype(np.uint8)
    g.alive[:n].copy_(torch.tensor(alive))
    return g


def _clone(api, g):
    h = api.Species.empty(g.capacity, 0, fields=True)
    for k in ("x", "y", "z", "px", "py", "pz", "w", "id", "alive", "n",
              "ex", "ey", "ez", "bx", "by", "bz"):
        getattr(h, k).copy_(getattr(g, k))
    return h


def test_noalloc_compaction_matches_context_compaction_twice():
    import __graft_entry__ as ge
    ge.build()
    from paper_1608_06356_gb300 import _binding as B, api
    ctx = api.qed_init_tables(api.config())
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call, (n, seed, dead) in enumerate(((300_000, 5, 0.3), (123_457, 6, 0.65))):
        g_ref = _photons(api, n, seed, dead)
        g_new = _clone(api, g_ref)
        api.qed_compact(ctx, g_ref)
        rc = B.lib().qed_compact_noalloc(C.byref(g_new.struct()), B.QED_FP32, status.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
        assert rc == 0, B.lib().qed_strerror(rc)
        torch.cuda.synchronize()
        assert g_new.count() == g_ref.count() < n, call
        a, b = g_ref.host(), g_new.host()
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"call {call}: {k}")
    assert int(status.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_static_limit():
    import __graft_entry__ as ge
    ge.build()
    from paper_1608_06356_gb300 import _binding as B
    s = B.qed_species()
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.d_n = n.data_ptr()
    s.capacity = (1 << 24) + 1
    assert B.lib().qed_compact_noalloc(C.byref(s), B.QED_FP32, None, None) == -3  # QED_ERR_CAPACITY
