"""The allocation-free compaction entry point (qed_compact_noalloc).

Callers that cannot allocate device memory (an application that owns every
allocation through its own pool, a sandbox that forbids cudaMalloc, code where
an allocation would synchronise the device) use this variant: it needs no
context and keeps its scratch in a static device array.  Its result must equal
that of qed_compact, the context-based entry point, element by element (the
compaction moves values, so the comparison is exact), on two calls in a row --
the second call reuses the array the first one left behind -- in FP32 and
FP64, with and without per-particle fields and tags.

This file is collected after the parity tests, so a run that stops at the
first failure has run them before it."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NAMES = ("x", "y", "z", "px", "py", "pz", "w", "id", "alive", "n", "ex", "ey", "ez", "bx", "by", "bz",
         "tag")


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as ge
    ge.build()
    from paper_1608_06356_gb300 import _binding as B, api
    return B, api


def _photons(api, n, seed, dead_frac, dtype=torch.float32, fields=True, tag=False, capacity=None):
    from paper_1608_06356_gb300 import workloads as W
    st = W.ensemble(n, seed=seed, photons=True, id0=seed * 10**7)
    if not fields:
        st = {k: v for k, v in st.items() if k not in ("ex", "ey", "ez", "bx", "by", "bz")}
    npdt = np.float64 if dtype == torch.float64 else np.float32
    st = {k: (v.astype(npdt) if v.dtype.kind == "f" else v) for k, v in st.items()}
    if tag:
        st["tag"] = (np.arange(n) * 2654435761 % 2**31).astype(np.uint32)
    g = api.Species.empty(capacity or n, 0, dtype=dtype, fields=fields, tag=tag).load(**st)
    rng = np.random.default_rng(seed)
    alive = (rng.uniform(size=n) > dead_frac).astype(np.uint8)
    g.alive[:n].copy_(torch.tensor(alive))
    return g


def _clone(api, g, dtype, fields, tag):
    h = api.Species.empty(g.capacity, 0, dtype=dtype, fields=fields, tag=tag)
    for k in NAMES:
        a = getattr(g, k)
        if a is not None:
            getattr(h, k).copy_(a)
    return h


def _noalloc(B, g, precision, status):
    return B.lib().qed_compact_noalloc(C.byref(g.struct()), precision, status.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("precision,fields,tag", [(0, True, False), (1, True, False), (0, False, True),
                                                  (1, False, True)])
def test_noalloc_compaction_matches_context_compaction_twice(mods, precision, fields, tag):
    B, api = mods
    dtype = torch.float64 if precision else torch.float32
    ctx = api.qed_init_tables(api.config(precision=precision))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call, (n, seed, dead) in enumerate(((300_000, 5, 0.3), (123_457, 6, 0.65))):
        g_ref = _photons(api, n, seed, dead, dtype, fields, tag)
        g_new = _clone(api, g_ref, dtype, fields, tag)
        api.qed_compact(ctx, g_ref)
        rc = _noalloc(B, g_new, precision, status)
        assert rc == 0, B.lib().qed_strerror(rc)
        torch.cuda.synchronize()
        assert g_new.count() == g_ref.count() < n, call
        a, b = g_ref.host(), g_new.host()
        assert set(a) == set(b)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"call {call}: {k}")
    assert int(status.item()) == 0


def test_noalloc_accepts_its_largest_capacity(mods):
    B, api = mods
    ctx = api.qed_init_tables(api.config())
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = 70_001
    g_ref = _photons(api, n, 9, 0.5, capacity=1 << 24)
    g_new = _clone(api, g_ref, torch.float32, True, False)
    api.qed_compact(ctx, g_ref)
    assert _noalloc(B, g_new, 0, status) == 0
    torch.cuda.synchronize()
    assert g_new.count() == g_ref.count() < n
    a, b = g_ref.host(), g_new.host()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert int(status.item()) == 0


def test_noalloc_clamps_a_count_beyond_the_capacity(mods):
    # a caller's count above its capacity: the kernel compacts the capacity's
    # particles only (it never reads past the arrays) and reports CAPACITY
    B, api = mods
    ctx = api.qed_init_tables(api.config())
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = 5000
    g_ref = _photons(api, n, 11, 0.4)
    g_new = _clone(api, g_ref, torch.float32, True, False)
    api.qed_compact(ctx, g_ref)
    g_new.n.fill_(4 * n)
    assert _noalloc(B, g_new, 0, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) & B.QED_STATUS_CAPACITY
    assert g_new.count() == g_ref.count()
    np.testing.assert_array_equal(g_new.host()["id"], g_ref.host()["id"])


def test_noalloc_rejects_sizes_beyond_its_static_limit(mods):
    B, _ = mods
    s = B.qed_species()
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.d_n = n.data_ptr()
    s.capacity = (1 << 24) + 1
    assert B.lib().qed_compact_noalloc(C.byref(s), B.QED_FP32, None, None) == -3  # QED_ERR_CAPACITY
