"""Failure detection of the bounded waits, with no GPU fault: the decoupled
look-back (the one wait the step kernels have) is launched behind a tile that
never publishes (qed_test_wait_expiry).  The wait must give up at its
iteration limit, within seconds, set QED_STATUS_TIMEOUT in the device status
word, and return; the host reads the status, and the same context then runs a
fused step with a clean status.

Collected last, so a run that stops at the first failure has run every other
test before it."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_lookback_wait_expires_with_status_and_context_stays_usable():
    import __graft_entry__ as ge
    ge.build()
    from paper_1608_06356_gb300 import _binding as B, api
    from paper_1608_06356_gb300 import workloads as W
    ctx = api.qed_init_tables(api.config(dt=0.01, seed=3))
    api.qed_reset_counters(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.qed_test_wait_expiry(ctx)
    bits, dropped = api.qed_last_device_status(ctx)  # waits for the kernel
    elapsed = time.perf_counter() - t0
    assert bits & B.QED_STATUS_TIMEOUT, bits
    assert dropped == 0
    assert elapsed < 60.0, elapsed
    assert api.qed_read_counters(ctx)["status"] & B.QED_STATUS_TIMEOUT
    # the context is usable afterwards: a fused step runs and reports clean
    api.qed_reset_counters(ctx)
    n = 3000
    st, _, _ = W.chi_target(n, seed=12)
    e = api.Species.empty(n, -1, fields=True).load(**{k: (v.astype(np.float32) if v.dtype.kind == "f" else v)
                                                      for k, v in st.items()})
    g = api.Species.empty(40 * n, 0, fields=True)
    api.qed_step_fused(ctx, e, api.Species.empty(0, 1, fields=True), g, api.Fields.per_particle(), 0)
    bits, dropped = api.qed_last_device_status(ctx)
    assert dropped == 0 and (bits & ~B.QED_STATUS_DOMAIN) == 0, bits
    assert g.count() > 0
