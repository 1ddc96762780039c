"""Host-side checks of the C-ABI boundary (no GPU needed): the shared library
loads, it exports every function include/qed.h declares, the Python binding
covers each of them, the ctypes struct layouts match the C compiler's, bad
arguments and null contexts are rejected before any CUDA call, and a missing
library raises.  Also the benchmark's host-only parts: the reference arm's
JSON line and the capacities of the default run."""
import ctypes as C
import json
import os
import re
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qed.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qed_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def qlib():
    from paper_1608_06356_gb300 import build, _binding
    build()
    return _binding


def test_library_exports_every_declared_symbol(qlib):
    names = _declared_functions()
    assert "qed_init_tables" in names and "qed_step_fused" in names
    lib = C.CDLL(qlib.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(qlib.SIGNATURES), set(names) ^ set(qlib.SIGNATURES)


def test_struct_layouts_match_c(qlib, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "qed.h"
        int main(void) {
          printf("%zu %zu %zu %zu\\n", sizeof(qed_config), sizeof(qed_species),
                 sizeof(qed_fields), sizeof(qed_counters));
          printf("%zu %zu %zu %zu\\n", offsetof(qed_config, seed), offsetof(qed_species, d_n),
                 offsetof(qed_fields, grid), offsetof(qed_counters, hist));
          printf("%zu %zu %zu %zu\\n", sizeof(qed_tuning), offsetof(qed_tuning, sched),
                 offsetof(qed_tuning, ms_per_step), offsetof(qed_tuning, sched_ms));
          printf("%zu %zu %zu %zu\\n", sizeof(qed_yee), offsetof(qed_yee, dx),
                 offsetof(qed_yee, ex), offsetof(qed_yee, nodes));
          return 0;
        }"""))
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    B = qlib
    assert [int(v) for v in out[:4]] == [C.sizeof(B.qed_config), C.sizeof(B.qed_species),
                                         C.sizeof(B.qed_fields), C.sizeof(B.qed_counters)]
    assert [int(v) for v in out[4:8]] == [B.qed_config.seed.offset, B.qed_species.d_n.offset,
                                          B.qed_fields.grid.offset, B.qed_counters.hist.offset]
    assert [int(v) for v in out[8:12]] == [C.sizeof(B.qed_tuning), B.qed_tuning.sched.offset,
                                           B.qed_tuning.ms_per_step.offset, B.qed_tuning.sched_ms.offset]
    assert [int(v) for v in out[12:]] == [C.sizeof(B.qed_yee), B.qed_yee.dx.offset, B.qed_yee.ex.offset,
                                          B.qed_yee.nodes.offset]


def test_config_defaults_and_strerror(qlib):
    lib = qlib.lib()
    c = qlib.qed_config()
    lib.qed_config_default(C.byref(c))
    assert c.wdt_max == 0.2 and c.xi_min_energy == 2.0 and c.pair_sign == 1
    assert abs(c.alpha - 1 / 137.035999) < 1e-15 and c.a_S == 412148.45
    assert lib.qed_strerror(-1) == b"invalid argument"
    assert lib.qed_strerror(0) == b"ok"


def test_invalid_arguments_rejected_without_gpu(qlib):
    # argument checks run on the host before any CUDA call
    lib = qlib.lib()
    c = qlib.qed_config()
    lib.qed_config_default(C.byref(c))
    c.dt = -1.0
    h = C.c_void_p()
    assert lib.qed_init_tables(C.byref(c), C.byref(h), None) == -1
    assert lib.qed_step_fused(None, None, None, None, None, 0, None) == -1
    assert lib.qed_sample_xi(None, None, None, None, 4, 0, None) == -1
    assert lib.qed_table_get(None, 1, None, 0, None) == -1


def test_workload_generators_are_seeded():
    from paper_1608_06356_gb300 import workloads as W
    a, _, _ = W.chi_target(1000, seed=3)
    b, chi, g = W.chi_target(1000, seed=3)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    # B is perpendicular to p and sized for the target chi
    p = np.stack([a["px"], a["py"], a["pz"]])
    Bv = np.stack([a["bx"], a["by"], a["bz"]])
    assert np.max(np.abs((p * Bv).sum(0)) / (np.linalg.norm(p, axis=0) * np.linalg.norm(Bv, axis=0))) < 1e-12
    np.testing.assert_allclose(np.linalg.norm(p, axis=0) * np.linalg.norm(Bv, axis=0) / W.A_S_1UM, chi,
                               rtol=1e-12)
    e = W.ensemble(500, seed=1)
    gam = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    assert gam.min() >= 100 * (1 - 1e-12) and gam.max() <= 1e4 * (1 + 1e-12)


def test_plasma_generator():
    from paper_1608_06356_gb300 import workloads as W
    a = W.plasma(6, 5, 4, 0.5, ppc=3, density=0.02, p_th=0.1, seed=2)
    b = W.plasma(6, 5, 4, 0.5, ppc=3, density=0.02, p_th=0.1, seed=2)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    n = 6 * 5 * 4 * 3
    assert len(a["x"]) == n and np.all(a["w"] == 0.02 * 0.5 ** 3 / 3)
    for c, L in (("x", 3.0), ("y", 2.5), ("z", 2.0)):
        assert a[c].min() >= 0 and a[c].max() < L
    # stored by cell: the same particles, cell indices non-decreasing (z, then y, then x)
    s = W.plasma(6, 5, 4, 0.5, ppc=3, density=0.02, p_th=0.1, seed=2, cell_order=True)
    cell = lambda d: ((np.floor(d["z"] / 0.5) * 5 + np.floor(d["y"] / 0.5)) * 6 + np.floor(d["x"] / 0.5))
    assert np.all(np.diff(cell(s)) >= 0)
    np.testing.assert_array_equal(np.sort(s["x"]), np.sort(a["x"]))
    # a lattice: one at each cell centre
    lat = W.plasma(4, 3, 2, 1.0, lattice=True, drift=(0.1, 0, 0))
    np.testing.assert_array_equal(np.unique(lat["x"]), [0.5, 1.5, 2.5, 3.5])
    assert np.all(lat["px"] == 0.1) and np.all(lat["py"] == 0)


def test_entry_points_reject_a_null_context(qlib):
    lib = qlib.lib()
    bits, dropped = C.c_uint32(7), C.c_int64(7)
    assert lib.qed_last_device_status(None, C.byref(bits), C.byref(dropped)) == -1
    assert bits.value == 7 and dropped.value == 7  # untouched on error
    assert lib.qed_count_alive(None, None, None, None) == -1
    assert lib.qed_compact_fill(None, None, None) == -1
    assert lib.qed_compact(None, None, None) == -1
    assert lib.qed_profile_end_phases(None, None, None) == -1
    assert lib.qed_test_wait_expiry(None, None) == -1
    assert lib.qed_pic_fields(None, None, 0, None) == -1
    assert lib.qed_pic_deposit(None, None, None, 1.0, None, None) == -1
    assert lib.qed_pic_step(None, None, None, None, None, 1.0, 0, None) == -1


def test_missing_library_fails_loudly(qlib, monkeypatch, tmp_path):
    # no fallback: without the built library every call path raises
    monkeypatch.setattr(qlib, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(qlib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        qlib.lib()


def test_reference_arm_prints_one_line():
    # the reference arm is the oracle on the host cores; a tiny sample here
    out = subprocess.check_output([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                   "--steps", "1", "--warmup", "3", "--ref-particles", "64"], text=True,
                                  cwd=ROOT)
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "particle-steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_bench_capacities_hold_any_step_count():
    # every headline step starts from the same ensemble, so the buffers do not
    # depend on the step count: the photon buffer holds one step's emissions
    # (the ensemble's mean W_rad Dt, an upper bound of the mean event count,
    # is 0.184 per electron at Dt = 0.01)
    sys.path.insert(0, ROOT)
    import bench
    n = bench.N_PART
    cap_e, cap_p, cap_g, maxp = bench.capacities(n)
    assert cap_e >= n and cap_g >= 1.5 * 0.184 * n
    assert maxp == max(cap_e, cap_g)


def test_bench_refuses_a_value_on_overflow():
    sys.path.insert(0, ROOT)
    import bench
    ok = {"dropped": 0, "status": 2}  # DOMAIN alone is informational
    assert bench.run_status(ok) == "ok"
    assert bench.run_status({"dropped": 5, "status": 0}) == "overflow"
    assert bench.run_status({"dropped": 0, "status": 1}) == "overflow"
    assert bench.run_status({"dropped": 0, "status": 8}).startswith("device-status")
