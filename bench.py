"""Benchmark of the per-macroparticle QED Monte Carlo step on GB300.

Headline workload (one step = one qed_step_fused pass): 2^26 = 64M electrons
with chi log-uniform in [1e-3, 1e2] and gamma log-uniform in [1e2, 1e4],
per-particle fields (B perpendicular to p, |B| = chi a_S/|p|, E = 0),
Dt = 0.01 / omega0, FP32 state.  Every step starts from the same momenta:
they are restored from a device copy and the photon buffer is emptied before
the step (inside the timed region); the positions keep advancing, which with
per-particle fields changes nothing the step computes.  So each step
advances exactly 64M electrons and the work per step does not drift with the
step count.  Two arms on identical inputs: the table sampler
and the learned sampler (network trained here on the device).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` = particle-steps per second of the table arm
over all ranks (device-resident inputs); `arms` holds both samplers;
`e2e` = the same metric with the ensemble on pinned host memory, copied in
and the results copied out around every step; `roofline` = the lepton step's
algorithmic bytes over its CUDA-event time against the measured HBM copy
bandwidth; `cpu_baseline` = the FP64 oracle on the host's cores on a bounded
sample.  No value is printed for a run that dropped appends (capacity
overflow).  Secondary blocks: the isolated sampler, batched runs, the paper's
single-particle, uniform-field and 3D cascade configurations, and the
settings of Figs. 1, 2 and 5.  `--impl reference` times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED particle-steps/s at 64M particles (table vs MLP) and % HBM roofline"
UNIT = "particle-steps/s"
N_PART = 1 << 26
DT = 0.01
DEFAULT_STEPS, DEFAULT_WARMUP, DEFAULT_E2E_STEPS = 10, 3, 10
LEPTON_BYTES = 84       # R x,y,z,px,py,pz,w (28) + id (8) + E,B (24); W x,y,z,px,py,pz (24)
LEPTON_STREAM_BYTES = 80  # streaming pass alone: R x..pz, id, E,B (56); W x..pz (24)
PHOTON_APPEND_BYTES = 61  # x,y,z,px,py,pz,w (28) + id (8) + alive (1) + inherited E,B (24)
# DRAM bytes of one k_lepton_onepass launch of the headline workload (2^26 electrons, table
# sampler), dram__bytes_read.sum + dram__bytes_write.sum = 4.17 + 2.42 GB from one ncu capture
# of the full-size run (profiles/dram_lepton_onepass_64M.txt); reported only for that workload
LEPTON_ONEPASS_TRAFFIC_64M = 6.59e9
# photons a fresh electron of the headline ensemble emits per step: the mean of
# W_rad Dt over the ensemble is 0.184 (an upper bound of the mean event count);
# the photon buffer holds 1.6x that
PHOTONS_PER_ELECTRON_CAP = 0.3
# the lepton step runs in a single pass, appending photons in no particular
# order (the same photons as the ordered multi-pass path, bit for bit)
APPEND_ORDER = 1
QED_STATUS_CAPACITY = 1
QED_STATUS_ERRORS = 1 | 4 | 8 | 32  # capacity, non-finite, timeout, replay


def workload_desc(n):
    return {"workload": f"chi-target ensemble of {n} electrons (chi log-uniform [1e-3,1e2], gamma "
                        "log-uniform [1e2,1e4], per-particle B perp p, E=0, Dt=0.01), one fused step "
                        "(gather+Boris+chi+rate+Method I sub-steps+xi+recoil+photon append; photon "
                        "stage empty) per step; every step starts from the same momenta (restored "
                        "from a device copy, photon buffer emptied, both timed; positions keep "
                        "advancing, which with per-particle fields changes no chi or rate)",
            "particles_per_step": n, "dt": DT, "precision": "fp32 state, fp64 chi where it cancels",
            "append_order": "any (single-pass lepton kernel; photons as a set identical to the "
                            "ordered path's)" if APPEND_ORDER else "ordered",
            "samplers": ["table", "mlp"], "value_arm": "table",
            "l2": "inputs larger than L2 (>= 5.6 GB read and written per step)"}


def capacities(n):
    """Buffers of the headline run: the electrons (room for pair electrons,
    which only a run with photons at the start of a step creates), positrons,
    and photons for one step's emissions.  Every step starts from the same
    ensemble, so nothing accumulates and the sizes do not depend on the
    number of steps.  Returns (cap_e, cap_p, cap_g, max_particles)."""
    cap_e = n + n // 2
    cap_p = n // 2
    cap_g = int(PHOTONS_PER_ELECTRON_CAP * n) + 4096
    return cap_e, cap_p, cap_g, max(cap_e, cap_g)


def run_status(counters: dict) -> str:
    """'ok', or why the run's throughput is not a measurement: appends were
    dropped (capacity overflow) or a device error bit was set."""
    if counters["dropped"] > 0 or counters["status"] & QED_STATUS_CAPACITY:
        return "overflow"
    if counters["status"] & QED_STATUS_ERRORS:
        return f"device-status-{counters['status']}"
    return "ok"


def rank_id_offset(rank: int) -> int:
    """Particle ids of rank r start at r << 40, so shards never share an id."""
    return int(rank) << 40


def reduce_over_ranks(dist, ms: float, particle_steps: float, device):
    """Timing across ranks: the slowest rank's time and the total work."""
    import torch
    tt = torch.tensor([ms, particle_steps], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


COUNTER_KEYS = ("emit_events", "pair_events", "substeps", "dropped", "domain", "deferred")


def reduce_counters(dist, c: dict, device) -> dict:
    """End-of-run reduction of the event counters and the 64-bin photon
    spectrum over ranks (sums; status bits OR-ed): the only collective of the
    multi-GPU path, about 1 KB."""
    import torch
    v = torch.tensor([c[k] for k in COUNTER_KEYS] + list(c["hist"]), dtype=torch.int64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    bits = torch.tensor([(c["status"] >> b) & 1 for b in range(32)], dtype=torch.int64, device=device)
    dist.all_reduce(bits, op=dist.ReduceOp.MAX)
    vl = [int(x) for x in v.cpu().tolist()]
    out = dict(zip(COUNTER_KEYS, vl[:len(COUNTER_KEYS)]))
    out["hist"] = vl[len(COUNTER_KEYS):]
    out["status"] = sum(int(b) << i for i, b in enumerate(bits.cpu().tolist()))
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_workload(n, seed, chunk=1 << 22):
    """Generate the chi-target ensemble in chunks (float32 host arrays)."""
    from paper_1608_06356_gb300 import workloads as W
    out = {k: np.empty(n, dtype=np.float32) for k in
           ("x", "y", "z", "px", "py", "pz", "w", "ex", "ey", "ez", "bx", "by", "bz")}
    out["id"] = np.empty(n, dtype=np.uint64)
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        st, _, _ = W.chi_target(m, seed=seed * 100003 + c0 // chunk, id0=c0)
        for k, v in st.items():
            out[k][c0:c0 + m] = v
    return out


MUTABLE = ("x", "y", "z", "px", "py", "pz")
LEPTON_ARRAYS = ("x", "y", "z", "px", "py", "pz", "w", "id", "ex", "ey", "ez", "bx", "by", "bz")


class Headline:
    """The headline ensemble on the device: electrons whose positions and
    momenta live in one [6, capacity] block, a pristine copy of the momenta,
    and the positron and photon buffers.  `restore()` puts the momenta back
    into their initial state (three device copies) and empties the photon
    and positron buffers, before every step.  The positions keep advancing:
    with per-particle fields they enter neither chi nor the rates, so every
    step does the same work."""

    RESTORED = ("px", "py", "pz")

    def __init__(self, api, torch, n, host):
        cap_e, cap_p, cap_g, self.max_particles = capacities(n)
        self.n = n
        self.torch = torch
        e = api.Species.empty(cap_e, -1, fields=True)
        self.blk = torch.empty((6, cap_e), dtype=torch.float32, device="cuda")
        for r, k in enumerate(MUTABLE):
            setattr(e, k, self.blk[r])
        e.load(**host)
        self.rows = [MUTABLE.index(k) for k in self.RESTORED]
        self.pristine = self.blk[self.rows, :n].clone()
        self.e = e
        self.p = api.Species.empty(cap_p, +1, fields=True)
        self.g = api.Species.empty(cap_g, 0, fields=True)

    def restore(self):
        # one contiguous device copy per array
        for q, r in enumerate(self.rows):
            self.blk[r, :self.n].copy_(self.pristine[q])
        self.e.n.fill_(self.n)
        self.p.n.zero_()
        self.g.n.zero_()


def time_arm(api, torch, ctx, H, F, steps, warmup, step0, dist=None, profile=True):
    """W untimed and K timed headline steps on one context; returns times,
    counters and the library's per-phase event times."""
    stream = torch.cuda.current_stream()
    for s in range(warmup):
        H.restore()
        api.qed_step_fused(ctx, H.e, H.p, H.g, F, step0 + s)
    torch.cuda.synchronize()
    api.qed_reset_counters(ctx)
    if profile:
        api.qed_profile_begin(ctx, steps)
    l0 = ctx.launches
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        H.restore()
        api.qed_step_fused(ctx, H.e, H.p, H.g, F, step0 + warmup + k)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    out = {"ms": ms, "launches": ctx.launches - l0 + 0, "counters": api.qed_read_counters(ctx),
           "photons_last_step": H.g.count()}
    if profile:
        out["phases"], out["nprof"] = api.qed_profile_end_phases(ctx)
    return out


def lepton_roofline(r, n, steps, peak, peak_kind, mlp=False):
    """Roofline of the lepton step (the per-lepton unit whose algorithmic
    bytes are 84 B + 61 B per emitted photon), timed by CUDA events that the
    library records on the launching stream: the single-pass kernel (and,
    with the learned sampler, its dense pass), or the ordered path's five
    phases (streaming pass, class list, counting pass, scan, writing pass)."""
    import paper_1608_06356_gb300.api as A
    phases, nprof = r["phases"], max(r["nprof"], 1)
    lep_ms = sum(phases[k] for k in A.PROF_PHASES[:5]) / nprof
    emitted = r["counters"]["emit_events"] / steps
    lep_bytes = LEPTON_BYTES * n + PHOTON_APPEND_BYTES * emitted
    achieved = lep_bytes / (lep_ms * 1e-3) / 1e9
    stream_ms = phases["lepton_stream"] / nprof
    return {"bound": "hbm",
            "kernel": (("lepton step: k_lepton_onepass + k_net_emit (the learned sampler's dense pass)"
                        if mlp else "lepton step: k_lepton_onepass") if APPEND_ORDER else
                       "lepton step: k_lepton_stream + k_cls_count/scan/scatter + k_substep_count + "
                       "k_sub_scan + k_substep_write_coop + k_substep_replay"),
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} HBM copy (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": (LEPTON_ONEPASS_TRAFFIC_64M if APPEND_ORDER and not mlp and n == N_PART else None),
            "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum of one launch, ncu capture "
                             "of this workload (profiles/dram_lepton_onepass_64M.txt)"
                             if APPEND_ORDER and not mlp and n == N_PART else
                             "not captured for this kernel and size"),
            "bytes_per_launch": lep_bytes, "ms_per_launch": lep_ms,
            "algorithmic_bytes": "84 B per lepton + 61 B per emitted photon",
            "emitted_per_step": emitted,
            "phases_ms_per_step": {k: v / nprof for k, v in phases.items()},
            "deferred_fraction": r["counters"]["deferred"] / max(n * steps, 1),
            "streaming_pass": {"bytes_per_launch": LEPTON_STREAM_BYTES * n,
                               "ms_per_launch": stream_ms,
                               "achieved_gbs": LEPTON_STREAM_BYTES * n / (stream_ms * 1e-3) / 1e9}}


E2E_CHUNKS = 16  # chunks the host-resident ensemble is streamed in


def e2e_arm(api, torch, ctx, H, F, host, steps, step0):
    """The headline step through the public API with the ensemble in pinned
    host memory: qed_lepton_step_host streams the 64M electrons through the
    GPU in chunks (each chunk copied in, stepped, copied back, the copies of
    one chunk overlapping the step of another) and copies the new photons to
    a pinned host mirror.  Each step is timed alone (the call is
    synchronous); between steps the host ensemble is put back to its initial
    state and the photon buffers emptied, outside the timed calls."""
    n = H.n
    cap_g = H.g.capacity
    lh = api.Species.empty(n, -1, fields=True, pinned=True)
    lh.load(**{k: host[k] for k in LEPTON_ARRAYS})
    pristine = {k: getattr(lh, k)[:n].clone() for k in MUTABLE}
    gh = api.Species.empty(cap_g, 0, fields=True, pinned=True)
    chunk = (n + E2E_CHUNKS - 1) // E2E_CHUNKS
    h2d = 60 * n  # x..pz, w (28 B), id (8 B), E, B (24 B) per electron
    d2h = 0
    times = []
    warm = 2  # untimed steps first (staging buffers, first use of the pinned pages)
    for k in range(steps + warm):
        for nm in MUTABLE:
            getattr(lh, nm)[:n].copy_(pristine[nm])
        H.g.n.zero_()
        gh.n.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.qed_lepton_step_host(ctx, lh, H.g, gh, F, step0 + k, chunk)
        dt = time.perf_counter() - t0
        if k >= warm:
            times.append(dt)
            m = int(gh.n[0])
            d2h += 24 * n + 61 * m + 8  # x..pz back, the photons, the photon count
    wall = sum(times)
    return {"value": n * steps / wall, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h // steps, "steps": steps,
            "ms_per_step": 1e3 * wall / steps, "ms_each_step": [round(1e3 * t, 2) for t in times],
            "ms_median_step": 1e3 * float(np.median(times)) if times else None,
            "chunks": E2E_CHUNKS,
            "note": "ensemble in pinned host memory; every step streams the 64M electrons "
                    "(60 B each) through qed_lepton_step_host in chunks, copies their positions "
                    "and momenta back and the new photons (61 B each) to a pinned host mirror"}


def sampler_edge_u(api, torch, ctx, which, chis, edges, gamma, iters=34):
    """For each chi of `chis` and each xi of `edges`, the uniform u of the
    first word whose sample (qed_sample_table `which`: 0 the inverse table, 2
    the learned sampler) reaches xi, found by bisection over the 2^32 words
    (the samplers are monotone in u).  Returns u[len(chis), len(edges)]; the
    differences along a row are the sampler's bin probabilities."""
    C_ = np.repeat(chis, len(edges))
    X = np.tile(edges, len(chis))
    chi_d = torch.tensor(C_, device="cuda")
    g_d = torch.full_like(chi_d, gamma)
    lo = np.zeros(len(C_), dtype=np.int64)
    hi = np.full(len(C_), 2 ** 32, dtype=np.int64)  # xi(word) >= edge for word >= hi
    for _ in range(iters):
        mid = (lo + hi) // 2
        w = torch.tensor((np.minimum(mid, 2 ** 32 - 1)).astype(np.uint32).view(np.int32), device="cuda")
        xi = api.qed_sample_table(ctx, which, chi_d, g_d, w).cpu().numpy()
        below = xi < X
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return (hi.astype(np.float64) * 2.0 ** -32).reshape(len(chis), len(edges))


def spectral_error(api, torch, ctx_m, ctx_judge, n_chi=64, gamma=1e4):
    """Deterministic spectral error of the learned sampler: at n_chi values of
    chi log-spaced over its domain [1e-3, 1e2], the bin probabilities of 64 log
    bins of xi over [2/gamma, 1] that the sampler implies (sampler_edge_u)
    against those of `ctx_judge`'s FP64-built inverse table.  Returns the
    largest relative error over bins with probability >= 1e-3 and the largest
    total-variation distance, over all chi."""
    chis = np.exp(np.linspace(np.log(1e-3), np.log(1e2), n_chi))
    edges = np.exp(np.linspace(np.log(2.0 / gamma), 0.0, 65))
    um = sampler_edge_u(api, torch, ctx_m, 2, chis, edges, gamma)
    ut = sampler_edge_u(api, torch, ctx_judge, 0, chis, edges, gamma)
    pm, pt = np.diff(um, axis=1), np.diff(ut, axis=1)
    big = pt >= 1e-3
    rel = np.where(big, np.abs(pm - pt) / np.maximum(pt, 1e-300), 0.0)
    tv = 0.5 * np.abs(pm - pt).sum(axis=1)
    return {"max_rel_error_bins_p_ge_1e-3": float(rel.max()),
            "median_rel_error_bins_p_ge_1e-3": float(np.median(rel[big])),
            "max_total_variation": float(tv.max()), "chi_nodes": n_chi, "bins": 64,
            "gamma": gamma, "judge": "inverse table of the same library, built in FP64 (bisection in u)"}


def sampler_comparison(api, torch, n, ctx_t, ctx_m, reps=5):
    """Isolated inverse-CDF sampler (qed_sample_xi) at n samples, table vs the
    learned network: 12 B per sample (chi, gamma read, xi written)."""
    rng = np.random.default_rng(123)
    chi = torch.tensor(np.exp(rng.uniform(np.log(1e-3), np.log(1e2), n)).astype(np.float32), device="cuda")
    gam = torch.tensor(np.exp(rng.uniform(np.log(1e2), np.log(1e4), n)).astype(np.float32), device="cuda")
    out = torch.empty(n, device="cuda")
    res = {}
    peak, _ = peaks()
    for name, ctx in (("table", ctx_t), ("mlp", ctx_m)):
        for s in range(3):
            api.qed_sample_xi(ctx, chi, gam, out, s)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for s in range(reps):
            api.qed_sample_xi(ctx, chi, gam, out, 10 + s)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        res[name] = {"samples_per_s": n / (ms * 1e-3), "ms_per_launch": ms,
                     "achieved_gbs": 12 * n / (ms * 1e-3) / 1e9,
                     "frac_hbm": 12 * n / (ms * 1e-3) / 1e9 / peak}
    # tensor work of the network: layers 2 and 3, 64x64 MACs, three split-BF16 products each
    res["mlp"]["tensor_tflops"] = 2 * 3 * 2 * 64 * 64 * res["mlp"]["samples_per_s"] / 1e12
    res["mlp_over_table_speed"] = res["mlp"]["samples_per_s"] / res["table"]["samples_per_s"]
    res["n"] = n
    return res


def batched_runs_bench(api, torch, mlp_weights, steps=4):
    """256 independent ensembles of uneven size (log-uniform in [1e3, 1e6]) with
    per-run chi ranges (two sorted log-uniform draws in [0.01, 10]), advanced
    together: eager launches vs one captured CUDA graph per `steps` steps,
    table and learned samplers, each with the launch sizes (CTAs per SM per
    kernel group) its autotuner chose on a copy of the runs."""
    from paper_1608_06356_gb300 import workloads as W
    sizes, ranges = W.batched_runs(256, seed=0)
    parts, off = [], 0
    for r, (n, (lo, hi)) in enumerate(zip(sizes, ranges)):
        st, _, _ = W.chi_target(int(n), seed=5000 + r, chi_lo=lo, chi_hi=hi, id0=off)
        st = {k: (v.astype(np.float32) if v.dtype.kind == "f" else v) for k, v in st.items()}
        st["tag"] = np.full(int(n), r, dtype=np.uint32)
        parts.append(st)
        off += int(n)
    host = {k: np.concatenate([q[k] for q in parts]) for k in parts[0]}
    n = off
    F = api.Fields.per_particle()
    out = {"runs": 256, "particles": int(n), "steps": steps}
    for name, sampler in (("table", 0), ("mlp", 1)):
        res = {}
        tuning = None
        for mode in ("eager", "graph"):
            ctx = api.qed_init_tables(api.config(dt=DT, seed=11, sampler=sampler,
                                                 max_particles=int(0.4 * n * (steps + 2)) + n,
                                                 append_order=APPEND_ORDER))
            if sampler:
                api.qed_mlp_load(ctx, mlp_weights)
            if tuning is None:  # launch sizes per kernel group, on disposable copies
                e = api.Species.empty(2 * n, -1, fields=True, tag=True).load(**host)
                p = api.Species.empty(n, 1, fields=True, tag=True)
                g = api.Species.empty(int(0.4 * n * (steps + 2)), 0, fields=True, tag=True)
                tuning = api.qed_autotune_groups(ctx, e, p, g, F, reps=2)
                res["tuning"] = {"grid_factor_ctas_per_sm": tuning["grid_factor"],
                                 "chain_scheduling": tuning["sched"],
                                 "ms_per_step_tuned": tuning["ms_per_step"],
                                 "ms_per_factor": tuning["ms"],
                                 "ms_per_scheduling_value": tuning["sched_ms"]}
                del e, p, g
            else:
                api.qed_set_tuning(ctx, tuning["grid_factor"], tuning["sched"])
            e = api.Species.empty(2 * n, -1, fields=True, tag=True).load(**host)
            p = api.Species.empty(n, 1, fields=True, tag=True)
            g = api.Species.empty(int(0.4 * n * (steps + 2)), 0, fields=True, tag=True)
            cnt = torch.zeros((steps, 3), dtype=torch.int64, device="cuda")
            if mode == "graph":  # capture (first call), then time a replay from the same state
                api.qed_run_batched(ctx, e, p, g, F, 0, steps)
            else:  # load kernels (ours and torch's) once, then restore the state
                cnt[0, 0].copy_(e.n[0] + p.n[0])
                cnt[0, 1].copy_(g.n[0])
                api.qed_step_fused(ctx, e, p, g, F, 0)
                api.qed_compact_fill(ctx, g)
            torch.cuda.synchronize()
            e.load(**host)
            p.n.zero_()
            g.n.zero_()
            api.qed_reset_counters(ctx)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = ctx.launches
            a.record()
            if mode == "graph":
                runs_out = api.qed_run_batched(ctx, e, p, g, F, 0, steps, n_runs=256)
            else:
                for k in range(steps):
                    cnt[k, 0].copy_(e.n[0] + p.n[0])
                    cnt[k, 1].copy_(g.n[0])
                    api.qed_step_fused(ctx, e, p, g, F, k)
                    api.qed_compact_fill(ctx, g)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            c = api.qed_read_counters(ctx)
            res[mode + "_status"] = run_status(c)
            if mode == "eager":
                res["particle_steps"] = float(cnt.sum().item())
                res["eager_launches"] = ctx.launches - l0
            res[mode + "_ms_per_step"] = ms / steps
            if mode == "graph":
                res["photons_per_run_min_max"] = [int(runs_out.min()), int(runs_out.max())]
        ps = res["particle_steps"]
        res["eager_particle_steps_per_s"] = ps / (res["eager_ms_per_step"] * steps * 1e-3)
        res["graph_particle_steps_per_s"] = ps / (res["graph_ms_per_step"] * steps * 1e-3)
        out[name] = res
    return out


def generator_rates(api, torch, steps=480, dt=0.01):
    """The paper's Fig. 2 setting: one electron per cell of 128 x 192 cells,
    gamma = 206, B giving chi_e = 0.1, 480 steps; the average photon
    generation rate with event generators I, II and III against W_rad at the
    initial state (Eq. 1 with the xi_min cut, from the GPU's tables)."""
    n, gamma0, bz = 128 * 192, 206.0, 200.0
    p0 = np.float32(np.sqrt(gamma0 ** 2 - 1.0))
    chi = float(p0) * bz / api.config().a_S  # |p x B| / a_S for p along x, B along z, E = 0
    out = {"electrons": n, "gamma0": gamma0, "chi0": chi, "steps": steps, "dt": dt}
    for gen, name in ((0, "I"), (1, "II"), (2, "III")):
        ctx = api.qed_init_tables(api.config(dt=dt, seed=17, generator=gen))
        z = np.zeros(n, np.float32)
        e = api.Species.empty(n, -1, od=gen != 0).load(
            x=z, y=z, z=z, px=np.full(n, p0, np.float32), py=z, pz=z, w=np.ones(n, np.float32),
            id=np.arange(n, dtype=np.uint64))
        g = api.Species.empty(n * 16, 0)
        F = api.Fields.uniform((0, 0, 0), (0, 0, bz))
        per_step = torch.zeros(steps, dtype=torch.int64, device="cuda")
        for s in range(steps):
            api.qed_gather_push(ctx, e, F, s)
            api.qed_emit(ctx, e, g, F, s)
            per_step[s].copy_(g.n[0])
        torch.cuda.synchronize()
        cum = per_step.cpu().numpy()
        W0 = float(api.qed_rates(ctx, 0, torch.tensor([chi], device="cuda"),
                                 torch.tensor([float(np.sqrt(1 + float(p0) ** 2))], device="cuda"))[0])
        out["W_rad_initial"] = W0
        out[name] = {"rate_first_48_steps": float(cum[47]) / (n * 48 * dt),
                     "rate_all_steps": float(cum[-1]) / (n * steps * dt),
                     "status": run_status(api.qed_read_counters(ctx))}
    return out


def spectra_fig1(api, torch, nu=1 << 20, gamma=1000.0):
    """Fig. 1's comparison: photon-energy spectra (dW/dxi, 16 log bins of xi
    over [2/gamma, 1]) sampled with the formula-I and the classic-limit
    tables at chi = 0.1, 1 and 10, and their ratio per bin (null where the
    formula-I bin is empty)."""
    edges = np.exp(np.linspace(np.log(2.0 / gamma), 0.0, 17))
    out = {"gamma": gamma, "samples": nu, "xi_edges": edges.tolist()}
    hist = {}
    for model, name in ((0, "formula_I"), (1, "classic")):
        ctx = api.qed_init_tables(api.config(model=model))
        for chi in (0.1, 1.0, 10.0):
            c = torch.full((nu,), chi, device="cuda")
            g = torch.full((nu,), gamma, device="cuda")
            xi = torch.empty(nu, device="cuda")
            api.qed_sample_xi(ctx, c, g, xi, 3)
            # rate-weighted: the classic and formula-I totals differ
            W = float(api.qed_rates(ctx, 0, torch.tensor([chi], device="cuda"),
                                    torch.tensor([gamma], device="cuda"))[0])
            cnt = np.histogram(xi.cpu().numpy(), edges)[0]
            hist[(name, chi)] = (cnt, cnt / nu * W / np.diff(edges))
    for chi in (0.1, 1.0, 10.0):
        cI, dI = hist[("formula_I", chi)]
        cC, dC = hist[("classic", chi)]
        ratio = [float(a / b) if n > 0 else None for a, b, n in zip(dC, dI, cI)]
        out[f"chi_{chi:g}"] = {"dW_dxi_formula_I": dI.tolist(), "classic_over_formula_I": ratio}
    return out


def cascade_fig5(api, torch, runs=4000, t_end_trad=2.5, steps_per_trad=60):
    """The paper's cascade benchmark setting (Fig. 5): one electron per run,
    gamma = 2e5, in a static B = 0.2 E_S perpendicular to its motion
    (chi_e = 4e4; tables extended to chi = 1e5); pairs with energy above
    100 MeV (positrons with gamma > 195.7) per run against time in units of
    t_rad = 1.16e-16 s, over `runs` independent runs (one ensemble: the runs
    do not interact).  Dead photons are compacted every step."""
    a_S = api.config().a_S
    lam = 1e-6
    omega0 = 2 * np.pi * 299792458.0 / lam
    t_rad = 1.16e-16 * omega0  # in 1/omega0
    dt = t_rad / steps_per_trad
    steps = int(round(t_end_trad * steps_per_trad))
    n = runs
    phi = np.random.default_rng(0).uniform(0, 2 * np.pi, n)
    p0 = np.sqrt(2e5 ** 2 - 1.0)
    z = np.zeros(n, np.float32)
    cap = 1 << 27  # ~1.4e4 leptons and ~1.7e4 photons per run by 2.5 t_rad
    ctx = api.qed_init_tables(api.config(dt=dt, seed=23, chi_max=1e5, chi_pair_max=1e5,
                                         max_particles=cap))
    e = api.Species.empty(cap, -1).load(x=z, y=z, z=z, px=(p0 * np.cos(phi)).astype(np.float32),
                                        py=(p0 * np.sin(phi)).astype(np.float32), pz=z,
                                        w=np.ones(n, np.float32), id=np.arange(n, dtype=np.uint64))
    p = api.Species.empty(cap, 1)
    g = api.Species.empty(cap, 0)
    F = api.Fields.uniform((0, 0, 0), (0, 0, 0.2 * a_S))
    g_cut = 100e6 / 510998.95  # 100 MeV in m c^2
    times, pairs = [0.0], [0.0]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps = 0
    t0.record()
    for s in range(steps):
        ps += e.count() + p.count() + g.count()
        api.qed_step_fused(ctx, e, p, g, F, s)
        api.qed_compact(ctx, g)
        if (s + 1) % (steps_per_trad // 4) == 0:
            m = p.count()
            gp = torch.sqrt(1 + p.px[:m].double() ** 2 + p.py[:m].double() ** 2 + p.pz[:m].double() ** 2)
            times.append((s + 1) / steps_per_trad)
            pairs.append(float((gp > g_cut).sum().item()) / n)
    t1.record()
    torch.cuda.synchronize()
    c = api.qed_read_counters(ctx)
    return {"runs": n, "gamma0": 2e5, "B_over_E_S": 0.2, "chi0": 2e5 * 0.2, "dt_over_t_rad": 1.0 / steps_per_trad,
            "t_rad_in_inverse_omega0": t_rad, "steps": steps,
            "t_over_t_rad": times, "pairs_above_100MeV_per_run": pairs,
            "pairs_per_run_total": c["pair_events"] / n, "photons_emitted_per_run": c["emit_events"] / n,
            "status": run_status(c), "dropped": c["dropped"],
            "particles_at_end": {"electrons": e.count(), "positrons": p.count(), "photons": g.count()},
            "particle_steps_per_s": ps / (t0.elapsed_time(t1) * 1e-3),
            "note": "wall time includes a host read of the counts every step"}


def _block_roofline(bytes_per_step, ms_per_step, peak, peak_kind, bound="hbm"):
    a = bytes_per_step / (ms_per_step * 1e-3) / 1e9
    return {"bound": bound, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
            "peak_source": f"{peak_kind} HBM copy"}


def _oracle_block_baseline(make_species, cfg_kw, fields, steps):
    """The oracle on a bounded sample of a configuration: particle-steps/s."""
    import oracle as O
    O.build()
    cfg = O.make_config(**cfg_kw)
    e, p, g = make_species(O)
    ps, t0 = 0, time.perf_counter()
    for s in range(steps):
        ps += e.n + p.n + g.n
        O.step(cfg, fields(O), e, p, g, s)
    dt = time.perf_counter() - t0
    return {"value": ps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "seconds": dt, "particle_steps": ps}


def config_single_particle(api, torch, n=10_000, steps=1000, cpu_n=2000, cpu_steps=2):
    """The paper's single-particle-type test: 10^4 electrons, gamma0 = 1000 along
    x, uniform B = 410 along z (chi_e ~ 1), E = 0, Dt = 0.01, 1000 steps, photon
    emission only (formula I), FP64, Philox seed 0; output: the photon
    spectrum in 64 log bins of energy over [2, 1000] m c^2.  Launch-bound
    (10^4 particles per launch), so its roofline is reported for context."""
    from paper_1608_06356_gb300 import workloads as W
    st, fld = W.single(n)
    ctx = api.qed_init_tables(api.config(dt=0.01, seed=0, precision=1, max_particles=1 << 22))
    e = api.Species.empty(n, -1, dtype=torch.float64).load(**st)
    g = api.Species.empty(1 << 22, 0, dtype=torch.float64)
    F = api.Fields.uniform(fld["E"], fld["B"])
    for s in range(3):  # load the kernels
        api.qed_gather_push(ctx, e, F, s)
        api.qed_emit(ctx, e, g, F, s)
    e.load(**st)
    g.n.zero_()
    api.qed_reset_counters(ctx)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for s in range(steps):
        api.qed_gather_push(ctx, e, F, s)
        api.qed_emit(ctx, e, g, F, s)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    c = api.qed_read_counters(ctx)
    peak, kind = peaks()
    # FP64: lepton 64 B read + 48 B written (push + emission read it again: 2x), photon append 64 B
    bytes_step = 2 * (64 + 48) * n + 64 * c["emit_events"] / steps
    base = _oracle_block_baseline(
        lambda O: (O.Species(cpu_n, -1.0).load(**{k: v[:cpu_n] for k, v in st.items()}),
                   O.Species(1, 1.0), O.Species(cpu_n * 4, 0.0, with_alive=True)),
        {"dt": 0.01, "seed": 0}, lambda O: O.uniform_fields(fld["E"], fld["B"]), cpu_steps)
    base["sample"] = f"{cpu_n} electrons x {cpu_steps} steps (fused oracle step; no photons present)"
    return {"electrons": n, "steps": steps, "precision": "fp64", "status": run_status(c),
            "particle_steps_per_s": n * steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "photons": g.count(), "emit_events": c["emit_events"],
            "photon_spectrum_64_log_bins_2_to_1000": c["hist"],
            "roofline": _block_roofline(bytes_step, ms / steps, peak, kind, bound="launch"),
            "cpu_baseline": base}


def config_uniform_ensemble(api, torch, n=1 << 20, steps=200, compact_every=4, cpu_n=1024):
    """The uniform-field ensemble: 2^20 electrons + 2^20 photons, gamma (and
    photon |p|) log-uniform in [1e2, 1e4], isotropic directions, per-particle E,
    B with isotropic directions and magnitudes log-uniform in [10, 2000];
    emission and Breit-Wheeler pairs, FP32 state (FP32 table look-ups, FP64
    chi where it cancels), Dt = 0.01, 200 steps; children inherit their
    parent's fields; photons appended in any order (the single-pass lepton
    step).  Dead photons are removed every 4 steps (qed_compact_fill)."""
    from paper_1608_06356_gb300 import workloads as W
    se = W.ensemble(n, seed=0)
    sg = W.ensemble(n, seed=1, photons=True, id0=1 << 32)
    f32 = lambda d: {k: (v.astype(np.float32) if v.dtype.kind == "f" else v) for k, v in d.items()}
    se, sg = f32(se), f32(sg)
    cap = 1 << 25
    ctx = api.qed_init_tables(api.config(dt=DT, seed=3, max_particles=cap, append_order=APPEND_ORDER))
    e = api.Species.empty(cap, -1, fields=True).load(**se)
    p = api.Species.empty(cap, 1, fields=True)
    g = api.Species.empty(cap, 0, fields=True).load(**sg)
    F = api.Fields.per_particle()
    cnt = torch.zeros((steps, 2), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for s in range(steps):
        cnt[s, 0].copy_(e.n[0] + p.n[0])
        api.qed_count_alive(ctx, g, cnt[s, 1:2])
        api.qed_step_fused(ctx, e, p, g, F, s)
        if (s + 1) % compact_every == 0:
            api.qed_compact_fill(ctx, g)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    c = api.qed_read_counters(ctx)
    cn = cnt.cpu().numpy()
    ps = float(cn.sum())
    peak, kind = peaks()
    # lepton 84 B, photon 68 B per particle-step; appends 61 B per photon, 2 x 61 + 1 B per pair
    bytes_total = 84 * cn[:, 0].sum() + 68 * cn[:, 1].sum() + 61 * c["emit_events"] + 123 * c["pair_events"]
    base = _oracle_block_baseline(
        lambda O: (O.Species(cpu_n * 4, -1.0, per_particle_fields=True).load(
                       **{k: v[:cpu_n].astype(np.float64) if v.dtype.kind == "f" else v[:cpu_n]
                          for k, v in se.items()}),
                   O.Species(cpu_n * 2, 1.0, per_particle_fields=True),
                   O.Species(cpu_n * 8, 0.0, per_particle_fields=True, with_alive=True).load(
                       **{k: v[:cpu_n].astype(np.float64) if v.dtype.kind == "f" else v[:cpu_n]
                          for k, v in sg.items()})),
        {"dt": DT, "seed": 3}, lambda O: O.per_particle_fields(), 2)
    base["sample"] = f"{cpu_n} electrons + {cpu_n} photons of the same ensemble x 2 steps"
    return {"electrons": n, "photons": n, "steps": steps, "status": run_status(c),
            "particle_steps_per_s": ps / (ms * 1e-3), "ms_per_step": ms / steps,
            "particles_at_end": {"leptons": e.count() + p.count(), "photons_alive": int(cn[-1, 1])},
            "emit_events": c["emit_events"], "pair_events": c["pair_events"],
            "roofline": _block_roofline(bytes_total / steps, ms / steps, peak, kind),
            "cpu_baseline": base}


def config_3d_cascade(api, torch, steps=28, seed_n=1 << 24, cap=1 << 28, nx=256, a0=800.0,
                      dt=0.1, compact_every=2, cpu_n=4096):
    """The 3D PIC-like cascade: a 256^3 periodic grid (dx = 2 pi / 32) of two
    counter-propagating circularly polarised standing waves of amplitude
    a0 = 800 each, filled on the device at every step's time; 16M electrons at
    rest, uniform in the central 64^3 cells; CIC gather + Boris + emission and
    pairs with in-place appends into preallocated 256M-slot buffers per species
    (photons in any order: the single-pass lepton step), FP32, Dt = 0.1.  The first `steps` of the 500-step run are timed (a slice):
    the particle count grows and the step cost with it.  Grid bytes: the field
    fill (32 B per node written) plus one read of the touched nodes' 32 B."""
    from paper_1608_06356_gb300 import workloads as W
    dx = 2 * np.pi / 32
    st = W.cascade_seed(seed_n, seed=0, nx=nx, dx=dx)
    st = {k: (v.astype(np.float32) if v.dtype.kind == "f" else v) for k, v in st.items()}
    ctx = api.qed_init_tables(api.config(dt=dt, seed=9, max_particles=cap, append_order=APPEND_ORDER))
    e = api.Species.empty(cap, -1).load(**st)
    p = api.Species.empty(cap, 1)
    g = api.Species.empty(cap, 0)
    grid = torch.zeros((nx, nx, nx, 8), dtype=torch.float32, device="cuda")
    F = api.Fields.grid(grid, dx, dx, dx)
    cnt = torch.zeros((steps, 2), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for s in range(steps):
        cnt[s, 0].copy_(e.n[0] + p.n[0])
        api.qed_count_alive(ctx, g, cnt[s, 1:2])
        api.qed_fill_standing_wave(ctx, grid, 0.0, dx, a0, s * dt)
        api.qed_step_fused(ctx, e, p, g, F, s)
        if (s + 1) % compact_every == 0:
            api.qed_compact_fill(ctx, g)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    c = api.qed_read_counters(ctx)
    cn = cnt.cpu().numpy()
    ps = float(cn.sum())
    peak, kind = peaks()
    nodes = nx ** 3
    bytes_total = (60 * cn[:, 0].sum() + 44 * cn[:, 1].sum() + 37 * c["emit_events"]
                   + 73 * c["pair_events"] + 2 * 32 * nodes * steps)
    e_n, p_n, g_n = e.count(), p.count(), g.count()
    del e, p, g, grid
    torch.cuda.empty_cache()

    def mk(O):
        sub = {k: (v[:cpu_n].astype(np.float64) if v.dtype.kind == "f" else v[:cpu_n]) for k, v in st.items()}
        return (O.Species(cpu_n * 4, -1.0).load(**sub), O.Species(cpu_n * 2, 1.0),
                O.Species(cpu_n * 8, 0.0, with_alive=True))

    def fields(O):
        return O.grid_fields(O.fill_standing_wave(nx, nx, nx, 0.0, dx, a0, 0.0), dx, dx, dx)

    try:
        base = _oracle_block_baseline(mk, {"dt": dt, "seed": 9}, fields, 2)
        base["sample"] = f"{cpu_n} seed electrons x 2 steps (grid fields at t = 0)"
    except Exception as ex:
        base = {"error": repr(ex)}
    return {"grid": [nx, nx, nx], "a0": a0, "seed_electrons": seed_n, "capacity_per_species": cap,
            "steps_timed": steps, "steps_of_run": 500, "dt": dt, "status": run_status(c),
            "particle_steps_per_s": ps / (ms * 1e-3), "ms_per_step": ms / steps,
            "particles_per_step_first_last": [int(cn[0].sum()), int(cn[-1].sum())],
            "particles_at_end": {"electrons": e_n, "positrons": p_n, "photons_slots": g_n},
            "emit_events": c["emit_events"], "pair_events": c["pair_events"],
            "roofline": _block_roofline(bytes_total / steps, ms / steps, peak, kind),
            "field_fill_bytes_per_step": 32 * nodes, "cpu_baseline": base}


def _pic_oracle_sample(W, cpu_nx, cpu_ppc, dx, dt):
    """The oracle loop (oracle step + numpy deposit and Yee step) on a small
    warm plasma, 2 cycles: particle-steps/s."""
    import oracle as O
    from oracle import pic as P
    O.build()
    sub = W.plasma(cpu_nx, cpu_nx, cpu_nx, dx, ppc=cpu_ppc, density=0.05, p_th=0.1, seed=4)
    sub = {k: (v.astype(np.float32).astype(np.float64) if v.dtype.kind == "f" else v) for k, v in sub.items()}
    cfg = O.make_config(dt=dt, seed=2)
    oe = O.Species(len(sub["x"]), -1.0).load(**sub)
    og = O.Species(16, 0.0, with_alive=True)
    grid = P.Grid(cpu_nx, cpu_nx, cpu_nx, dx, dx, dx)
    t0 = time.perf_counter()
    for s in range(2):
        P.loop_step(cfg, grid, oe, None, og, s)
    sec = time.perf_counter() - t0
    return {"value": 2 * oe.n / sec, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{cpu_nx}^3 cells x {cpu_ppc} electrons per cell x 2 cycles "
                      "(oracle step + numpy deposit and Yee step)", "seconds": sec}


def pic_loop_bench(api, torch, nx=256, ppc=1, steps=20, dx=0.25, dt=0.1, cpu_nx=24, cpu_ppc=4,
                   cell_order=True):
    """The self-consistent loop (qed_pic_step): a warm electron plasma at
    0.05 n_c, thermal momenta 0.1 m c per axis, `ppc` electrons per cell at
    random positions on a periodic nx^3 Yee grid (dx = 0.25, Dt = 0.1); at
    256^3 the field arrays (1.1 GB) and the particles are larger than L2.
    Each cycle is the QED step gathering from the node grid, the current
    deposit and the field leapfrog with the node grid.  The cycles are timed
    whole, then once more with events between the phases.  Field bytes: 188 B
    per cell per cycle (B half-step 36, E step 60 with J zeroed, B half-step
    36, nodes 56); the deposit reads 28 B per particle and adds its 24 CIC
    contributions (about 15 atomic operations) into J.  cell_order: the
    particles stored by cell (as a PIC code's periodic sort keeps them), else
    in random order, where the gather and the deposit touch a random cell per
    particle."""
    from paper_1608_06356_gb300 import workloads as W
    st = W.plasma(nx, nx, nx, dx, ppc=ppc, density=0.05, p_th=0.1, seed=4, cell_order=cell_order)
    st = {k: (v.astype(np.float32) if v.dtype.kind == "f" else v) for k, v in st.items()}
    n = len(st["x"])
    ctx = api.qed_init_tables(api.config(dt=dt, seed=2, max_particles=n))
    e = api.Species.empty(n, -1).load(**st)
    p = api.Species.empty(0, 1)
    g = api.Species.empty(1 << 16, 0)
    y = api.Yee(nx, nx, nx, dx, dx, dx)
    api.qed_pic_fields(ctx, y, advance=False)
    for s in range(3):  # warm-up cycles
        api.qed_pic_step(ctx, e, p, g, y, 1.0, s)
    api.qed_reset_counters(ctx)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for s in range(3, 3 + steps):
        api.qed_pic_step(ctx, e, p, g, y, 1.0, s)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # the same cycle by its parts, with events between them
    F = y.fields()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for s in range(steps):
        k = 3 + steps + s
        ev[s][0].record()
        api.qed_step_fused(ctx, e, p, g, F, k)
        ev[s][1].record()
        api.qed_pic_deposit(ctx, e, y, 1.0)
        ev[s][2].record()
        api.qed_pic_fields(ctx, y, advance=True)
        ev[s][3].record()
    torch.cuda.synchronize()
    ph = [sum(ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(steps)) / steps for i in range(3)]
    c = api.qed_read_counters(ctx)
    peak, kind = peaks()
    cells = nx ** 3
    field_bytes = 188 * cells
    if cpu_nx > 0:
        try:
            base = _pic_oracle_sample(W, cpu_nx, cpu_ppc, dx, dt)
        except Exception as ex:
            base = {"error": repr(ex)}
    else:
        base = {"note": "no CPU sample for this variant: the oracle's rate does not depend on the "
                        "particle order (see the cell-ordered block)"}
    return {"grid": [nx, nx, nx], "electrons": n, "electrons_per_cell": ppc, "steps_timed": steps,
            "particle_order": "by cell" if cell_order else "random",
            "dt": dt, "dx": dx, "status": run_status(c),
            "particle_steps_per_s": n / (ms * 1e-3), "ms_per_cycle": ms,
            "ms_per_phase": {"qed_step": ph[0], "deposit": ph[1], "fields": ph[2]},
            "fields_roofline": _block_roofline(field_bytes, ph[2], peak, kind),
            "deposit_contributions_per_s": 24 * n / (ph[1] * 1e-3),
            "deposit_read_gbs": 28 * n / (ph[1] * 1e-3) / 1e9,
            "photons": g.count(), "cpu_baseline": base}


def oracle_sample_rate(sample_n, steps, seed=0):
    """The FP64 oracle as it stands on `sample_n` electrons of the headline
    ensemble, `steps` steps, each from the same initial state (as the
    headline's steps are); returns (particle-steps/s, cores, seconds)."""
    import oracle as O
    from paper_1608_06356_gb300 import workloads as W
    O.build()
    st, _, _ = W.chi_target(sample_n, seed=seed)
    st = {k: (v.astype(np.float32).astype(np.float64) if v.dtype.kind == "f" else v)
          for k, v in st.items()}
    cfg = O.make_config(dt=DT, seed=1)
    f = O.per_particle_fields()
    total = 0.0
    for s in range(steps):
        e = O.Species(sample_n * 2, -1.0, per_particle_fields=True).load(**st)
        p = O.Species(sample_n, 1.0, per_particle_fields=True)
        g = O.Species(sample_n * 2, 0.0, per_particle_fields=True, with_alive=True)
        t0 = time.perf_counter()
        O.step(cfg, f, e, p, g, s)
        total += time.perf_counter() - t0
    return sample_n * steps / total, O.num_threads(), total


def cpu_baseline(sample_n=12288, steps=2):
    v, cores, secs = oracle_sample_rate(sample_n, steps)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sample_n} electrons of the headline ensemble x {steps} step(s), each from "
                      f"the initial state ({sample_n * steps} particle-steps in {secs:.1f} s), "
                      "FP64 quadrature rates"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.ref_particles
    oracle_sample_rate(n, args.warmup)  # warm-up steps (untimed)
    v, cores, secs = oracle_sample_rate(n, args.steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_desc(N_PART),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} electrons of the headline ensemble per step, each step "
                                       "from the initial state"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=DEFAULT_STEPS)
    ap.add_argument("--warmup", type=int, default=DEFAULT_WARMUP)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--particles", type=int, default=N_PART)
    ap.add_argument("--e2e-steps", type=int, default=DEFAULT_E2E_STEPS)
    ap.add_argument("--ref-particles", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mlp-train-samples", type=float, default=1.6e10)
    ap.add_argument("--sampler-bench", type=int, default=1)
    ap.add_argument("--batched-bench", type=int, default=1)
    ap.add_argument("--configs-bench", type=int, default=1)
    ap.add_argument("--generator-bench", type=int, default=1)
    ap.add_argument("--cascade-bench", type=int, default=1)
    ap.add_argument("--spectra-bench", type=int, default=1)
    ap.add_argument("--pic-bench", type=int, default=1)
    ap.add_argument("--append-order", choices=["any", "ordered"], default="any",
                    help="lepton step of the headline arms: single pass (any) or the ordered path")
    args = ap.parse_args()
    global APPEND_ORDER
    APPEND_ORDER = 1 if args.append_order == "any" else 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1608_06356_gb300 import api

    n = args.particles
    host = host_workload(n, seed=rank)
    host["id"] += np.uint64(rank_id_offset(rank))
    H = Headline(api, torch, n, host)
    F = api.Fields.per_particle()
    ctx_t = api.qed_init_tables(api.config(dt=DT, seed=1 + rank, max_particles=H.max_particles,
                                           append_order=APPEND_ORDER))
    ctx_m = api.qed_init_tables(api.config(dt=DT, seed=1 + rank, max_particles=H.max_particles,
                                           sampler=1, append_order=APPEND_ORDER))
    api.qed_mlp_load(ctx_m, api.mlp_init_params(0))
    t_train = time.perf_counter()
    train_loss = api.qed_mlp_train(ctx_m, int(args.mlp_train_samples), lr=6e-3, seed=7)
    train_s = time.perf_counter() - t_train
    wts = api.qed_mlp_get(ctx_m)
    dd = dist if world > 1 else None

    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    arms = {}
    for name, ctx in (("table", ctx_t), ("mlp", ctx_m)):
        arms[name] = time_arm(api, torch, ctx, H, F, args.steps, args.warmup, 0, dd)
    clocks = clk.stop()

    peak, peak_kind = peaks()
    arm_out = {}
    for name, r in arms.items():
        c = r["counters"]
        t_max, ps_total = r["ms"], float(n * args.steps)
        if world > 1:
            t_max, ps_total = reduce_over_ranks(dist, r["ms"], ps_total, "cuda")
            c = reduce_counters(dist, c, "cuda")
        status = run_status(c)
        arm_out[name] = {"value": ps_total / (t_max * 1e-3) if status == "ok" else None,
                         "status": status, "ms_per_step": t_max / args.steps,
                         "gpu_launches": r["launches"],
                         "roofline": lepton_roofline(r, n, args.steps, peak, peak_kind, mlp=name == "mlp"),
                         "counters": {k: c[k] for k in COUNTER_KEYS + ("status",)},
                         "photons_per_step": r["photons_last_step"],
                         "hist_64_log_bins_2_to_1000": c["hist"]}
    arm_out["mlp"]["train"] = {"samples": int(args.mlp_train_samples), "seconds": train_s,
                               "final_mse_lndelta": train_loss}
    arm_out["mlp_over_table_speed"] = arm_out["table"]["ms_per_step"] / arm_out["mlp"]["ms_per_step"]
    T = arm_out["table"]
    status = T["status"]

    e2e = None
    if args.e2e_steps > 0 and status == "ok":
        e2e = e2e_arm(api, torch, ctx_t, H, F, host, args.e2e_steps, 10_000)
        if world > 1:  # whole job: all ranks' particle-steps over the slowest rank's time
            wall_ms, ps = reduce_over_ranks(dist, e2e["ms_per_step"] * args.e2e_steps,
                                            float(n * args.e2e_steps), "cuda")
            e2e["value"] = ps / (wall_ms * 1e-3)
            e2e["ms_per_step"] = wall_ms / args.e2e_steps
            nb = torch.tensor([e2e["h2d_bytes_per_step"], e2e["d2h_bytes_per_step"]],
                              dtype=torch.float64, device="cuda")
            dist.all_reduce(nb, op=dist.ReduceOp.SUM)
            e2e["h2d_bytes_per_step"], e2e["d2h_bytes_per_step"] = int(nb[0]), int(nb[1])
    del host

    extra = {}
    if rank == 0:
        try:
            extra["spectral_error_mlp"] = spectral_error(api, torch, ctx_m, ctx_t)
        except Exception as ex:  # report, do not hide the headline
            extra["spectral_error_mlp"] = {"error": repr(ex)}
        if args.sampler_bench:
            extra["sampler_table_vs_mlp"] = sampler_comparison(api, torch, n, ctx_t, ctx_m)
    del H
    torch.cuda.empty_cache()
    if rank == 0:
        if args.batched_bench:
            extra["batched_runs"] = batched_runs_bench(api, torch, wts)
        if args.configs_bench:
            extra["config_single_particle_fp64"] = config_single_particle(api, torch)
            extra["config_uniform_field_ensemble"] = config_uniform_ensemble(api, torch)
            extra["config_3d_cascade"] = config_3d_cascade(api, torch)
        if args.pic_bench:
            try:
                extra["pic_loop"] = pic_loop_bench(api, torch)
                extra["pic_loop_random_order"] = pic_loop_bench(api, torch, cell_order=False,
                                                                cpu_nx=0)
            except Exception as ex:  # report, do not hide the headline
                extra["pic_loop"] = {"error": repr(ex)}
        if args.generator_bench:
            extra["event_generators_fig2"] = generator_rates(api, torch)
        if args.cascade_bench:
            extra["cascade_fig5"] = cascade_fig5(api, torch)
        if args.spectra_bench:
            extra["spectra_fig1"] = spectra_fig1(api, torch)

    line = {"metric": METRIC, "value": T["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": T["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "status": status, "config": workload_desc(n),
            "roofline": T["roofline"], "e2e": e2e, "gpu_launches": T["gpu_launches"],
            "clocks": clocks, "arms": arm_out}
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
