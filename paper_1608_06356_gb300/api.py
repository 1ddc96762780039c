"""Python face of libqed: the C-ABI calls under the same names, with torch
tensors as the caller-owned device buffers.

    ctx = qed_init_tables(config(dt=0.01))
    e = Species.empty(capacity, q=-1, device="cuda")
    qed_step_fused(ctx, e, p, g, Fields.uniform(E, B), step)

Only marshalling happens here; all particle work is done by the kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as B

STATE = ("x", "y", "z", "px", "py", "pz", "w")
FIELD_NAMES = ("ex", "ey", "ez", "bx", "by", "bz")


def config(**kw) -> B.qed_config:
    """qed_config with the library defaults, overridden by keyword."""
    c = B.qed_config()
    B.lib().qed_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Context:
    """Owns a qed_ctx (tables, scan state, counters)."""

    def __init__(self, cfg: B.qed_config, stream=None):
        self.cfg = cfg
        self.handle = C.c_void_p()
        B.check(B.lib().qed_init_tables(C.byref(cfg), C.byref(self.handle), _stream(stream)),
                "qed_init_tables")
        self.dtype = torch.float64 if cfg.precision == B.QED_FP64 else torch.float32

    def close(self):
        if self.handle:
            B.lib().qed_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return B.lib().qed_launch_count(self.handle)


def qed_init_tables(cfg: B.qed_config | None = None, stream=None) -> Context:
    return Context(cfg if cfg is not None else config(), stream)


def qed_destroy(ctx: Context) -> None:
    ctx.close()


@dataclass
class Species:
    """Structure-of-arrays particle buffers (torch device tensors)."""
    x: torch.Tensor
    y: torch.Tensor
    z: torch.Tensor
    px: torch.Tensor
    py: torch.Tensor
    pz: torch.Tensor
    w: torch.Tensor
    id: torch.Tensor          # int64 storage of the uint64 ids
    n: torch.Tensor           # int64[1] device count
    q: int
    alive: torch.Tensor | None = None
    ex: torch.Tensor | None = None
    ey: torch.Tensor | None = None
    ez: torch.Tensor | None = None
    bx: torch.Tensor | None = None
    by: torch.Tensor | None = None
    bz: torch.Tensor | None = None
    tag: torch.Tensor | None = None   # int32 storage of the uint32 tags
    od_p: torch.Tensor | None = None  # event generators II/III: cumulative probability
    od_r: torch.Tensor | None = None  # ... and its random number r3 (0 = not drawn yet)

    @property
    def capacity(self) -> int:
        return int(self.x.numel())

    @staticmethod
    def empty(capacity: int, q: int, dtype=torch.float32, device="cuda", fields=False,
              alive=None, tag=False, od=False, pinned=False) -> "Species":
        """Zeroed buffers on `device`; pinned=True: page-locked host memory
        (device "cpu"), for qed_lepton_step_host."""
        cap = max(int(capacity), 0)
        if pinned:
            device = "cpu"
        z = lambda n, dt: torch.zeros(n, dtype=dt, device=device, pin_memory=pinned)
        mk = lambda: z(cap, dtype)
        kw = {k: mk() for k in STATE}
        if fields:
            kw.update({k: mk() for k in FIELD_NAMES})
        if alive is None:
            alive = q == 0
        return Species(id=z(cap, torch.int64), n=z(1, torch.int64), q=q,
                       alive=z(cap, torch.uint8) if alive else None,
                       tag=z(cap, torch.int32) if tag else None,
                       od_p=mk() if od else None, od_r=mk() if od else None,
                       **kw)

    def load(self, **arrays) -> "Species":
        """Copy host/device arrays into the first n slots and set n."""
        n = None
        for k, v in arrays.items():
            t = torch.as_tensor(np.ascontiguousarray(v)) if isinstance(v, np.ndarray) else v
            if k == "id":
                t = t.to(torch.int64) if t.dtype != torch.uint64 else t.view(torch.int64)
            if k == "tag":
                t = t.to(torch.int32)
            n = t.numel() if n is None else n
            getattr(self, k)[:n].copy_(t.reshape(-1))
        if self.alive is not None and "alive" not in arrays and n:
            self.alive[:n] = 1
        self.n.fill_(n or 0)
        return self

    def count(self) -> int:
        return int(self.n.item())

    def host(self, names=None) -> dict:
        n = self.count()
        names = names or [k for k in STATE + ("id", "alive", "tag", "od_p", "od_r") + FIELD_NAMES
                          if getattr(self, k) is not None]
        out = {}
        for k in names:
            t = getattr(self, k)
            if t is None:
                continue
            a = t[:n].cpu().numpy()
            out[k] = a.view(np.uint64) if k == "id" else (a.view(np.uint32) if k == "tag" else a)
        return out

    def struct(self) -> B.qed_species:
        s = B.qed_species()
        for k in STATE + FIELD_NAMES + ("id", "alive", "tag", "od_p", "od_r"):
            t = getattr(self, k)
            setattr(s, k, t.data_ptr() if t is not None and t.numel() else None)
        s.d_n = self.n.data_ptr()
        s.capacity = self.capacity
        s.q = self.q
        return s


class Fields:
    @staticmethod
    def uniform(E, Bf) -> B.qed_fields:
        f = B.qed_fields()
        f.mode = B.QED_FIELDS_UNIFORM
        for c in range(3):
            f.e[c] = float(E[c])
            f.b[c] = float(Bf[c])
        return f

    @staticmethod
    def per_particle() -> B.qed_fields:
        f = B.qed_fields()
        f.mode = B.QED_FIELDS_PER_PARTICLE
        return f

    @staticmethod
    def grid(grid: torch.Tensor, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0) -> B.qed_fields:
        assert grid.dtype == torch.float32 and grid.is_contiguous() and grid.shape[-1] == 8
        nz, ny, nx = grid.shape[:3]
        f = B.qed_fields()
        f.mode = B.QED_FIELDS_GRID
        f.nx, f.ny, f.nz = nx, ny, nz
        f.grid = grid.data_ptr()
        f.dx, f.dy, f.dz, f.x0, f.y0, f.z0 = dx, dy, dz, x0, y0, z0
        f._keep = grid
        return f


YEE_ARRAYS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")


class Yee:
    """Fields of the PIC loop on a periodic Yee grid (include/qed.h,
    qed_yee): nine float arrays [nz, ny, nx] at their staggered positions
    and the node grid [nz, ny, nx, 8] the particle gather reads."""

    def __init__(self, nx, ny, nz, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0, device="cuda"):
        self.shape = (int(nz), int(ny), int(nx))
        self.dx, self.dy, self.dz = float(dx), float(dy), float(dz)
        self.x0, self.y0, self.z0 = float(x0), float(y0), float(z0)
        for nm in YEE_ARRAYS:
            setattr(self, nm, torch.zeros(self.shape, dtype=torch.float32, device=device))
        self.nodes = torch.zeros(self.shape + (8,), dtype=torch.float32, device=device)

    def struct(self) -> B.qed_yee:
        y = B.qed_yee()
        y.nz, y.ny, y.nx = self.shape
        y.dx, y.dy, y.dz, y.x0, y.y0, y.z0 = self.dx, self.dy, self.dz, self.x0, self.y0, self.z0
        for nm in YEE_ARRAYS + ("nodes",):
            setattr(y, nm, getattr(self, nm).data_ptr())
        return y

    def fields(self) -> B.qed_fields:
        """The node grid as qed_fields (mode GRID)."""
        return Fields.grid(self.nodes, self.dx, self.dy, self.dz, self.x0, self.y0, self.z0)


def qed_pic_deposit(ctx: Context, s: Species, y: Yee, weight_unit: float = 1.0,
                    d_count: torch.Tensor | None = None, stream=None) -> None:
    B.check(B.lib().qed_pic_deposit(ctx.handle, C.byref(s.struct()), C.byref(y.struct()),
                                    float(weight_unit), d_count.data_ptr() if d_count is not None else None,
                                    _stream(stream)), "qed_pic_deposit")


def qed_pic_fields(ctx: Context, y: Yee, advance: bool = True, stream=None) -> None:
    B.check(B.lib().qed_pic_fields(ctx.handle, C.byref(y.struct()), int(bool(advance)), _stream(stream)),
            "qed_pic_fields")


def qed_pic_step(ctx: Context, e: Species | None, p: Species | None, g: Species, y: Yee,
                 weight_unit: float, step: int, stream=None) -> None:
    B.check(B.lib().qed_pic_step(ctx.handle, C.byref(_sp(e)), C.byref(_sp(p)), C.byref(g.struct()),
                                 C.byref(y.struct()), float(weight_unit), int(step), _stream(stream)),
            "qed_pic_step")


def _sp(s: Species | None) -> B.qed_species:
    if s is None:  # an empty species with a zero count
        z = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = B.qed_species()
        st.d_n = z.data_ptr()
        st.capacity = 0
        st._keep = z
        return st
    return s.struct()


def qed_gather_push(ctx: Context, s: Species, f, step: int, stream=None) -> None:
    B.check(B.lib().qed_gather_push(ctx.handle, C.byref(s.struct()), C.byref(f), int(step),
                                    _stream(stream)), "qed_gather_push")


def qed_emit(ctx: Context, lepton: Species, photons: Species, f, step: int, stream=None) -> None:
    B.check(B.lib().qed_emit(ctx.handle, C.byref(lepton.struct()), C.byref(photons.struct()),
                             C.byref(f), int(step), _stream(stream)), "qed_emit")


def qed_pair(ctx: Context, photons: Species, electrons: Species, positrons: Species, f, step: int,
             stream=None) -> None:
    B.check(B.lib().qed_pair(ctx.handle, C.byref(photons.struct()), C.byref(electrons.struct()),
                             C.byref(positrons.struct()), C.byref(f), int(step), _stream(stream)),
            "qed_pair")


def qed_compact(ctx: Context, s: Species, stream=None) -> None:
    B.check(B.lib().qed_compact(ctx.handle, C.byref(s.struct()), _stream(stream)), "qed_compact")


def qed_count_alive(ctx: Context, s: Species, out=None, stream=None):
    """Live particles of s, written on the device into `out` (an int64 CUDA
    tensor element, e.g. counts[k, 1]; a new one-element tensor if None)."""
    if out is None:
        out = torch.zeros(1, dtype=torch.int64, device=s.x.device)
    assert out.dtype == torch.int64 and out.is_cuda
    B.check(B.lib().qed_count_alive(ctx.handle, C.byref(s.struct()), C.c_void_p(out.data_ptr()),
                                    _stream(stream)), "qed_count_alive")
    return out


def qed_compact_fill(ctx: Context, s: Species, stream=None) -> None:
    B.check(B.lib().qed_compact_fill(ctx.handle, C.byref(s.struct()), _stream(stream)),
            "qed_compact_fill")


def qed_step_fused(ctx: Context, e: Species | None, p: Species | None, g: Species, f, step: int,
                   stream=None) -> None:
    se, sp_, sg = _sp(e), _sp(p), _sp(g)
    B.check(B.lib().qed_step_fused(ctx.handle, C.byref(se), C.byref(sp_), C.byref(sg), C.byref(f),
                                   int(step), _stream(stream)), "qed_step_fused")


def qed_lepton_step_host(ctx: Context, l_host: Species, g: Species, g_host: Species | None, fields,
                         step: int, chunk: int, stream=None) -> None:
    """The lepton stage of a step for leptons in (pinned) host memory,
    streamed through the GPU in chunks; g_host (optional) receives the new
    photons.  Synchronous."""
    gh = C.byref(g_host.struct()) if g_host is not None else None
    B.check(B.lib().qed_lepton_step_host(ctx.handle, C.byref(l_host.struct()), C.byref(g.struct()), gh,
                                         C.byref(fields), int(step), int(chunk), _stream(stream)),
            "qed_lepton_step_host")


def qed_sample_xi(ctx: Context, chi: torch.Tensor, gamma: torch.Tensor, xi: torch.Tensor, step: int,
                  stream=None) -> None:
    n = chi.numel()
    B.check(B.lib().qed_sample_xi(ctx.handle, chi.data_ptr(), gamma.data_ptr(), xi.data_ptr(), n,
                                  int(step), _stream(stream)), "qed_sample_xi")


def qed_rates(ctx: Context, which: int, chi: torch.Tensor, gamma: torch.Tensor,
              stream=None) -> torch.Tensor:
    chi = chi.to(torch.float64).contiguous()
    gamma = gamma.to(torch.float64).contiguous()
    out = torch.empty_like(chi)
    B.check(B.lib().qed_rates(ctx.handle, int(which), chi.data_ptr(), gamma.data_ptr(),
                              out.data_ptr(), chi.numel(), _stream(stream)), "qed_rates")
    return out


def qed_sample_table(ctx: Context, which: int, chi: torch.Tensor, gamma: torch.Tensor | None,
                     word: torch.Tensor, stream=None) -> torch.Tensor:
    chi = chi.to(torch.float64).contiguous()
    g = gamma.to(torch.float64).contiguous() if gamma is not None else chi
    word = word.to(torch.int32).contiguous()
    out = torch.empty_like(chi)
    B.check(B.lib().qed_sample_table(ctx.handle, int(which), chi.data_ptr(), g.data_ptr(),
                                     word.data_ptr(), out.data_ptr(), chi.numel(), _stream(stream)),
            "qed_sample_table")
    return out


def qed_chi(ctx: Context, s: Species, stream=None) -> torch.Tensor:
    """chi_e (leptons) or chi_ph (photons, q = 0) of every particle of s, from
    its momentum and per-particle fields (device float64 tensor)."""
    out = torch.zeros(max(s.capacity, 1), dtype=torch.float64, device=s.x.device)
    B.check(B.lib().qed_chi(ctx.handle, C.byref(s.struct()), out.data_ptr(), _stream(stream)),
            "qed_chi")
    return out[:s.count()]


def qed_fill_standing_wave(ctx: Context, grid: torch.Tensor, x0: float, dx: float, a0: float,
                           t: float, stream=None) -> None:
    nz, ny, nx = grid.shape[:3]
    B.check(B.lib().qed_fill_standing_wave(ctx.handle, grid.data_ptr(), nx, ny, nz, float(x0),
                                           float(dx), float(a0), float(t), _stream(stream)),
            "qed_fill_standing_wave")


def qed_table_get(ctx: Context, which: int):
    """Returns (table as 2-D float64 array, grid info dict)."""
    dims = (C.c_double * 6)()
    B.check(B.lib().qed_table_get(ctx.handle, int(which), None, 0, dims), "qed_table_get")
    n0, n1 = int(dims[0]), int(dims[1])
    out = np.zeros(n0 * n1, dtype=np.float64)
    B.check(B.lib().qed_table_get(ctx.handle, int(which), out.ctypes.data, out.size, dims),
            "qed_table_get")
    return out.reshape(n0, n1), {"n0": n0, "n1": n1, "x0_0": dims[2], "h_0": dims[3],
                                 "x0_1": dims[4], "h_1": dims[5]}


def qed_read_counters(ctx: Context, stream=None) -> dict:
    c = B.qed_counters()
    code = B.lib().qed_read_counters(ctx.handle, C.byref(c), _stream(stream))
    if code not in (B.QED_OK, -5):
        B.check(code, "qed_read_counters")
    return c.as_dict()


def qed_reset_counters(ctx: Context, stream=None) -> None:
    B.check(B.lib().qed_reset_counters(ctx.handle, _stream(stream)), "qed_reset_counters")


def qed_last_device_status(ctx: Context) -> tuple[int, int]:
    """(status bits, dropped appends) since the last reset; waits for the device.
    A set QED_STATUS_TIMEOUT bit is returned, not raised."""
    bits, dropped = C.c_uint32(0), C.c_int64(0)
    code = B.lib().qed_last_device_status(ctx.handle, C.byref(bits), C.byref(dropped))
    if code not in (B.QED_OK, -5):
        B.check(code, "qed_last_device_status")
    return int(bits.value), int(dropped.value)


def qed_test_wait_expiry(ctx: Context, stream=None) -> None:
    """Launch the bounded-wait expiry check (sets QED_STATUS_TIMEOUT on the device)."""
    B.check(B.lib().qed_test_wait_expiry(ctx.handle, _stream(stream)), "qed_test_wait_expiry")


def qed_profile_begin(ctx: Context, max_steps: int) -> None:
    B.check(B.lib().qed_profile_begin(ctx.handle, int(max_steps)), "qed_profile_begin")


def qed_profile_end(ctx: Context) -> tuple[float, float, int]:
    """(lepton kernel ms, photon kernel ms, steps recorded)."""
    a, b, n = C.c_double(), C.c_double(), C.c_int64()
    B.check(B.lib().qed_profile_end(ctx.handle, C.byref(a), C.byref(b), C.byref(n)), "qed_profile_end")
    return a.value, b.value, n.value


PROF_PHASES = ("lepton_stream", "lepton_class_list", "lepton_count", "photon_count_scan",
               "lepton_write", "photon_stream", "photon_ordered")


def qed_profile_end_phases(ctx: Context) -> tuple[dict, int]:
    """({phase name: summed ms}, steps recorded)."""
    ms = (C.c_double * B.QED_PROF_PHASES)()
    n = C.c_int64()
    B.check(B.lib().qed_profile_end_phases(ctx.handle, ms, C.byref(n)), "qed_profile_end_phases")
    return dict(zip(PROF_PHASES, list(ms))), n.value


def qed_mlp_load(ctx: Context, weights) -> None:
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
    B.check(B.lib().qed_mlp_load(ctx.handle, w.ctypes.data, w.size), "qed_mlp_load")


def qed_mlp_get(ctx: Context) -> np.ndarray:
    w = np.zeros(B.MLP_NP, dtype=np.float32)
    B.check(B.lib().qed_mlp_get(ctx.handle, w.ctypes.data, w.size), "qed_mlp_get")
    return w


def qed_mlp_train(ctx: Context, n_samples: int, lr: float = 3e-3, seed: int = 1, stream=None) -> float:
    loss = C.c_double()
    B.check(B.lib().qed_mlp_train(ctx.handle, int(n_samples), float(lr), int(seed), C.byref(loss),
                                  _stream(stream)), "qed_mlp_train")
    return loss.value


def qed_mlp_grad(ctx: Context, x: torch.Tensor, t: torch.Tensor, stream=None):
    x = x.to(torch.float32).contiguous()
    t = t.to(torch.float32).contiguous()
    g = torch.zeros(B.MLP_NP, dtype=torch.float32, device=x.device)
    loss = C.c_double()
    B.check(B.lib().qed_mlp_grad(ctx.handle, x.data_ptr(), t.data_ptr(), t.numel(), g.data_ptr(),
                                 C.byref(loss), _stream(stream)), "qed_mlp_grad")
    return g, loss.value


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Initial weights of the learned inverse CDF: uniform(+-sqrt(6/(fan_in +
    fan_out))) weights, zero biases, in the C ABI's parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out, is_w in ((2, 64, 1), (0, 64, 0), (64, 64, 1), (0, 64, 0), (64, 64, 1),
                                  (0, 64, 0), (64, 1, 1), (0, 1, 0)):
        if is_w:
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        else:
            parts.append(np.zeros(fan_out))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == B.MLP_NP
    return w


def qed_run_batched(ctx: Context, e: Species, p: Species, g: Species, f, step0: int, steps: int,
                    n_runs: int = 0, stream=None) -> torch.Tensor | None:
    """Advance the concatenated runs by `steps` fused steps as one CUDA graph.
    Returns the alive photons per run (device int64[n_runs]) when n_runs > 0."""
    out = torch.zeros(max(n_runs, 1), dtype=torch.int64, device="cuda") if n_runs else None
    B.check(B.lib().qed_run_batched(ctx.handle, C.byref(e.struct()), C.byref(p.struct()),
                                    C.byref(g.struct()), C.byref(f), int(step0), int(steps),
                                    int(n_runs), out.data_ptr() if out is not None else None,
                                    _stream(stream)), "qed_run_batched")
    return out


def qed_autotune(ctx: Context, e: Species, p: Species, g: Species, f, reps: int = 3,
                 stream=None) -> tuple[int, list]:
    best = C.c_int()
    ms = (C.c_double * 8)()
    B.check(B.lib().qed_autotune(ctx.handle, C.byref(e.struct()), C.byref(p.struct()),
                                 C.byref(g.struct()), C.byref(f), int(reps), C.byref(best), ms,
                                 _stream(stream)), "qed_autotune")
    return best.value, [ms[i] for i in range(8)]


def qed_autotune_groups(ctx: Context, e: Species, p: Species, g: Species, f, reps: int = 2,
                        stream=None) -> dict:
    """Tune the CTAs per SM of each kernel group, then the Method I chain
    scheduling, on disposable species (they are advanced).  Returns
    {"grid_factor": {group: factor}, "sched": {parameter: value},
    "ms_per_step": .., "ms": {group: [ms per factor 1..8]},
    "sched_ms": {parameter: {value: ms}}}; the values stay in the context."""
    t = B.qed_tuning()
    B.check(B.lib().qed_autotune_groups(ctx.handle, C.byref(e.struct()), C.byref(p.struct()),
                                        C.byref(g.struct()), C.byref(f), int(reps), C.byref(t),
                                        _stream(stream)), "qed_autotune_groups")
    return {"grid_factor": {n: int(t.grid_factor[k]) for k, n in enumerate(B.TUNE_GROUP_NAMES)},
            "sched": {n: int(t.sched[k]) for k, n in enumerate(B.SCHED_NAMES)},
            "ms_per_step": t.ms_per_step,
            "ms": {n: [float(t.ms[k][j]) for j in range(B.QED_TUNE_MAX_FACTOR)]
                   for k, n in enumerate(B.TUNE_GROUP_NAMES)},
            "sched_ms": {n: {int(t.sched_tried[k][j]): float(t.sched_ms[k][j])
                             for j in range(B.QED_SCHED_MAX_CANDIDATES) if t.sched_tried[k][j]}
                         for k, n in enumerate(B.SCHED_NAMES)}}


def qed_set_tuning(ctx: Context, grid_factor: dict, sched: dict | None = None) -> None:
    """Set the CTAs per SM of kernel groups ({group: factor}) and the chain
    scheduling ({parameter: value}); absent entries and 0 mean the default."""
    t = B.qed_tuning()
    for k, n in enumerate(B.TUNE_GROUP_NAMES):
        t.grid_factor[k] = int(grid_factor.get(n, 0))
    for k, n in enumerate(B.SCHED_NAMES):
        t.sched[k] = int((sched or {}).get(n, 0))
    B.check(B.lib().qed_set_tuning(ctx.handle, C.byref(t)), "qed_set_tuning")
