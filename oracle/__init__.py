"""FP64 CPU oracle for the QED Monte Carlo step (arXiv:1608.06356).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code allowed to import this package.
It shares no code with the CUDA path (``paper_1608_06356_gb300``); the two
meet only through the seeded input generators, which hold none of the
method's arithmetic.

The numerics live in ``qed_oracle.c`` (plain C, FP64): Bessel functions and
their integrals by adaptive Gauss-Kronrod quadrature of the integral
representations, the spectra of Eqs. (1), (4), (5) and (6), rates by
quadrature, the inverse CDF of Eq. (7) by safeguarded Newton iteration,
chi from Eqs. (2)/(3), Philox4x32-10, a Boris push, CIC gather, and Method I
with the adaptive sub-step rule.  This module only builds the library with
gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

# Physical constants of the reading used on both sides (see the C header).
A_S_1UM = 412148.45          # m_e c^2 / (hbar omega0) at lambda = 1 um
ALPHA = 1.0 / 137.035999     # CODATA fine-structure constant

FIELDS_UNIFORM, FIELDS_PER_PARTICLE, FIELDS_GRID = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile qed_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Config(C.Structure):
    _fields_ = [("a_S", C.c_double), ("alpha", C.c_double), ("dt", C.c_double),
                ("wdt_max", C.c_double), ("xi_min_energy", C.c_double),
                ("pair_sign", C.c_int), ("generator", C.c_int), ("seed", C.c_uint64),
                ("spec_lo", C.c_double), ("spec_hi", C.c_double), ("model", C.c_int),
                ("pad_", C.c_int)]


GEN_METHOD_I, GEN_METHOD_II, GEN_METHOD_III = 0, 1, 2


MODEL_FORMULA_I, MODEL_CLASSIC = 0, 1


def make_config(dt=0.01, a_S=A_S_1UM, alpha=ALPHA, wdt_max=0.2, xi_min_energy=2.0,
                pair_sign=1, seed=0, spec_lo=2.0, spec_hi=1000.0, generator=GEN_METHOD_I,
                model=MODEL_FORMULA_I) -> Config:
    """generator: photon event generator, Method I (default), II or III.
    model: photon spectrum, formula I (Eq. 1, default) or the classic limit
    (Eq. 5) restricted to 0 < xi < 1."""
    return Config(a_S, alpha, dt, wdt_max, xi_min_energy, pair_sign, generator, seed, spec_lo,
                  spec_hi, model, 0)


class Fields(C.Structure):
    _fields_ = [("mode", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("e", C.c_double * 3), ("b", C.c_double * 3),
                ("grid", C.POINTER(C.c_float)),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double)]


_PD = C.POINTER(C.c_double)


class _Species(C.Structure):
    _fields_ = [("x", _PD), ("y", _PD), ("z", _PD), ("px", _PD), ("py", _PD), ("pz", _PD),
                ("w", _PD), ("id", C.POINTER(C.c_uint64)), ("alive", C.POINTER(C.c_uint8)),
                ("ex", _PD), ("ey", _PD), ("ez", _PD), ("bx", _PD), ("by", _PD), ("bz", _PD),
                ("n", C.c_int64), ("capacity", C.c_int64), ("q", C.c_double),
                ("tag", C.POINTER(C.c_uint32)), ("od_p", _PD), ("od_r", _PD)]


class Counters(C.Structure):
    _fields_ = [("events", C.c_int64), ("substeps", C.c_int64), ("dropped", C.c_int64),
                ("hist", C.c_int64 * 64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i64, P = C.c_double, C.c_int64, C.POINTER
        sig = {
            "orc_besselk": (d, [d, d]),
            "orc_besselk_int": (d, [d, d]),
            "orc_spec_I": (d, [d, d]),
            "orc_spec_II": (d, [d, d]),
            "orc_spec_classic": (d, [d, d]),
            "orc_spec_pair": (d, [d, d, C.c_int]),
            "orc_J": (d, [C.c_int, d]),
            "orc_cum_photon": (d, [d, d, d]),
            "orc_cum_photon_m": (d, [d, d, d, C.c_int]),
            "orc_cum_pair": (d, [d, d, d, C.c_int]),
            "orc_rate_photon": (d, [P(Config), d, d]),
            "orc_rate_pair": (d, [P(Config), d, d]),
            "orc_sample_photon": (d, [P(Config), d, d, d, d]),
            "orc_sample_pair": (d, [P(Config), d, d, d]),
            "orc_chi_lepton": (d, [_PD, _PD, _PD, d]),
            "orc_chi_photon": (d, [_PD, _PD, _PD, d]),
            "orc_boris": (d, [_PD, _PD, _PD, d, d]),
            "orc_cic_gather": (None, [P(Fields), d, d, d, _PD, _PD]),
            "orc_fill_standing_wave": (None, [P(C.c_float), C.c_int, C.c_int, C.c_int, d, d, d, d]),
            "orc_gk15_monomial": (None, [C.c_int, d, d, _PD, _PD]),
            "orc_philox4x32_10": (None, [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]),
            "orc_philox_v": (None, [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32), i64]),
            "orc_step": (None, [P(Config), P(Fields), P(_Species), P(_Species), P(_Species), i64,
                                P(Counters), P(Counters)]),
            "orc_emit_pass": (None, [P(Config), P(Fields), P(_Species), P(_Species), i64,
                                     P(Counters)]),
            "orc_compact": (i64, [P(_Species)]),
            "orc_num_threads": (C.c_int, []),
            "orc_set_num_threads": (None, [C.c_int]),
            "orc_rate_photon_v": (None, [P(Config), _PD, _PD, _PD, i64]),
            "orc_rate_pair_v": (None, [P(Config), _PD, _PD, _PD, i64]),
            "orc_sample_photon_v": (None, [P(Config), _PD, _PD, _PD, _PD, _PD, i64]),
            "orc_sample_pair_v": (None, [P(Config), _PD, _PD, _PD, _PD, i64]),
            "orc_cum_photon_v": (None, [_PD, _PD, _PD, _PD, i64]),
            "orc_cum_pair_v": (None, [_PD, _PD, _PD, C.c_int, _PD, i64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- scalar math
def besselk(nu, x):
    return lib().orc_besselk(float(nu), float(x))


def besselk_int(nu, x):
    return lib().orc_besselk_int(float(nu), float(x))


def spec_I(xi, chi):
    return lib().orc_spec_I(float(xi), float(chi))


def spec_II(xi, chi):
    return lib().orc_spec_II(float(xi), float(chi))


def spec_classic(xi, chi):
    return lib().orc_spec_classic(float(xi), float(chi))


def spec_pair(xi, chi, sign=1):
    return lib().orc_spec_pair(float(xi), float(chi), int(sign))


def cum_photon(a, b, chi, model=MODEL_FORMULA_I):
    return lib().orc_cum_photon_m(float(a), float(b), float(chi), int(model))


def cum_pair(a, b, chi, sign=1):
    return lib().orc_cum_pair(float(a), float(b), float(chi), int(sign))


def gk15_monomial(k, a=-1.0, b=1.0):
    kr, g = C.c_double(), C.c_double()
    lib().orc_gk15_monomial(int(k), float(a), float(b), C.byref(kr), C.byref(g))
    return kr.value, g.value


def chi_lepton(p, E, B, a_S=A_S_1UM):
    p, E, B = _f64(p), _f64(E), _f64(B)
    return lib().orc_chi_lepton(_dp(p), _dp(E), _dp(B), float(a_S))


def chi_photon(p, E, B, a_S=A_S_1UM):
    p, E, B = _f64(p), _f64(E), _f64(B)
    return lib().orc_chi_photon(_dp(p), _dp(E), _dp(B), float(a_S))


def boris(p, E, B, q, dt):
    """Returns (new p, new gamma)."""
    p = _f64(p).copy()
    E, B = _f64(E), _f64(B)
    g = lib().orc_boris(_dp(p), _dp(E), _dp(B), float(q), float(dt))
    return p, g


def cic_gather(fields: Fields, x, y, z):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().orc_cic_gather(C.byref(fields), float(x), float(y), float(z), _dp(E), _dp(B))
    return E, B


def fill_standing_wave(nx, ny, nz, x0, dx, a0, t) -> np.ndarray:
    g = np.zeros((nz, ny, nx, 8), dtype=np.float32)
    lib().orc_fill_standing_wave(g.ctypes.data_as(C.POINTER(C.c_float)), nx, ny, nz,
                                 float(x0), float(dx), float(a0), float(t))
    return g


def grid_fields(grid: np.ndarray, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0) -> Fields:
    assert grid.dtype == np.float32 and grid.flags.c_contiguous and grid.shape[-1] == 8
    nz, ny, nx = grid.shape[:3]
    f = Fields()
    f.mode, f.nx, f.ny, f.nz = FIELDS_GRID, nx, ny, nz
    f.grid = grid.ctypes.data_as(C.POINTER(C.c_float))
    f.dx, f.dy, f.dz, f.x0, f.y0, f.z0 = dx, dy, dz, x0, y0, z0
    f._keep = grid
    return f


def uniform_fields(E, B) -> Fields:
    f = Fields()
    f.mode = FIELDS_UNIFORM
    for c in range(3):
        f.e[c] = float(E[c])
        f.b[c] = float(B[c])
    return f


def per_particle_fields() -> Fields:
    f = Fields()
    f.mode = FIELDS_PER_PARTICLE
    return f


def philox(ctr, key):
    """Philox4x32-10 of arrays ctr (n,4) uint32 and key (n,2) uint32."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(ctr)
    P = C.POINTER(C.c_uint32)
    lib().orc_philox_v(ctr.ctypes.data_as(P), key.ctypes.data_as(P), out.ctypes.data_as(P),
                       ctr.shape[0])
    return out


# -------------------------------------------------------------- vector forms
def rate_photon(cfg: Config, chi, gamma):
    chi, gamma = np.broadcast_arrays(_f64(chi), _f64(gamma))
    chi, gamma = _f64(chi.ravel()), _f64(gamma.ravel())
    out = np.zeros_like(chi)
    lib().orc_rate_photon_v(C.byref(cfg), _dp(chi), _dp(gamma), _dp(out), chi.size)
    return out


def rate_pair(cfg: Config, chi, gamma):
    chi, gamma = np.broadcast_arrays(_f64(chi), _f64(gamma))
    chi, gamma = _f64(chi.ravel()), _f64(gamma.ravel())
    out = np.zeros_like(chi)
    lib().orc_rate_pair_v(C.byref(cfg), _dp(chi), _dp(gamma), _dp(out), chi.size)
    return out


def sample_photon(cfg: Config, chi, gamma, r2, c2):
    arrs = [_f64(a.ravel()) for a in np.broadcast_arrays(_f64(chi), _f64(gamma), _f64(r2), _f64(c2))]
    out = np.zeros_like(arrs[0])
    lib().orc_sample_photon_v(C.byref(cfg), *[_dp(a) for a in arrs], _dp(out), out.size)
    return out


def sample_pair(cfg: Config, chi, r2, c2):
    arrs = [_f64(a.ravel()) for a in np.broadcast_arrays(_f64(chi), _f64(r2), _f64(c2))]
    out = np.zeros_like(arrs[0])
    lib().orc_sample_pair_v(C.byref(cfg), *[_dp(a) for a in arrs], _dp(out), out.size)
    return out


def cum_photon_v(a, b, chi):
    arrs = [_f64(x.ravel()) for x in np.broadcast_arrays(_f64(a), _f64(b), _f64(chi))]
    out = np.zeros_like(arrs[0])
    lib().orc_cum_photon_v(*[_dp(x) for x in arrs], _dp(out), out.size)
    return out


def cum_pair_v(a, b, chi, sign=1):
    arrs = [_f64(x.ravel()) for x in np.broadcast_arrays(_f64(a), _f64(b), _f64(chi))]
    out = np.zeros_like(arrs[0])
    lib().orc_cum_pair_v(*[_dp(x) for x in arrs], int(sign), _dp(out), out.size)
    return out


def uniform_from_word(w):
    """u = (w + 1/2) 2^-32 and its complement, exactly as the oracle draws them."""
    w = np.asarray(w, dtype=np.uint64)
    return (w.astype(np.float64) + 0.5) * 2.0 ** -32, ((0xFFFFFFFF - w).astype(np.float64) + 0.5) * 2.0 ** -32


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


# ------------------------------------------------------------------ species
_FIELD_NAMES = ("ex", "ey", "ez", "bx", "by", "bz")
_STATE_NAMES = ("x", "y", "z", "px", "py", "pz", "w")


class Species:
    """FP64 SoA particle buffers owned by numpy, with capacity for appends."""

    def __init__(self, capacity: int, q: float, per_particle_fields: bool = False,
                 with_alive: bool = False, with_tag: bool = False, with_od: bool = False):
        self.capacity = int(capacity)
        self.q = float(q)
        cap = max(self.capacity, 1)
        for nm in _STATE_NAMES:
            setattr(self, nm, np.zeros(cap))
        self.id = np.zeros(cap, dtype=np.uint64)
        self.alive = np.ones(cap, dtype=np.uint8) if with_alive else None
        self.has_fields = per_particle_fields
        for nm in _FIELD_NAMES:
            setattr(self, nm, np.zeros(cap) if per_particle_fields else None)
        self.tag = np.zeros(cap, dtype=np.uint32) if with_tag else None
        # Methods II/III state: cumulative probability and r3 (0 = not drawn yet)
        self.od_p = np.zeros(cap) if with_od else None
        self.od_r = np.zeros(cap) if with_od else None
        self.n = 0

    def load(self, **arrays):
        n = None
        for k, v in arrays.items():
            v = np.asarray(v)
            n = len(v) if n is None else n
            assert len(v) == n
            getattr(self, k)[:n] = v
        if self.alive is not None and "alive" not in arrays:
            self.alive[:n] = 1
        self.n = n
        return self

    def view(self, name):
        a = getattr(self, name)
        return None if a is None else a[: self.n]

    def _struct(self) -> _Species:
        s = _Species()
        for nm in _STATE_NAMES:
            setattr(s, nm, _dp(getattr(self, nm)))
        s.id = self.id.ctypes.data_as(C.POINTER(C.c_uint64))
        s.alive = (self.alive.ctypes.data_as(C.POINTER(C.c_uint8)) if self.alive is not None
                   else C.POINTER(C.c_uint8)())
        for nm in _FIELD_NAMES:
            a = getattr(self, nm)
            setattr(s, nm, _dp(a) if a is not None else _PD())
        s.n, s.capacity, s.q = self.n, self.capacity, self.q
        s.tag = (self.tag.ctypes.data_as(C.POINTER(C.c_uint32)) if self.tag is not None
                 else C.POINTER(C.c_uint32)())
        s.od_p = _dp(self.od_p) if self.od_p is not None else _PD()
        s.od_r = _dp(self.od_r) if self.od_r is not None else _PD()
        return s


def step(cfg: Config, fields: Fields, electrons: Species | None, positrons: Species | None,
         photons: Species | None, step_index: int):
    """One QED step (electrons, positrons, then photons alive at step start).

    Returns (lepton counters, pair counters)."""
    structs = [sp._struct() if sp is not None else None for sp in (electrons, positrons, photons)]
    ptrs = [C.byref(s) if s is not None else C.POINTER(_Species)() for s in structs]
    lc, pc = Counters(), Counters()
    lib().orc_step(C.byref(cfg), C.byref(fields), *ptrs, int(step_index), C.byref(lc), C.byref(pc))
    for sp, s in zip((electrons, positrons, photons), structs):
        if sp is not None:
            sp.n = s.n
    return lc, pc


def emit(cfg: Config, fields: Fields, leptons: Species, photons: Species, step_index: int):
    """Photon emission of every lepton at its current momentum and fields, no
    push (the counterpart of the library's qed_emit).  Returns the counters."""
    sl, sg = leptons._struct(), photons._struct()
    c = Counters()
    lib().orc_emit_pass(C.byref(cfg), C.byref(fields), C.byref(sl), C.byref(sg), int(step_index),
                        C.byref(c))
    leptons.n, photons.n = sl.n, sg.n
    return c


def compact(sp: Species) -> int:
    s = sp._struct()
    n = lib().orc_compact(C.byref(s))
    sp.n = n
    return n
