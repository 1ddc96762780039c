"""ctypes binding of libqed (include/qed.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
builds the C structs from torch tensors (device memory, owned by the caller)
and forwards the calls.  It raises if the library is missing -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqed.so")

QED_OK = 0
QED_FP32, QED_FP64 = 0, 1
QED_SAMPLER_TABLE, QED_SAMPLER_MLP = 0, 1
MLP_NP = 8577
QED_FIELDS_UNIFORM, QED_FIELDS_PER_PARTICLE, QED_FIELDS_GRID = 0, 1, 2
QED_STATUS_CAPACITY, QED_STATUS_DOMAIN, QED_STATUS_NONFINITE = 1, 2, 4
QED_STATUS_TIMEOUT, QED_STATUS_SUBSTEPS, QED_STATUS_REPLAY = 8, 16, 32
QED_PROF_PHASES = 7
QED_GEN_METHOD_I, QED_GEN_METHOD_II, QED_GEN_METHOD_III = 0, 1, 2
QED_MODEL_FORMULA_I, QED_MODEL_CLASSIC = 0, 1
QED_APPEND_ORDERED, QED_APPEND_ANY = 0, 1

ERRORS = {-1: "QED_ERR_ARG", -2: "QED_ERR_CUDA", -3: "QED_ERR_CAPACITY", -4: "QED_ERR_DOMAIN",
          -5: "QED_ERR_TIMEOUT", -6: "QED_ERR_NOCONV", -7: "QED_ERR_NOMEM", -8: "QED_ERR_UNSUPPORTED"}


class QedError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed: {ERRORS.get(code, code)}")
        self.code = code


class qed_config(C.Structure):
    _fields_ = [("a_S", C.c_double), ("alpha", C.c_double), ("dt", C.c_double),
                ("wdt_max", C.c_double), ("xi_min_energy", C.c_double),
                ("pair_sign", C.c_int), ("precision", C.c_int),
                ("chi_min", C.c_double), ("chi_max", C.c_double),
                ("chi_pair_min", C.c_double), ("chi_pair_max", C.c_double),
                ("fwd_per_unit", C.c_double), ("inv_per_unit", C.c_double),
                ("seed", C.c_uint64), ("spec_lo", C.c_double), ("spec_hi", C.c_double),
                ("max_particles", C.c_int64), ("max_substeps", C.c_int64),
                ("sampler", C.c_int), ("generator", C.c_int), ("model", C.c_int),
                ("append_order", C.c_int)]


class qed_species(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "z", "px", "py", "pz", "w")] + \
               [("id", C.c_void_p), ("alive", C.c_void_p)] + \
               [(n, C.c_void_p) for n in ("ex", "ey", "ez", "bx", "by", "bz")] + \
               [("d_n", C.c_void_p), ("capacity", C.c_int64), ("q", C.c_int), ("pad_", C.c_int),
                ("tag", C.c_void_p), ("od_p", C.c_void_p), ("od_r", C.c_void_p)]


class qed_fields(C.Structure):
    _fields_ = [("mode", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("e", C.c_double * 3), ("b", C.c_double * 3), ("grid", C.c_void_p),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double)]


class qed_counters(C.Structure):
    _fields_ = [("emit_events", C.c_int64), ("pair_events", C.c_int64), ("substeps", C.c_int64),
                ("dropped", C.c_int64), ("domain", C.c_int64), ("status", C.c_uint32),
                ("pad_", C.c_uint32), ("hist", C.c_int64 * 64), ("deferred", C.c_int64)]

    def as_dict(self):
        return {"emit_events": self.emit_events, "pair_events": self.pair_events,
                "substeps": self.substeps, "dropped": self.dropped, "domain": self.domain,
                "status": self.status, "hist": list(self.hist), "deferred": self.deferred}


class qed_yee(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("pad_", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double)] + \
               [(n, C.c_void_p) for n in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz", "nodes")]


QED_TUNE_GROUPS, QED_TUNE_MAX_FACTOR = 5, 8
TUNE_GROUP_NAMES = ("stream", "chains", "order", "photon", "compact")
QED_SCHED_PARAMS, QED_SCHED_MAX_CANDIDATES = 5, 6
SCHED_NAMES = ("emit_lanes", "round_lanes", "scan_draws", "scan_left", "queue_trigger")


class qed_tuning(C.Structure):
    _fields_ = [("grid_factor", C.c_int * QED_TUNE_GROUPS), ("sched", C.c_int * QED_SCHED_PARAMS),
                ("ms_per_step", C.c_double),
                ("ms", (C.c_double * QED_TUNE_MAX_FACTOR) * QED_TUNE_GROUPS),
                ("sched_tried", (C.c_int * QED_SCHED_MAX_CANDIDATES) * QED_SCHED_PARAMS),
                ("sched_ms", (C.c_double * QED_SCHED_MAX_CANDIDATES) * QED_SCHED_PARAMS)]


# name -> (restype, argtypes); the exported C ABI, one entry per declaration
_P = C.c_void_p
SIGNATURES = {
    "qed_config_default": (None, [C.POINTER(qed_config)]),
    "qed_strerror": (C.c_char_p, [C.c_int]),
    "qed_init_tables": (C.c_int, [C.POINTER(qed_config), C.POINTER(_P), _P]),
    "qed_destroy": (None, [_P]),
    "qed_gather_push": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int64, _P]),
    "qed_emit": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species), C.POINTER(qed_fields),
                           C.c_int64, _P]),
    "qed_pair": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species), C.POINTER(qed_species),
                           C.POINTER(qed_fields), C.c_int64, _P]),
    "qed_compact": (C.c_int, [_P, C.POINTER(qed_species), _P]),
    "qed_compact_fill": (C.c_int, [_P, C.POINTER(qed_species), _P]),
    "qed_count_alive": (C.c_int, [_P, C.POINTER(qed_species), _P, _P]),
    "qed_step_fused": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species),
                                 C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int64, _P]),
    "qed_sample_xi": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, _P]),
    "qed_rates": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int64, _P]),
    "qed_sample_table": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int64, _P]),
    "qed_chi": (C.c_int, [_P, C.POINTER(qed_species), _P, _P]),
    "qed_fill_standing_wave": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_double, _P]),
    "qed_table_get": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.POINTER(C.c_double)]),
    "qed_read_counters": (C.c_int, [_P, C.POINTER(qed_counters), _P]),
    "qed_reset_counters": (C.c_int, [_P, _P]),
    "qed_last_device_status": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_int64)]),
    "qed_test_wait_expiry": (C.c_int, [_P, _P]),
    "qed_launch_count": (C.c_int64, [_P]),
    "qed_profile_begin": (C.c_int, [_P, C.c_int]),
    "qed_compact_noalloc": (C.c_int, [C.POINTER(qed_species), C.c_int, _P, _P]),
    "qed_run_batched": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species),
                                  C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int64, C.c_int,
                                  C.c_int, _P, _P]),
    "qed_autotune": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species),
                               C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int,
                               C.POINTER(C.c_int), C.POINTER(C.c_double), _P]),
    "qed_autotune_groups": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species),
                                      C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int,
                                      C.POINTER(qed_tuning), _P]),
    "qed_set_tuning": (C.c_int, [_P, C.POINTER(qed_tuning)]),
    "qed_lepton_step_host": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species),
                                       C.POINTER(qed_species), C.POINTER(qed_fields), C.c_int64,
                                       C.c_int64, _P]),
    "qed_pic_deposit": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_yee), C.c_double, _P, _P]),
    "qed_pic_fields": (C.c_int, [_P, C.POINTER(qed_yee), C.c_int, _P]),
    "qed_pic_step": (C.c_int, [_P, C.POINTER(qed_species), C.POINTER(qed_species), C.POINTER(qed_species),
                               C.POINTER(qed_yee), C.c_double, C.c_int64, _P]),
    "qed_mlp_load": (C.c_int, [_P, _P, C.c_size_t]),
    "qed_mlp_get": (C.c_int, [_P, _P, C.c_size_t]),
    "qed_mlp_train": (C.c_int, [_P, C.c_int64, C.c_float, C.c_uint64, C.POINTER(C.c_double), _P]),
    "qed_mlp_grad": (C.c_int, [_P, _P, _P, C.c_int64, _P, C.POINTER(C.c_double), _P]),
    "qed_profile_end": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int64)]),
    "qed_profile_end_phases": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}

_lib = None


def lib():
    """Load libqed.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1608_06356_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int, what: str) -> None:
    if code != QED_OK:
        raise QedError(code, what)
