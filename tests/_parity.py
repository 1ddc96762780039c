"""Helpers for element-wise GPU-vs-oracle comparisons of a QED step.

The Method I decision W*Dt_s > r1 is an integer decided by floating point.
The GPU (FP32 tables) and the oracle (FP64 quadrature) agree on W within the
rate tolerance, so a particle whose draw lies within that tolerance of the
threshold may legitimately flip; such particles (and their children) are
excluded from the element-wise comparison and counted.  Everything else must
match: counts, child ids, momenta, positions, weights."""
from __future__ import annotations

import math

import numpy as np


def first_substep_threshold(orc, cfg, states, fields_fn, q, photon=False, rtol=1e-4, push=True):
    """Per particle: W*Dt_s of its first sub-step (after the oracle's push,
    unless push=False), and whether the sub-step count N = ceil(W Dt /
    wdt_max) is within the rate tolerance of changing."""
    n = len(states["x"])
    chis, gammas = np.zeros(n), np.zeros(n)
    for i in range(n):
        E, B = fields_fn(i)
        p = np.array([states["px"][i], states["py"][i], states["pz"][i]], dtype=np.float64)
        if photon:
            g = float(np.linalg.norm(p))
            chi = orc.chi_photon(p, E, B, cfg.a_S)
        else:
            if push:
                p, g = orc.boris(p, E, B, q, cfg.dt)
            else:
                g = float(np.sqrt(1.0 + p @ p))
            chi = orc.chi_lepton(p, E, B, cfg.a_S)
        chis[i], gammas[i] = chi, g
    W = (orc.rate_pair if photon else orc.rate_photon)(cfg, chis, gammas)
    amb = np.zeros(n, dtype=bool)
    thr = np.zeros(n)
    for i in range(n):
        wdt = W[i] * cfg.dt
        N = 1 if wdt <= cfg.wdt_max else math.ceil(wdt / cfg.wdt_max)
        frac = wdt / cfg.wdt_max
        if frac > 1 - rtol and abs(frac - round(frac)) < rtol * frac:
            amb[i] = True
        thr[i] = W[i] * cfg.dt / N
    return amb, thr


def ambiguous(orc, cfg, states, fields_fn, q, step, photon=False, rtol=1e-4, atol=1e-7, push=True):
    """Indices whose first-sub-step Method I decision is within tolerance."""
    amb, thr = first_substep_threshold(orc, cfg, states, fields_fn, q, photon, rtol, push)
    n = len(states["x"])
    ids = np.asarray(states["id"], dtype=np.uint64)
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = (ids & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (ids >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = step
    ctr[:, 3] = 1 if photon else 0
    key = np.array([cfg.seed & 0xFFFFFFFF, cfg.seed >> 32], dtype=np.uint32)
    words = orc.philox(ctr, np.tile(key, (n, 1)))[:, 0]
    r1, _ = orc.uniform_from_word(words)
    tol = np.maximum(atol, rtol * thr)
    amb |= np.abs(r1 - thr) <= tol
    return amb


def to32(d):
    """Round float arrays to float32 (then back to float64) so that both sides
    start from identical inputs."""
    out = {}
    for k, v in d.items():
        v = np.asarray(v)
        out[k] = v.astype(np.float32).astype(np.float64) if v.dtype.kind == "f" else v
    return out


def by_id(h):
    ids = np.asarray(h["id"], dtype=np.uint64)
    order = np.argsort(ids, kind="stable")
    return ids[order], {k: np.asarray(v)[order] for k, v in h.items()}


def oracle_species(orc, cap, q, st, fields=False, alive=False):
    s = orc.Species(cap, q, per_particle_fields=fields, with_alive=alive)
    s.load(**st)
    return s


def oracle_host(s):
    out = {k: s.view(k).copy() for k in ("x", "y", "z", "px", "py", "pz", "w", "id")}
    if s.alive is not None:
        out["alive"] = s.view("alive").copy()
    return out
