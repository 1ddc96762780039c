"""The oracle's Methods II and III (the paper's alternative photon event
generators, text around Fig. 2) against closed forms.

For identical electrons in a uniform magnetic field perpendicular to p the
push keeps gamma and chi, so W_rad -- and a = W_rad Dt per step -- is the same
for every particle until its first emission.  The probability that a particle
has not emitted after n steps is then
  Method II  (emit when 1 - exp(-P_cum) > r3):  exp(-n a)
  Method III (emit when P_cum > r3):            max(0, 1 - n a)
i.e. Method II is a Poisson process of rate W_rad (equivalent to Method I),
while Method III as printed emits at twice that rate (mean optical depth 1/2
at emission).  The state reset after an emission (P_cum = 0, a fresh r3) and
the Philox words used are checked directly."""
import numpy as np
import pytest

N_PART = 2000
STEPS = 12


def _ensemble(orc, generator, dt=0.04, gamma0=1000.0, chi0=0.5, seed=3):
    cfg = orc.make_config(dt=dt, seed=seed, generator=generator)
    bz = chi0 * orc.A_S_1UM / gamma0
    fields = orc.uniform_fields((0, 0, 0), (0, 0, bz))
    p0 = np.sqrt(gamma0 ** 2 - 1.0)
    n = N_PART
    e = orc.Species(n, -1.0, with_od=True).load(
        x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), px=np.full(n, p0), py=np.zeros(n),
        pz=np.zeros(n), w=np.ones(n), id=np.arange(100, 100 + n, dtype=np.uint64))
    chi = orc.chi_lepton([p0, 0, 0], [0, 0, 0], [0, 0, bz])
    a = float(orc.rate_photon(cfg, chi, gamma0)[0]) * dt
    return cfg, fields, e, a


def _first_emission(orc, generator):
    cfg, fields, e, a = _ensemble(orc, generator)
    g = orc.Species(N_PART * STEPS + 16, 0.0, with_alive=True)
    first = np.full(N_PART, -1)
    for s in range(STEPS):
        orc.step(cfg, fields, e, None, g, s)
        emitted = e.view("od_p") == 0.0
        first[(first < 0) & emitted] = s
    return first, a


def _check_survival(first, expected):
    for n in range(1, STEPS + 1):
        s_meas = np.mean((first < 0) | (first >= n))
        s_exp = expected(n)
        sigma = np.sqrt(max(s_exp * (1 - s_exp), 1e-4) / N_PART)
        assert abs(s_meas - s_exp) < 5 * sigma + 1e-3, (n, s_meas, s_exp)


def test_method_ii_is_poisson_at_rate_w(orc):
    first, a = _first_emission(orc, orc.GEN_METHOD_II)
    assert 0.03 < a < 0.1
    _check_survival(first, lambda n: np.exp(-n * a))


def test_method_iii_emits_at_twice_the_rate(orc):
    first, a = _first_emission(orc, orc.GEN_METHOD_III)
    # the waiting optical depth is uniform on (0, 1) (mean 1/2) instead of
    # exponential (mean 1): the printed Method III is not equivalent to I and II
    _check_survival(first, lambda n: max(0.0, 1.0 - n * a))


def test_state_update_uses_the_emission_draw(orc):
    cfg, fields, e, a = _ensemble(orc, orc.GEN_METHOD_II, dt=0.5)  # a ~ 0.8: many emit
    g = orc.Species(N_PART + 16, 0.0, with_alive=True)
    orc.step(cfg, fields, e, None, g, 7)
    n = N_PART
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(100, 100 + n)
    ctr[:, 2] = 7
    words = orc.philox(ctr, np.tile(np.array([cfg.seed & 0xFFFFFFFF, cfg.seed >> 32], dtype=np.uint32), (n, 1)))
    r3_first, _ = orc.uniform_from_word(words[:, 3])
    r3_next, _ = orc.uniform_from_word(words[:, 2])
    od_p, od_r = e.view("od_p"), e.view("od_r")
    emit = od_p == 0.0
    # one step from P = 0: an emission exactly when 1 - exp(-a) > r3 (word 3)
    np.testing.assert_array_equal(emit, -np.expm1(-a) > r3_first)
    assert 0.2 * n < emit.sum() < 0.9 * n and g.n == emit.sum()
    np.testing.assert_array_equal(od_r[emit], r3_next[emit])
    np.testing.assert_array_equal(od_r[~emit], r3_first[~emit])
    np.testing.assert_allclose(od_p[~emit], a, rtol=1e-12)
