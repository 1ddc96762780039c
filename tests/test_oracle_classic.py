"""The oracle's classic-limit photon model (Eq. 5, zeta = 2 xi / (3 chi)),
the alternative to formula I used for Fig. 1's comparison.

Pins: over 0 < xi < infinity the classic spectrum integrates in closed form
to (5 / (2 sqrt 3)) chi for every chi (int_0^inf x K_{5/3}(x) dx = 5 pi / 3),
so at small chi its rate over 0 < xi < 1 is that value; at chi = 1 and 10 it
exceeds formula I (the classic spectrum overestimates hard photons); and the
model switch reaches the rate and the sampler (inverse-CDF round trip)."""
import numpy as np
import pytest


def test_classic_rate_closed_form_small_chi(orc):
    for chi in (1e-3, 3e-3, 1e-2):
        val = orc.cum_photon(0.0, 1.0, chi, model=orc.MODEL_CLASSIC)
        assert val == pytest.approx(5.0 / (2.0 * np.sqrt(3.0)) * chi, rel=1e-8)


def test_classic_exceeds_formula_i_for_hard_photons(orc):
    for chi in (1.0, 10.0):
        hard_c = orc.cum_photon(0.5, 1.0, chi, model=orc.MODEL_CLASSIC)
        hard_i = orc.cum_photon(0.5, 1.0, chi, model=orc.MODEL_FORMULA_I)
        assert hard_c > 1.3 * hard_i
    # and they agree for soft photons
    chi = 1.0
    soft_c = orc.cum_photon(0.0, 1e-4, chi, model=orc.MODEL_CLASSIC)
    soft_i = orc.cum_photon(0.0, 1e-4, chi, model=orc.MODEL_FORMULA_I)
    assert soft_c == pytest.approx(soft_i, rel=2e-3)


def test_model_switch_reaches_rate_and_sampler(orc):
    chi, gamma = 2.0, 500.0
    for model in (orc.MODEL_FORMULA_I, orc.MODEL_CLASSIC):
        cfg = orc.make_config(model=model)
        W = float(orc.rate_photon(cfg, chi, gamma)[0])
        total = orc.cum_photon(2.0 / gamma, 1.0, chi, model=model)
        assert W == pytest.approx(cfg.alpha * cfg.a_S / gamma * total, rel=1e-12)
        for r2 in (0.1, 0.5, 0.9):
            xi = float(orc.sample_photon(cfg, chi, gamma, r2, 1.0 - r2)[0])
            part = orc.cum_photon(2.0 / gamma, xi, chi, model=model)
            assert part / total == pytest.approx(r2, rel=1e-9)
