"""Pins of the FP64 oracle's special functions and spectra to things the
mathematics and the paper fix independently of the oracle's own code:
quadrature exactness on polynomials, closed forms of K_{1/2}, SciPy's kv,
the K_{5/3} identity, the equality of formula I (Eq. 1) and formula II
(Eq. 4), the classic limit (Eq. 5), and the known asymptotes of the total
photon and pair rates."""
import math

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")
scipy_integrate = pytest.importorskip("scipy.integrate")


# ----------------------------------------------------------------- quadrature
def test_gk15_rule_exact_on_polynomials(orc):
    # Kronrod 15 points integrate degree <= 22 exactly, Gauss 7 degree <= 13;
    # a wrong node or weight breaks one of these.
    for k in range(0, 23):
        kr, g = orc.gk15_monomial(k, 0.0, 1.0)
        exact = 1.0 / (k + 1)
        assert abs(kr - exact) < 1e-14, k
        if k <= 13:
            assert abs(g - exact) < 1e-14, k
    kr, g = orc.gk15_monomial(14, -1.0, 1.0)
    assert abs(g - 2.0 / 15.0) > 1e-6  # the 7-point Gauss rule is not exact at 14


# ------------------------------------------------------------------- Bessel K
@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.1, 1.0, 7.5, 40.0, 300.0])
def test_besselk_half_closed_form(orc, x):
    exact = math.sqrt(math.pi / (2 * x)) * math.exp(-x)
    assert orc.besselk(0.5, x) == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("x", [1e-4, 0.01, 0.5, 3.0, 30.0, 200.0])
def test_besselk_int_half_closed_form(orc, x):
    # int_x^inf K_{1/2} = (pi/sqrt 2) erfc(sqrt x)
    exact = math.pi / math.sqrt(2) * math.erfc(math.sqrt(x))
    assert orc.besselk_int(0.5, x) == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("nu", [1 / 3, 2 / 3, 5 / 3])
def test_besselk_vs_scipy(orc, nu):
    for x in np.logspace(-6, 2.7, 40):
        assert orc.besselk(nu, x) == pytest.approx(scipy_special.kv(nu, x), rel=1e-12)


@pytest.mark.parametrize("nu", [1 / 3, 5 / 3])
def test_besselk_int_vs_scipy_quad(orc, nu):
    for x in (1e-3, 0.05, 0.7, 4.0, 25.0):
        ref, _ = scipy_integrate.quad(lambda s: scipy_special.kv(nu, s), x, np.inf,
                                      epsabs=0, epsrel=1e-12, limit=400)
        assert orc.besselk_int(nu, x) == pytest.approx(ref, rel=1e-9)


def test_k53_identity(orc):
    # K_{nu-1} + K_{nu+1} = -2 K'_nu  =>  int_x^inf K_{5/3} = 2 K_{2/3}(x) - int_x^inf K_{1/3}
    for x in np.logspace(-4, 2, 25):
        lhs = orc.besselk_int(5 / 3, x)
        rhs = 2 * orc.besselk(2 / 3, x) - orc.besselk_int(1 / 3, x)
        assert lhs == pytest.approx(rhs, rel=1e-11)


# ------------------------------------------------------------------- spectra
@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("xi", [1e-3, 0.1, 0.5, 0.9])
def test_formula_I_equals_formula_II(orc, xi, chi):
    # Fig. 1 / text: formula I [Eq. (1)] and formula II [Eq. (4)] coincide.
    assert orc.spec_I(xi, chi) == pytest.approx(orc.spec_II(xi, chi), rel=1e-6)


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
def test_classic_limit_small_xi(orc, chi):
    # Eq. (5) with zeta = 2 xi/(3 chi) is the xi -> 0 limit of Eq. (1):
    # the ratio tends to 1 linearly in xi.
    for xi in (1e-5, 1e-6):
        r = orc.spec_classic(xi, chi) / orc.spec_I(xi, chi)
        assert abs(r - 1) < 50 * xi


def test_classic_limit_small_chi(orc):
    # chi -> 0 at fixed delta: the quantum spectrum tends to the classic one.
    # At fixed delta, zeta = delta (1 - xi) with xi ~ 1.5 chi delta, so the
    # ratio approaches 1 linearly in chi (roughly as 1.5 chi delta^2).
    for delta in (0.01, 0.3, 2.0, 8.0):
        devs = []
        for chi in (1e-3, 1e-4):
            xi = 1.5 * chi * delta / (1 + 1.5 * chi * delta)
            devs.append(abs(orc.spec_classic(xi, chi) / orc.spec_I(xi, chi) - 1))
        assert devs[1] < 2.0 * 1e-4 * (1 + delta) ** 2
        assert devs[1] < 0.15 * devs[0] + 1e-12


def test_classic_overestimates_hard_photons(orc):
    # Text after Fig. 1: the classic formula overestimates the high-energy part.
    for chi in (0.1, 1.0, 10.0):
        assert orc.spec_classic(0.5, chi) > orc.spec_I(0.5, chi)


# ---------------------------------------------------------- rate asymptotes
def test_photon_rate_small_chi_expansion(orc):
    # Total rate for xi_min = 0: (5/(2 sqrt 3)) chi (1 - (8 sqrt 3/15) chi + O(chi^2)),
    # the classical photon number rate plus its first quantum correction.
    c0 = 5 / (2 * math.sqrt(3))
    c1 = 8 * math.sqrt(3) / 15
    for chi in (1e-2, 1e-3, 1e-4):
        r = orc.cum_photon(0.0, 1.0, chi) / (c0 * chi)
        assert abs(r - (1 - c1 * chi)) < 5 * chi * chi


def test_photon_rate_large_chi(orc):
    # chi -> inf: delta -> 0, K_{2/3}(delta) ~ Gamma(2/3)/2 (2/delta)^{2/3}, and the
    # xi integral is a sum of two Beta functions: (14/27) Gamma(2/3) 3^{2/3} chi^{2/3}.
    c = 14 / 27 * math.gamma(2 / 3) * 3 ** (2 / 3)
    devs = [abs(orc.cum_photon(0.0, 1.0, chi) / (c * chi ** (2 / 3)) - 1) for chi in (1e3, 1e4, 1e5)]
    assert devs[2] < devs[1] < devs[0]
    assert devs[2] < 0.02


@pytest.mark.parametrize("sign", [1, -1])
def test_pair_rate_small_chi_laplace(orc, sign):
    # Laplace's method at xi = 1/2 (delta_min = 8/(3 chi)):
    # int spec_pair -> (2 + sign) sqrt(3)/(16 sqrt 2) chi exp(-8/(3 chi)).
    # sign=+1 gives the textbook Breit-Wheeler value (3/16) sqrt(3/2).
    c = (2 + sign) * math.sqrt(3) / (16 * math.sqrt(2))
    prev = None
    for chi in (0.04, 0.02, 0.01):
        r = orc.cum_pair(0.0, 1.0, chi, sign) / (c * chi * math.exp(-8 / (3 * chi)))
        dev = abs(r - 1)
        assert dev < 3 * chi
        if prev is not None:
            assert dev < prev
        prev = dev


def test_pair_rate_large_chi(orc):
    # chi -> inf: (15/14) 3^{2/3} Gamma(2/3)^3 / (sqrt 3 pi Gamma(1/3)) chi^{2/3}
    c = 15 / 14 * 3 ** (2 / 3) * math.gamma(2 / 3) ** 3 / (math.sqrt(3) * math.pi * math.gamma(1 / 3))
    devs = [abs(orc.cum_pair(0.0, 1.0, chi, 1) / (c * chi ** (2 / 3)) - 1) for chi in (1e3, 1e4, 1e5)]
    assert devs[2] < devs[1] < devs[0]
    assert devs[2] < 0.02


def test_pair_spectrum_symmetric(orc):
    for chi in (0.3, 3.0):
        for xi in (0.05, 0.2, 0.45):
            assert orc.spec_pair(xi, chi) == pytest.approx(orc.spec_pair(1 - xi, chi), rel=1e-13)


# ------------------------------------------------ cumulative integration
@pytest.mark.parametrize("chi", [1e-3, 0.3, 20.0])
def test_cum_photon_vs_independent_quadrature(orc, chi):
    # Integrate the oracle's own spectrum with SciPy (different rule, xi^(1/3)
    # substitution written here) to check the oracle's outer integration.
    f = lambda t: 3 * t * t * orc.spec_I(t ** 3, chi)
    for a, b in ((0.0, 1.0), (1e-4, 0.5), (0.01, 1.0)):
        ref, _ = scipy_integrate.quad(f, a ** (1 / 3), b ** (1 / 3), epsabs=0, epsrel=1e-11, limit=500)
        assert orc.cum_photon(a, b, chi) == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("chi", [0.2, 5.0])
def test_cum_pair_vs_independent_quadrature(orc, chi):
    f = lambda x: orc.spec_pair(x, chi)
    ref, _ = scipy_integrate.quad(f, 0.0, 1.0, points=[0.5], epsabs=0, epsrel=1e-11, limit=500)
    assert orc.cum_pair(0.0, 1.0, chi) == pytest.approx(ref, rel=1e-9)
