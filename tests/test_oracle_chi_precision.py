"""Pins of the oracle's chi (Eqs. 2 and 3) where the vector sum cancels: a
lepton or photon moving along (or close to) the propagation direction of a
plane wave E = E0 y, B = E0 z travelling along x.

References, independent of the oracle:
- Eq. (2) / Eq. (3) evaluated on the same inputs in 50-digit arithmetic
  (mpmath), for any direction and field;
- closed forms for inputs in the x-y plane: a lepton at angle theta to x,
  chi_e = (E0 / a_S) gamma (1 - beta cos theta)
        = (E0 / a_S) (1 / (gamma + p) + 2 p sin^2(theta / 2)),
  and a photon, chi_ph = (k E0 / a_S) 2 sin^2(theta / 2).

The oracle evaluates the printed formula in FP64.  Its error is the
rounding of the vector sum E + v x B (a few units of eps |E|, eps |B|)
amplified by the cancellations in it and in (E + v x B)^2 - (v.E)^2:
`literal_bound` states that bound per input, and the pins hold the oracle to
it (for an exact plane wave it is about 2 gamma^2 eps for the lepton and
eps / (1 - cos theta) for the photon)."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

A_S = 412148.45
EPS = 2.0 ** -52


def chi_exact(p, E, B, a_S, photon, dps=50):
    """Eq. (2) (lepton) or Eq. (3) (photon) on the given inputs, 50 digits."""
    with mp.workdps(dps):
        p = [mp.mpf(float(v)) for v in p]
        E = [mp.mpf(float(v)) for v in E]
        B = [mp.mpf(float(v)) for v in B]
        pp = p[0] ** 2 + p[1] ** 2 + p[2] ** 2
        g = mp.sqrt(pp) if photon else mp.sqrt(1 + pp)
        v = [c / g for c in p]
        f = [E[0] + v[1] * B[2] - v[2] * B[1], E[1] + v[2] * B[0] - v[0] * B[2],
             E[2] + v[0] * B[1] - v[1] * B[0]]
        ve = v[0] * E[0] + v[1] * E[1] + v[2] * E[2]
        s = f[0] ** 2 + f[1] ** 2 + f[2] ** 2 - ve ** 2
        return float(g / a_S * mp.sqrt(max(s, mp.mpf(0))))


def literal_bound(p, E, B, photon):
    """Relative error bound of chi from Eq. (2)/(3) evaluated as printed in
    FP64: each component of f = E + v x B carries <= 3 eps (|E| + |B|), v.E
    <= 3 eps |E|, so s = f^2 - (v.E)^2 carries <= 6 eps (|E| + |B|) (2|f| +
    |v.E|), and chi = sqrt(s) half of that relative to s (times 2 for the
    rounding of v and the final operations)."""
    p, E, B = (np.asarray(v, dtype=np.float64) for v in (p, E, B))
    g = np.linalg.norm(p) if photon else np.sqrt(1.0 + p @ p)
    v = p / g
    f = E + np.cross(v, B)
    ve = v @ E
    s = f @ f - ve * ve
    nE, nB = np.linalg.norm(E), np.linalg.norm(B)
    return 6.0 * EPS * (nE + nB) * (2 * np.linalg.norm(f) + abs(ve)) / max(s, 1e-300) + 1e-13


def lepton_case(gamma, theta, chi_target=1.0):
    p = np.sqrt(gamma * gamma - 1.0)
    one_m = 1.0 / (gamma * (gamma + p)) + 2.0 * (p / gamma) * np.sin(theta / 2) ** 2
    E0 = chi_target * A_S / (gamma * one_m)
    return np.array([p * np.cos(theta), p * np.sin(theta), 0.0]), np.array([0.0, E0, 0.0]), \
        np.array([0.0, 0.0, E0]), E0


@pytest.mark.parametrize("gamma", [10.0, 1e2, 1e3, 1e4])
@pytest.mark.parametrize("theta", [0.0, 1e-4, 1e-2])
def test_oracle_chi_lepton_comoving(orc, gamma, theta):
    p, E, B, E0 = lepton_case(gamma, theta)
    pm = np.sqrt(gamma * gamma - 1.0)
    # closed form on the exact inputs (p along (cos, sin) is rounded: use its angle)
    th = np.arctan2(p[1], p[0])
    pe = np.hypot(p[0], p[1])
    ge = np.sqrt(1.0 + pe * pe)
    closed = E0 / A_S * (1.0 / (ge + pe) + 2.0 * pe * np.sin(th / 2) ** 2)
    exact = chi_exact(p, E, B, A_S, photon=False)
    assert exact == pytest.approx(closed, rel=1e-13)
    got = orc.chi_lepton(p, E, B, A_S)
    bound = literal_bound(p, E, B, photon=False)
    assert abs(got - exact) <= bound * exact, (got, exact, bound)
    assert pm > 0


@pytest.mark.parametrize("theta", [1e-3, 1e-2, 0.3, 1.0])
@pytest.mark.parametrize("k", [10.0, 1e4])
def test_oracle_chi_photon_comoving(orc, theta, k):
    E0 = 1e3
    p = np.array([k * np.cos(theta), k * np.sin(theta), 0.0])
    E, B = np.array([0.0, E0, 0.0]), np.array([0.0, 0.0, E0])
    th = np.arctan2(p[1], p[0])
    closed = np.hypot(p[0], p[1]) * E0 / A_S * 2.0 * np.sin(th / 2) ** 2
    exact = chi_exact(p, E, B, A_S, photon=True)
    assert exact == pytest.approx(closed, rel=1e-13)
    got = orc.chi_photon(p, E, B, A_S)
    bound = literal_bound(p, E, B, photon=True)
    assert abs(got - exact) <= bound * exact, (got, exact, bound)


def test_oracle_chi_rotated_fields(orc):
    """Random rotations of co-moving configurations (rotated inputs rounded
    to FP32, so the field is no longer an exact plane wave): the oracle
    against the 50-digit evaluation of Eq. (2) on those inputs."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        gamma = float(np.exp(rng.uniform(np.log(10.0), np.log(1e4))))
        theta = float(rng.choice([0.0, 1e-4, 1e-3, 1e-2]))
        p, E, B, _ = lepton_case(gamma, theta)
        q, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        p, E, B = ((q @ v).astype(np.float32).astype(np.float64) for v in (p, E, B))
        exact = chi_exact(p, E, B, A_S, photon=False)
        got = orc.chi_lepton(p, E, B, A_S)
        assert abs(got - exact) <= literal_bound(p, E, B, photon=False) * exact
