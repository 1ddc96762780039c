"""GPU tables, rates and inverse CDF against the FP64 oracle.

Tolerances (stated in the tests): FP64 table entries and FP64 rates 1e-6
relative; FP32 rates 1e-4 relative; xi from the inverse CDF 1e-5 relative."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1608_06356_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx32(api):
    return api.qed_init_tables(api.config(precision=0))


@pytest.fixture(scope="module")
def ctx64(api):
    return api.qed_init_tables(api.config(precision=1))


def _pick(rng, n, k):
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def _kappa_oracle(orc, chi, delta):
    xi = 1.5 * chi * delta / (1 + 1.5 * chi * delta)
    tot = orc.cum_photon(0, 1, chi)
    lo, hi = orc.cum_photon(0, xi, chi), orc.cum_photon(xi, 1, chi)
    w = -math.log1p(-lo / tot) if lo < 0.5 * tot else -math.log(hi / tot)
    return math.log(w)


@pytest.mark.parametrize("prec", [0, 1])
def test_photon_tables_match_oracle(api, orc, ctx32, ctx64, prec):
    ctx = ctx64 if prec else ctx32
    rng = np.random.default_rng(1 + prec)
    R, gR = api.qed_table_get(ctx, 0)
    F, gF = api.qed_table_get(ctx, 1)
    Y, gY = api.qed_table_get(ctx, 2)
    # rate rows
    for i in _pick(rng, gR["n0"], 12):
        chi = math.exp(gR["x0_0"] + i * gR["h_0"])
        assert R[i, 0] == pytest.approx(math.log(orc.cum_photon(0, 1, chi)), abs=1e-6)
    # forward entries kappa(l, y)
    for _ in range(40):
        i, j = rng.integers(0, gF["n0"]), rng.integers(0, gF["n1"])
        chi = math.exp(gF["x0_0"] + i * gF["h_0"])
        y = gF["x0_1"] + j * gF["h_1"]
        assert F[i, j] == pytest.approx(_kappa_oracle(orc, chi, math.exp(y)), abs=1e-6), (chi, y)
    # inverse entries ln delta(l, kappa): xi compared at 1e-6 relative
    cfg0 = orc.make_config(xi_min_energy=0.0)
    for _ in range(40):
        i, m = rng.integers(0, gY["n0"]), rng.integers(0, gY["n1"])
        chi = math.exp(gY["x0_0"] + i * gY["h_0"])
        k = gY["x0_1"] + m * gY["h_1"]
        if k > 4.0:
            continue  # u within e^-50 of 1: below the oracle's double resolution of 1 - u
        w = math.exp(k)
        u, c = -math.expm1(-w), math.exp(-w)
        xo = orc.sample_photon(cfg0, chi, 1e6, u, c)[0]
        a = 1.5 * chi * math.exp(Y[i, m])
        assert a / (1 + a) == pytest.approx(xo, rel=1e-6), (chi, k)


@pytest.mark.parametrize("prec", [0, 1])
def test_pair_tables_match_oracle(api, orc, ctx32, ctx64, prec):
    ctx = ctx64 if prec else ctx32
    rng = np.random.default_rng(11 + prec)
    P, gP = api.qed_table_get(ctx, 3)
    Yp, gYp = api.qed_table_get(ctx, 4)
    for i in _pick(rng, gP["n0"], 10):
        chi = math.exp(gP["x0_0"] + i * gP["h_0"])
        ref = math.log(orc.cum_pair(0, 1, chi, 1)) + 8 / (3 * chi)
        assert P[i, 0] == pytest.approx(ref, abs=1e-6), chi
    cfg = orc.make_config()
    for _ in range(40):
        i, m = rng.integers(0, gYp["n0"]), rng.integers(0, gYp["n1"])
        chi = math.exp(gYp["x0_0"] + i * gYp["h_0"])
        k = gYp["x0_1"] + m * gYp["h_1"]
        L = math.exp(k)
        u = 0.5 * math.exp(-L)
        if u < 1e-300:
            continue
        xo = orc.sample_pair(cfg, chi, u, 1 - u)[0]
        D = math.exp(Yp[i, m])
        r = math.sqrt(D / (1 + D))
        xg = 1 / (2 * (1 + D) * (1 + r))
        assert xg == pytest.approx(xo, rel=1e-6), (chi, k)


@pytest.mark.parametrize("prec,rtol", [(0, 1e-4), (1, 1e-6)])
def test_photon_rate_matches_oracle(api, orc, ctx32, ctx64, prec, rtol):
    ctx = ctx64 if prec else ctx32
    rng = np.random.default_rng(5)
    n = 400
    chi = np.exp(rng.uniform(np.log(1e-4), np.log(500), n))
    gamma = np.exp(rng.uniform(np.log(3), np.log(1e5), n))
    Wg = api.qed_rates(ctx, 0, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda")).cpu().numpy()
    Wo = orc.rate_photon(orc.make_config(), chi, gamma)
    big = Wo > 1e-30 * Wo.max()
    np.testing.assert_allclose(Wg[big], Wo[big], rtol=rtol)
    assert np.all(Wg[~big] <= 1e-25 * Wo.max())


@pytest.mark.parametrize("prec,rtol", [(0, 1e-4), (1, 1e-6)])
def test_pair_rate_matches_oracle(api, orc, ctx32, ctx64, prec, rtol):
    ctx = ctx64 if prec else ctx32
    rng = np.random.default_rng(6)
    n = 300
    chi = np.exp(rng.uniform(np.log(0.03), np.log(500), n))
    gamma = np.exp(rng.uniform(np.log(2.5), np.log(1e5), n))
    Wg = api.qed_rates(ctx, 1, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda")).cpu().numpy()
    Wo = orc.rate_pair(orc.make_config(), chi, gamma)
    np.testing.assert_allclose(Wg, Wo, rtol=rtol)
    # below chi_pair_min and below threshold the rate is zero on both sides
    z = api.qed_rates(ctx, 1, torch.tensor([0.01, 1.0], device="cuda", dtype=torch.float64),
                      torch.tensor([1e3, 1.5], device="cuda", dtype=torch.float64)).cpu().numpy()
    assert np.all(z == 0)
    assert orc.rate_pair(orc.make_config(), np.array([1.0]), np.array([1.5]))[0] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_photon_xi_matches_oracle(api, orc, ctx32, ctx64, prec):
    ctx = ctx64 if prec else ctx32
    from paper_1608_06356_gb300 import workloads as W
    rng = np.random.default_rng(7 + prec)
    n = 600
    chi = np.exp(rng.uniform(np.log(1e-3), np.log(100), n))
    gamma = np.exp(rng.uniform(np.log(10), np.log(1e4), n))
    words = W.uniform_words(n, seed=3 + prec)
    words[:4] = [0, 1, 2**32 - 1, 2**32 - 2]
    xg = api.qed_sample_table(ctx, 0, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda"),
                              torch.tensor(words.view(np.int32), device="cuda")).cpu().numpy()
    r2, c2 = orc.uniform_from_word(words)
    xo = orc.sample_photon(orc.make_config(), chi, gamma, r2, c2)
    rel = np.abs(xg / xo - 1)
    worst = np.argsort(rel)[-5:]
    assert rel.max() <= 1e-5, [(chi[i], gamma[i], r2[i], xg[i], xo[i], rel[i]) for i in worst]


@pytest.mark.parametrize("prec", [0, 1])
def test_pair_xi_matches_oracle(api, orc, ctx32, ctx64, prec):
    ctx = ctx64 if prec else ctx32
    from paper_1608_06356_gb300 import workloads as W
    rng = np.random.default_rng(9 + prec)
    n = 400
    chi = np.exp(rng.uniform(np.log(0.05), np.log(300), n))
    words = W.uniform_words(n, seed=13 + prec)
    words[:4] = [0, 5, 2**32 - 1, 2**31]
    xg = api.qed_sample_table(ctx, 1, torch.tensor(chi, device="cuda"), None,
                              torch.tensor(words.view(np.int32), device="cuda")).cpu().numpy()
    r2, c2 = orc.uniform_from_word(words)
    xo = orc.sample_pair(orc.make_config(), chi, r2, c2)
    rel = np.abs(xg / xo - 1)
    worst = np.argsort(rel)[-5:]
    assert rel.max() <= 1e-5, [(chi[i], r2[i], xg[i], xo[i], rel[i]) for i in worst]


def test_isolated_sampler_matches_oracle(api, orc, ctx32):
    # qed_sample_xi: r2 from Philox(seed; id = i, step, sub 0, stream 0) word 1
    from paper_1608_06356_gb300 import workloads as W
    n, step = 3000, 17
    _, chi, gamma = W.chi_target(n, seed=4)
    x = torch.empty(n, device="cuda")
    api.qed_sample_xi(ctx32, torch.tensor(chi, dtype=torch.float32, device="cuda"),
                      torch.tensor(gamma, dtype=torch.float32, device="cuda"), x, step)
    xg = x.cpu().numpy().astype(np.float64)
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = step
    words = orc.philox(ctr, np.zeros((n, 2), dtype=np.uint32))[:, 1]
    r2, c2 = orc.uniform_from_word(words)
    chi32 = chi.astype(np.float32).astype(np.float64)
    g32 = gamma.astype(np.float32).astype(np.float64)
    sel = np.arange(0, n, 5)  # every 5th: the oracle inverts by quadrature
    xo = orc.sample_photon(orc.make_config(), chi32[sel], g32[sel], r2[sel], c2[sel])
    ok = xo > 0
    np.testing.assert_allclose(xg[sel][ok], xo[ok], rtol=2e-5)
