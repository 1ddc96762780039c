"""The classic-limit photon model (Eq. 5, QED_MODEL_CLASSIC) on the GPU: the
tables built from it against the oracle's model switch, and Fig. 1's
comparison (the classic spectrum overestimates hard photons).

Tolerances: FP32 rates 1e-4 relative, FP64 1e-6 (1e-3 for rates below 1e-8
of the largest, deep in the xi_min cut's exponential tail); xi from the
inverse CDF 1e-5 relative (both precisions), wherever the rate is not zero
to within e^-69 (there the cut leaves nothing to sample); chi in [1e-3, 3].
The classic spectrum's tail near xi = 1 varies like exp(-2 / (3 chi)) with chi,
so the FP32 classic tables have 10 rows per unit of ln chi (formula I's have
4)."""
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


def test_classic_rate_and_xi_match_oracle(api, orc):
    from paper_1608_06356_gb300 import workloads as W
    rng = np.random.default_rng(21)
    n = 2000
    chi = np.exp(rng.uniform(np.log(1e-3), np.log(3.0), n))
    gamma = np.exp(rng.uniform(np.log(10), np.log(1e5), n))
    cfg = orc.make_config(model=orc.MODEL_CLASSIC)
    Wo = orc.rate_photon(cfg, chi, gamma)
    assert np.max(Wo / orc.rate_photon(orc.make_config(), chi, gamma)) > 1.05  # not formula I
    words = W.uniform_words(n, seed=8)
    words[:4] = [0, 1, 2**32 - 1, 2**32 - 2]
    r2, c2 = orc.uniform_from_word(words)
    xo = orc.sample_photon(cfg, chi, gamma, r2, c2)
    # rates in the exponential tail of the xi_min cut (below 1e-8 of the
    # largest) carry the forward table's absolute error in kappa_min: 1e-3
    big = Wo > 1e-8 * Wo.max()
    tail = ~big & (Wo > 1e-20 * Wo.max())
    for prec, rtol in ((0, 1e-4), (1, 1e-6)):
        ctx = api.qed_init_tables(api.config(precision=prec, model=1))
        Wg = api.qed_rates(ctx, 0, torch.tensor(chi, device="cuda"),
                           torch.tensor(gamma, device="cuda")).cpu().numpy()
        np.testing.assert_allclose(Wg[big], Wo[big], rtol=rtol)
        np.testing.assert_allclose(Wg[tail], Wo[tail], rtol=1e-3)
        assert np.all(Wg[~big] <= 2e-8 * Wo.max())
        xg = api.qed_sample_table(ctx, 0, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda"),
                                  torch.tensor(words.view(np.int32), device="cuda")).cpu().numpy()
        live = Wo > 1e-30 * Wo.max()
        rel = np.abs(xg / xo - 1)[live]
        assert live.sum() >= n - 10
        assert rel.max() <= 1e-5, (prec, rel.max())


def test_fig1_classic_overestimates_hard_photons(api):
    """Photon-energy spectra sampled with each model at chi = 0.1, 1, 10
    (gamma = 1000): the classic model puts more photons above xi = 0.5."""
    nu = 1 << 20
    frac = {}
    for model in (0, 1):
        ctx = api.qed_init_tables(api.config(model=model))
        for chi in (0.1, 1.0, 10.0):
            c = torch.full((nu,), chi, device="cuda")
            g = torch.full((nu,), 1000.0, device="cuda")
            xi = torch.empty(nu, device="cuda")
            api.qed_sample_xi(ctx, c, g, xi, 3)
            frac[(model, chi)] = float((xi > 0.5).float().mean())
    for chi in (0.1, 1.0, 10.0):
        assert frac[(1, chi)] > 1.2 * frac[(0, chi)] + 1e-5, (chi, frac)
