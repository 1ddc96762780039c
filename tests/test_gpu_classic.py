"""The classic-limit photon model (Eq. 5, QED_MODEL_CLASSIC) on the GPU: the
tables built from it against the oracle's model switch, and Fig. 1's
comparison (the classic spectrum overestimates hard photons).

Tolerances as for formula I: FP32 rates 1e-4 relative, FP64 1e-6; xi from
the inverse CDF 1e-5 relative.  chi stays at or below 3, where the dropped
tail beyond delta = 200 (1 - xi < 1/(1 + 300 chi)) is below 1e-6 of the rate."""
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


@pytest.mark.parametrize("prec,rtol", [(0, 1e-4), (1, 1e-6)])
def test_classic_rate_matches_oracle(api, orc, prec, rtol):
    ctx = api.qed_init_tables(api.config(precision=prec, model=1))
    rng = np.random.default_rng(21)
    n = 300
    chi = np.exp(rng.uniform(np.log(1e-3), np.log(3.0), n))
    gamma = np.exp(rng.uniform(np.log(10), np.log(1e5), n))
    Wg = api.qed_rates(ctx, 0, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda")).cpu().numpy()
    Wo = orc.rate_photon(orc.make_config(model=orc.MODEL_CLASSIC), chi, gamma)
    np.testing.assert_allclose(Wg, Wo, rtol=rtol)
    # and it is not formula I's rate
    Wi = orc.rate_photon(orc.make_config(), chi, gamma)
    assert np.max(Wo / Wi) > 1.05


@pytest.mark.parametrize("prec", [0, 1])
def test_classic_xi_matches_oracle(api, orc, prec):
    from paper_1608_06356_gb300 import workloads as W
    ctx = api.qed_init_tables(api.config(precision=prec, model=1))
    rng = np.random.default_rng(33 + prec)
    n = 400
    chi = np.exp(rng.uniform(np.log(1e-3), np.log(3.0), n))
    gamma = np.exp(rng.uniform(np.log(10), np.log(1e4), n))
    words = W.uniform_words(n, seed=8 + prec)
    words[:4] = [0, 1, 2**32 - 1, 2**32 - 2]
    xg = api.qed_sample_table(ctx, 0, torch.tensor(chi, device="cuda"), torch.tensor(gamma, device="cuda"),
                              torch.tensor(words.view(np.int32), device="cuda")).cpu().numpy()
    r2, c2 = orc.uniform_from_word(words)
    xo = orc.sample_photon(orc.make_config(model=orc.MODEL_CLASSIC), chi, gamma, r2, c2)
    rel = np.abs(xg / xo - 1)
    assert rel.max() <= 1e-5, rel.max()


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
