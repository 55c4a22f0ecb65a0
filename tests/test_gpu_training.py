"""GPU parity of the training path the paper uses (Sec. III.A): the NEP loss
(RMSE energy, force and virial terms, L1 and L2 regularisers) of a whole SNES
population in one launch, and the SNES generation (candidates, ranking,
utilities, mean and step-size update), against the training-side oracle."""
import numpy as np
import pytest

from oracle import training as T
from paper_2305_08140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WEIGHTS = {"energy": 1.0, "force": 1.0, "virial": 0.1, "l1": 0.05, "l2": 0.05}


def _setup(n_configs=6, seed=41, max_atoms=128):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs = [s for s in I.c4(64, seed=seed) if s.n <= max_atoms][:n_configs]
    Et, Ft, Wt = T.evaluate(I.nep_model(101), structs)
    W6t = T.virial6(Wt)
    hv = np.ones(len(structs), np.uint8)
    hv[1::3] = 0
    dev = dict(dtype=torch.float64, device="cuda")
    targets = (torch.tensor(Et, **dev), torch.tensor(np.concatenate(Ft).T.copy(), **dev),
               torch.tensor(W6t, **dev), hv)
    return structs, (Et, Ft, W6t, hv), targets, N.Batch(structs)


def _oracle_losses(model, structs, thetas, tg):
    Et, Ft, W6t, hv = tg
    N = [s.n for s in structs]
    out = []
    for th in thetas:
        E, F, W = T.evaluate(model, structs, th)
        r = T.rmse_terms(E, F, T.virial6(W), Et, Ft, W6t, N, hv)
        d = T.nep_loss(th, r, WEIGHTS)
        out.append([d[k] for k in ("total", "l1", "l2", "energy", "force", "virial")])
    return np.array(out)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_population_loss_matches_oracle(precision):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs, tg, (Etd, Ftd, Wtd, hv), b = _setup()
    model = I.nep_model(1)
    rng = np.random.default_rng(42)
    thetas = model.params[None, :] + 0.05 * rng.normal(size=(5, model.n_params))
    nep = N.NEP(model, precision)
    L = N.population_loss(nep, b, torch.tensor(thetas, device="cuda"), Etd, Ftd, Wtd, hv,
                          WEIGHTS).cpu().numpy()
    Lo = _oracle_losses(model, structs, thetas, tg)
    rel = 1e-10 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(L, Lo, rtol=rel, atol=1e-12)
    # the same numbers whatever else runs: the population's first member
    # evaluated alone
    L1 = N.population_loss(nep, b, torch.tensor(thetas[:1], device="cuda"), Etd, Ftd, Wtd, hv,
                           WEIGHTS).cpu().numpy()
    np.testing.assert_allclose(L1[0], L[0], rtol=1e-13)
    nep.close()


def test_population_loss_without_virial_targets_and_large_population():
    """No virial targets: RMSE_V = 0; a population of 64 over 12 configurations
    (768 work items) agrees with the oracle on a sample of its members."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs, (Et, Ft, W6t, hv), (Etd, Ftd, _, _), b = _setup(n_configs=12, seed=43)
    model = I.nep_model(1)
    rng = np.random.default_rng(44)
    thetas = model.params[None, :] + 0.1 * rng.normal(size=(64, model.n_params))
    nep = N.NEP(model, "fp32")
    L = N.population_loss(nep, b, torch.tensor(thetas, device="cuda"), Etd, Ftd, None, None,
                          WEIGHTS).cpu().numpy()
    assert np.all(L[:, 5] == 0.0)
    pick = [0, 17, 63]
    Lo = _oracle_losses(model, structs, thetas[pick], (Et, Ft, W6t, np.zeros(len(structs))))
    np.testing.assert_allclose(L[pick], Lo, rtol=2e-5, atol=1e-12)
    nep.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_snes_generation_matches_oracle(precision):
    """One generation from mu = the seed-1 parameters, sigma = 0.02: the
    GPU's candidate losses equal the oracle's, and mu', sigma' equal the
    oracle's SNES step applied to the oracle's losses (the ranking is
    unambiguous: checked)."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs, tg, (Etd, Ftd, Wtd, hv), b = _setup(n_configs=4, seed=45)
    model = I.nep_model(1)
    d = model.n_params
    n_pop = 8
    rng = np.random.default_rng(46)
    samples = rng.normal(size=(n_pop, d))
    mu0 = model.params.copy()
    sigma0 = np.full(d, 0.02)
    nep = N.NEP(model, precision)
    mu = torch.tensor(mu0, device="cuda")
    sigma = torch.tensor(sigma0, device="cuda")
    eta_mu, eta_sigma = T.snes_default_rates(d)
    L = N.snes_generation(nep, b, mu, sigma, torch.tensor(samples, device="cuda"), Etd, Ftd, Wtd,
                          hv, WEIGHTS, eta_mu, eta_sigma).cpu().numpy()
    Lo = _oracle_losses(model, structs, mu0[None, :] + sigma0[None, :] * samples, tg)
    rel = 1e-10 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(L, Lo, rtol=rel, atol=1e-12)
    srt = np.sort(Lo[:, 0])
    assert np.min(np.diff(srt)) > 1e-3 * srt[0]          # unambiguous ranking
    mu1, sigma1 = T.snes_step(mu0, sigma0, samples, Lo[:, 0], eta_mu, eta_sigma)
    np.testing.assert_allclose(mu.cpu().numpy(), mu1, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(sigma.cpu().numpy(), sigma1, rtol=1e-13)
    nep.close()


def test_snes_reduces_the_loss():
    """Twenty generations of SNES on the GPU (samples from a seeded host
    generator) lower the training loss of the mean; the run is deterministic."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs, tg, (Etd, Ftd, Wtd, hv), b = _setup(n_configs=6, seed=47)
    model = I.nep_model(1)
    d = model.n_params
    nep = N.NEP(model, "fp32")
    runs = []
    for _ in range(2):
        rng = np.random.default_rng(48)
        mu = torch.tensor(model.params, device="cuda")
        sigma = torch.full((d,), 0.05, dtype=torch.float64, device="cuda")
        L0 = N.population_loss(nep, b, mu[None, :], Etd, Ftd, Wtd, hv, WEIGHTS)[0, 0].item()
        for _ in range(20):
            s = torch.tensor(rng.normal(size=(16, d)), device="cuda")
            N.snes_generation(nep, b, mu, sigma, s, Etd, Ftd, Wtd, hv, WEIGHTS)
        L1 = N.population_loss(nep, b, mu[None, :], Etd, Ftd, Wtd, hv, WEIGHTS)[0, 0].item()
        runs.append((L0, L1, mu.cpu().numpy()))
    assert runs[0][1] < 0.9 * runs[0][0], runs[0][:2]
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
    nep.close()


def test_population_argument_errors():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs, tg, (Etd, Ftd, Wtd, hv), b = _setup(n_configs=2, seed=49)
    nep = N.NEP(I.nep_model(1), "fp32")
    th = torch.zeros((1025, 1051), dtype=torch.float64, device="cuda")
    with pytest.raises(N.NepError):
        N.population_loss(nep, b, th, Etd, Ftd)
    with pytest.raises(N.NepError):
        N.population_loss(nep, b, th[:2].cpu(), Etd, Ftd)      # host memory
    nep.close()
