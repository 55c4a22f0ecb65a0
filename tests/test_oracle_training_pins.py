"""Pins of the training-side oracle (NEP loss terms and the SNES generation)
against facts fixed by their definitions and by the behaviour the SNES paper
establishes: closed forms, invariances, and convergence on a separable
quadratic.  CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import training as T
from paper_2305_08140_gb300 import inputs as I


def test_utilities_closed_forms():
    # lambda = 2: raw weights (ln 2, 0) -> (1, 0) - 1/2
    np.testing.assert_allclose(T.snes_utilities(2), [0.5, -0.5], atol=1e-15)
    for lam in (4, 10, 50):
        u = T.snes_utilities(lam)
        assert abs(u.sum()) < 1e-14
        assert np.all(np.diff(u) <= 1e-15)                  # non-increasing in rank
        # only ranks r < lambda/2 + 1 get a positive raw weight
        n_pos = int(np.sum(np.arange(1, lam + 1) < lam / 2 + 1))
        assert np.all(u[n_pos:] == pytest.approx(-1.0 / lam))
        assert np.all(u[:n_pos] > -1.0 / lam)


def test_default_rates():
    eta_mu, eta_sigma = T.snes_default_rates(1051)
    assert eta_mu == 1.0
    assert eta_sigma == pytest.approx((3 + math.log(1051)) / (5 * math.sqrt(1051)))


def test_snes_step_depends_only_on_the_ranking():
    rng = np.random.default_rng(1)
    d, lam = 7, 12
    mu, sigma = rng.normal(size=d), rng.uniform(0.1, 1.0, d)
    s = rng.normal(size=(lam, d))
    losses = rng.uniform(0, 5, lam)
    ref = T.snes_step(mu, sigma, s, losses, 1.0, 0.3)
    for f in (lambda x: 3 * x + 7, np.exp, lambda x: x ** 3):
        got = T.snes_step(mu, sigma, s, f(losses), 1.0, 0.3)
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-14)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-14)
    # two candidates: the better one's sample moves mu by sigma * s / 2 towards
    # it and half that away from the other (utilities +1/2, -1/2)
    mu2, _ = T.snes_step(mu, sigma, s[:2], [1.0, 2.0], 1.0, 0.3)
    np.testing.assert_allclose(mu2, mu + sigma * 0.5 * (s[0] - s[1]), rtol=1e-14)


def test_snes_solves_a_separable_quadratic():
    """sNES on f(x) = sum_i c_i (x_i - x*_i)^2 in 10 dimensions: from sigma = 1
    the mean converges to x* and the step sizes shrink (the separable case
    sNES is designed for).  A sign error in either update diverges."""
    d, lam = 10, 10
    rng = np.random.default_rng(3)
    c = np.logspace(0, 2, d)
    xs = rng.uniform(-2, 2, d)
    f = lambda x: np.sum(c * (x - xs) ** 2, axis=-1)
    mu, sigma = np.zeros(d), np.ones(d)
    eta_mu, eta_sigma = T.snes_default_rates(d)
    f0 = f(mu)
    for _ in range(600):
        s = rng.normal(size=(lam, d))
        mu, sigma = T.snes_step(mu, sigma, s, f(mu + sigma * s), eta_mu, eta_sigma)
    assert f(mu) < 1e-8 * f0
    assert np.all(sigma < 1e-3)


def test_rmse_terms_closed_forms():
    rng = np.random.default_rng(5)
    natoms = np.array([54, 128, 250])
    Et = rng.normal(size=3)
    Ft = [rng.normal(size=(n, 3)) for n in natoms]
    W6t = rng.normal(size=(3, 6))
    hv = np.array([1, 0, 1])
    # exact predictions: every term is zero
    assert T.rmse_terms(Et, Ft, W6t, Et, Ft, W6t, natoms, hv) == (0.0, 0.0, 0.0)
    # a uniform per-atom energy offset delta gives RMSE_E = |delta|
    re, _, _ = T.rmse_terms(Et + 0.003 * natoms, Ft, W6t, Et, Ft, W6t, natoms, hv)
    assert re == pytest.approx(0.003, rel=1e-12)
    # every force component off by the same amount
    _, rf, _ = T.rmse_terms(Et, [f + 0.02 for f in Ft], W6t, Et, Ft, W6t, natoms, hv)
    assert rf == pytest.approx(0.02, rel=1e-12)
    # configurations without a virial target do not count
    W6 = W6t.copy()
    W6[1] += 1e3
    assert T.rmse_terms(Et, Ft, W6, Et, Ft, W6t, natoms, hv)[2] == 0.0
    W6[0] += 0.5 * natoms[0]
    _, _, rv = T.rmse_terms(Et, Ft, W6, Et, Ft, W6t, natoms, hv)
    assert rv == pytest.approx(0.5 / math.sqrt(2), rel=1e-12)   # one of two configs, all 6
    # order of the configurations does not matter
    p = [2, 0, 1]
    got = T.rmse_terms(Et[p] + 0.1, [Ft[i] for i in p], W6[p], Et[p], [Ft[i] for i in p], W6t[p],
                       natoms[p], hv[p])
    ref = T.rmse_terms(Et + 0.1, Ft, W6, Et, Ft, W6t, natoms, hv)
    np.testing.assert_allclose(got, ref, rtol=1e-14)


def test_regularisers_closed_forms():
    theta = np.full(1051, -0.3)
    r1, r2 = T.regularisers(theta, 0.05, 0.05)
    assert r1 == pytest.approx(0.05 * 0.3, rel=1e-14)
    assert r2 == pytest.approx(0.05 * 0.3, rel=1e-14)
    theta = np.array([3.0, 4.0])
    assert T.regularisers(theta, 1.0, 1.0) == pytest.approx((3.5, math.sqrt(12.5)))


def test_virial6_of_the_oracle_is_symmetric_and_ordered():
    """The oracle's virial of a strained periodic box is symmetric, so the six
    stored components hold all of it; order xx, yy, zz, yz, zx, xy."""
    s = I.small_box((4, 4, 4), sigma=0.1, seed=9)
    E, F, W = T.evaluate(I.nep_model(1), [s])
    np.testing.assert_allclose(W[0], W[0].T, atol=1e-9)
    w6 = T.virial6(W)[0]
    assert w6[0] == W[0][0, 0] and w6[3] == W[0][1, 2] and w6[4] == W[0][2, 0]
    assert w6[5] == W[0][0, 1]


def test_evaluate_with_theta_matches_model():
    m = I.nep_model(1)
    s = I.small_box((3, 3, 3), sigma=0.1, seed=10)
    theta = m.params * 0.9
    E, F, W = T.evaluate(m, [s], theta)
    m2 = I.nep_model(1)
    m2.params = theta
    e2, f2, w2, _ = O.energy_forces_virial(m2, s.pos, s.box, s.pbc)
    assert E[0] == e2
    np.testing.assert_array_equal(F[0], f2)
