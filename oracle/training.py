"""Training-side oracle: the losses of NEP training and one generation of the
separable natural evolution strategy, in plain numpy over the FP64 oracle's
energies, forces and virials.

TEST INFRASTRUCTURE ONLY (imported by the tests and nothing else).  It reads
the seeded inputs module and ``oracle.oracle``; it shares nothing with the
CUDA library.

What it computes, from the definitions:

* NEP training loss (Sec. III.A; its terms are the curves of Fig. 1(a)):
    L(theta) = lambda_e RMSE_E + lambda_f RMSE_F + lambda_v RMSE_V + L1 + L2,
    RMSE_E = sqrt(mean_s ((E_s - E_s^t) / N_s)^2)            (eV/atom)
    RMSE_F = sqrt(mean over all atoms and x, y, z of (F - F^t)^2)   (eV/A)
    RMSE_V = sqrt(mean over configurations with a virial target and the six
             components xx, yy, zz, yz, zx, xy of ((W_s - W_s^t) / N_s)^2)
    L1 = lambda_1 * (1/P) sum_p |theta_p|,  L2 = lambda_2 * sqrt((1/P) sum_p theta_p^2)
  (the RMSE form and the parameter-averaged regularisers of the NEP
  training the paper uses; Sec. III.A gives lambda_1 = lambda_2 = 0.05,
  lambda_e = lambda_f = 1, lambda_v = 0.1).
* The smooth (mean-square) loss of the gradient path:
    L = w_e mean_s ((dE_s/N_s)^2) + w_f mean(dF^2) + w_v mean_{s in V, c} ((dW_sc/N_s)^2).
* SNES (Schaul et al., 2011, the optimiser Sec. III.A names): with mean mu,
  step sizes sigma and standard-normal samples s_k (k = 1..lambda), the
  candidates theta_k = mu + sigma * s_k are ranked by loss (best first, ties
  by index); rank r gets the utility
    u_r = max(0, ln(lambda/2 + 1) - ln r) / sum_j max(0, ln(lambda/2 + 1) - ln j) - 1/lambda;
  then  g_mu = sum_k u_k s_k,  g_sigma = sum_k u_k (s_k^2 - 1),
        mu <- mu + eta_mu sigma g_mu,  sigma <- sigma exp(eta_sigma / 2 g_sigma),
  with default rates eta_mu = 1, eta_sigma = (3 + ln d) / (5 sqrt d).
  The random samples are inputs, never drawn here.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

# the six virial components, in the order the library stores them
VIRIAL6 = ((0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (0, 1))


def evaluate(model, structs, theta=None):
    """Energies (S,), forces (list of (N_s, 3)) and virials (S, 3, 3)."""
    m = model
    if theta is not None:
        m = I.NepModel(**{k: getattr(model, k) for k in (
            "rc_radial", "rc_angular", "n_max_radial", "n_max_angular", "basis_size_radial",
            "basis_size_angular", "l_max", "use_4body", "n_hidden", "species", "zbl_r_inner",
            "zbl_r_outer")})
        m.params = np.asarray(theta, dtype=np.float64)
        m.scaler = model.scaler
    E, F, W = [], [], []
    for s in structs:
        e, f, w, _ = O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=s.types)
        E.append(e)
        F.append(f)
        W.append(w)
    return np.array(E), F, np.array(W)


def virial6(W):
    """(S, 3, 3) -> (S, 6) in the order xx, yy, zz, yz, zx, xy."""
    W = np.asarray(W)
    return np.stack([W[:, a, b] for a, b in VIRIAL6], axis=1)


def rmse_terms(E, F, W6, Et, Ft, W6t, natoms, has_virial):
    """(RMSE_E, RMSE_F, RMSE_V) as defined above; RMSE_V = 0 without targets."""
    natoms = np.asarray(natoms, dtype=np.float64)
    re = np.sqrt(np.mean(((np.asarray(E) - np.asarray(Et)) / natoms) ** 2))
    dF = np.concatenate(F) - np.concatenate(Ft)
    rf = np.sqrt(np.mean(dF ** 2))
    hv = np.asarray(has_virial, dtype=bool)
    if hv.any():
        dW = (np.asarray(W6) - np.asarray(W6t))[hv] / natoms[hv, None]
        rv = np.sqrt(np.mean(dW ** 2))
    else:
        rv = 0.0
    return re, rf, rv


def regularisers(theta, l1, l2):
    theta = np.asarray(theta, dtype=np.float64)
    return l1 * np.mean(np.abs(theta)), l2 * np.sqrt(np.mean(theta ** 2))


def nep_loss(theta, rmse, weights):
    """Total and terms: dict(total, l1, l2, energy, force, virial)."""
    r1, r2 = regularisers(theta, weights["l1"], weights["l2"])
    re, rf, rv = rmse
    total = weights["energy"] * re + weights["force"] * rf + weights["virial"] * rv + r1 + r2
    return {"total": total, "l1": r1, "l2": r2, "energy": re, "force": rf, "virial": rv}


def mse_loss(E, F, W6, Et, Ft, W6t, natoms, has_virial, we, wf, wv):
    """The smooth loss of the gradient path (terms: energy, force, virial)."""
    natoms = np.asarray(natoms, dtype=np.float64)
    le = we * np.mean(((np.asarray(E) - np.asarray(Et)) / natoms) ** 2)
    lf = wf * np.mean((np.concatenate(F) - np.concatenate(Ft)) ** 2)
    hv = np.asarray(has_virial, dtype=bool)
    lv = 0.0
    if hv.any():
        lv = wv * np.mean(((np.asarray(W6) - np.asarray(W6t))[hv] / natoms[hv, None]) ** 2)
    return le + lf + lv, le, lf, lv


def snes_utilities(n_pop):
    """Utilities of ranks 1..n_pop (best first)."""
    r = np.arange(1, n_pop + 1, dtype=np.float64)
    a = np.maximum(0.0, np.log(n_pop / 2.0 + 1.0) - np.log(r))
    return a / a.sum() - 1.0 / n_pop


def snes_default_rates(d):
    return 1.0, (3.0 + np.log(d)) / (5.0 * np.sqrt(d))


def snes_step(mu, sigma, samples, losses, eta_mu, eta_sigma):
    """One SNES generation given the samples (n_pop, d) and the losses of the
    candidates mu + sigma * samples[k].  Returns (mu', sigma')."""
    samples = np.asarray(samples, dtype=np.float64)
    losses = np.asarray(losses, dtype=np.float64)
    n_pop = len(losses)
    order = np.argsort(losses, kind="stable")      # best first, ties by index
    u = np.empty(n_pop)
    u[order] = snes_utilities(n_pop)
    g_mu = u @ samples
    g_sigma = u @ (samples ** 2 - 1.0)
    return mu + eta_mu * sigma * g_mu, sigma * np.exp(0.5 * eta_sigma * g_sigma)
