"""Pins of the oracle in triclinic cells (rows of H are the cell vectors):
an equivalent re-description of an orthorhombic crystal, rigid rotation of
cell and atoms, finite-difference forces and virial in a skewed cell, and MD
wrapping with energy conservation.  CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

MODEL = I.nep_model(1)


def _crystal(n=4, sigma=0.08, seed=71):
    s = I.small_box((n, n, n), sigma=sigma, seed=seed)
    return s.pos, np.diag(s.box)


def test_unimodular_redescription_is_the_same_system():
    """H' = (a, b + a, c + b) generates the same periodic images as
    H = (a, b, c): energy, forces and virial agree with the orthorhombic
    evaluation."""
    pos, H = _crystal()
    H2 = np.array([H[0], H[1] + H[0], H[2] + H[1]])
    E, F, W, U = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)
    E2, F2, W2, U2 = O.energy_forces_virial(MODEL, pos, H2, [1, 1, 1], use_grid=False)
    assert E2 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F, atol=1e-10)
    np.testing.assert_allclose(W2, W, atol=1e-9)
    np.testing.assert_allclose(U2, U, atol=1e-11)


def test_rotation_of_cell_and_atoms():
    """Rotating H and the positions together leaves E unchanged and rotates F
    and W (W' = R W R^T)."""
    pos, H = _crystal(seed=72)
    R = Rotation.random(random_state=73).as_matrix()
    E, F, W, U = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)
    E2, F2, W2, U2 = O.energy_forces_virial(MODEL, pos @ R.T, H @ R.T, [1, 1, 1],
                                            use_grid=False)
    assert E2 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-10)
    np.testing.assert_allclose(W2, R @ W @ R.T, atol=1e-9)


def _skewed(seed=74):
    rng = np.random.default_rng(seed)
    n = 3
    H = np.diag([n * I.A_W] * 3) + rng.uniform(-2.0, 2.0, (3, 3)) * (1 - np.eye(3))
    frac = (I.bcc(n, n, n) / (n * I.A_W)) + rng.normal(0, 0.01, (2 * n ** 3, 3))
    return frac @ H, H


def test_forces_finite_difference_skewed_cell():
    pos, H = _skewed()
    E, F, W, U = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)
    h = 1e-5
    for i in (0, 11, 40):
        for a in range(3):
            p, m = pos.copy(), pos.copy()
            p[i, a] += h
            m[i, a] -= h
            fd = -(O.energy_forces_virial(MODEL, p, H, [1, 1, 1], use_grid=False)[0]
                   - O.energy_forces_virial(MODEL, m, H, [1, 1, 1], use_grid=False)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    np.testing.assert_allclose(F.sum(axis=0), 0, atol=1e-10)


def test_virial_strain_derivative_skewed_cell():
    """W = -dE/d(eps) under the homogeneous strain x -> x (I + eps),
    H -> H (I + eps), for every component."""
    pos, H = _skewed(seed=75)
    E, F, W, U = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)
    h = 1e-6
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3))
            e[a, b] = h
            Ep = O.energy_forces_virial(MODEL, pos @ (np.eye(3) + e), H @ (np.eye(3) + e),
                                        [1, 1, 1], use_grid=False)[0]
            Em = O.energy_forces_virial(MODEL, pos @ (np.eye(3) - e), H @ (np.eye(3) - e),
                                        [1, 1, 1], use_grid=False)[0]
            # x_b' = x_b + sum_a x_a eps_ab: dE/d eps_ab = sum_i x_ia dE/dx_ib = -W_ab
            assert -(Ep - Em) / (2 * h) == pytest.approx(W[a, b], rel=1e-6, abs=1e-6)


def test_md_wraps_into_the_cell_and_conserves_energy():
    pos, H = _skewed(seed=76)
    vel = I.maxwell_boltzmann(np.random.default_rng(77), len(pos), 600.0)
    E0 = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)[0]
    ke0 = 0.5 * I.MASS_W * np.sum(vel ** 2) / I.EV_PER_AMU_A2_FS2
    drift = []
    for dt in (1.0, 0.5):
        p, v, F, th = O.md(MODEL, pos, vel, H, [1, 1, 1], I.MASS_W, dt, int(40 / dt),
                           use_grid=False)
        frac = p @ np.linalg.inv(H)
        assert np.all(frac >= 0) and np.all(frac < 1)
        drift.append(np.max(np.abs(th[:, 2] + th[:, 3] - (E0 + ke0))))
    assert 2.5 < drift[0] / drift[1] < 6.0, drift
    assert drift[1] < 1e-2 * ke0


def test_images_extensivity_small_skewed_cell():
    """A skewed 54-atom cell narrower than 2 r_c replicated 2 x 2 x 2 (cell 2H)
    has 8x the energy and the same per-atom forces: checks that every periodic
    image within the cutoff is enumerated."""
    pos, H = _skewed(seed=78)
    E, F, W, U = O.energy_forces_virial(MODEL, pos, H, [1, 1, 1], use_grid=False)
    reps = [np.array([i, j, k]) for i in range(2) for j in range(2) for k in range(2)]
    big = np.vstack([pos + r @ H for r in reps])
    E8, F8, W8, U8 = O.energy_forces_virial(MODEL, big, 2 * H, [1, 1, 1], use_grid=False)
    assert E8 == pytest.approx(8 * E, rel=1e-11)
    np.testing.assert_allclose(F8[:len(F)], F, atol=1e-9)
