"""Pins of the FP64 oracle's multi-species form (coefficients c^{t_i t_j} per
ordered species pair; Z_i, Z_j of the pair in Eq. 2 and 4; a mass per
species) against facts that hold by construction: reduction to one species,
an ordered crystal whose sites see a single species pair, independent
sub-lattices when the cross-species coefficients vanish, relabelling of the
species, the Coulomb limit of the mixed-Z pair term, finite differences, and
conservation of momentum and energy in NVE.  CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

W_MODEL = I.nep_model(1)


def _blocks(model):
    """(w0 b0 w1 b1) head, cR[T][T][nR][KR], cA[T][T][nA][KA] of a model."""
    T = model.n_types
    nR, KR = model.n_max_radial + 1, model.basis_size_radial + 1
    nA, KA = model.n_max_angular + 1, model.basis_size_angular + 1
    head = model.n_hidden * model.dim + 2 * model.n_hidden + 1
    p = model.params
    cR = p[head:head + T * T * nR * KR].reshape(T, T, nR, KR)
    cA = p[head + T * T * nR * KR:].reshape(T, T, nA, KA)
    return p[:head], cR, cA


def _assemble(species, head, cR, cA, scaler, **hyper):
    m = I.NepModel(species=tuple(species), **hyper)
    m.params = np.concatenate([head, np.asarray(cR).ravel(), np.asarray(cA).ravel()])
    assert len(m.params) == m.n_params
    m.scaler = scaler
    return m


def _random_species_model(species, seed, **hyper):
    """Random blocks (each its own draw) on the W model's network and scaler."""
    head, cR1, cA1 = _blocks(W_MODEL)
    T = len(species)
    rng = np.random.default_rng(seed)
    cR = rng.uniform(-0.5, 0.5, (T, T) + cR1.shape[2:])
    cA = rng.uniform(-0.5, 0.5, (T, T) + cA1.shape[2:])
    return _assemble(species, head, cR, cA, W_MODEL.scaler, **hyper)


def test_parameter_count_and_layout():
    m = I.nep_model(301, species=("W", "Mo"))
    assert m.n_params == 30 * 30 + 61 + 4 * (45 + 45)
    m4 = I.nep_model(401, species=("W", "Mo", "Ta", "Nb"))
    assert m4.n_params == 30 * 30 + 61 + 16 * 90
    assert m4.zs == [74, 42, 73, 41]


def test_identical_blocks_reduce_to_one_species():
    """T = 2 with every block equal to the W model's and Z = 74 for both
    species gives the one-species result for any labelling."""
    head, cR1, cA1 = _blocks(W_MODEL)
    m2 = _assemble(("W", "W"), head, np.tile(cR1, (2, 2, 1, 1)), np.tile(cA1, (2, 2, 1, 1)),
                   W_MODEL.scaler)
    s = I.alloy(I.small_box((4, 4, 4), sigma=0.1, seed=31), [0.5, 0.5], seed=32)
    s.pos[3] = s.pos[0] + np.array([0.7, 0.6, 0.5])     # a ZBL pair of mixed labels
    E1, F1, W1, U1 = O.energy_forces_virial(W_MODEL, s.pos, s.box, s.pbc)
    E2, F2, W2, U2 = O.energy_forces_virial(m2, s.pos, s.box, s.pbc, types=s.types)
    assert E2 == pytest.approx(E1, rel=1e-13, abs=1e-12)
    np.testing.assert_allclose(F2, F1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(W2, W1, rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(U2, U1, rtol=1e-12, atol=1e-12)


def test_b2_sites_see_one_ordered_pair():
    """With r_c = 3.0 A only the first bcc shell (8 atoms at sqrt(3) a / 2 =
    2.74 A) is inside the cutoffs.  In the B2 (CsCl) crystal those 8 are all of
    the other species, so a species-0 site has exactly the energy of a pure bcc
    site whose coefficients are the block (centre 0, neighbour 1), and a
    species-1 site that of the block (1, 0).  Blocks (0, 0) and (1, 1) must not
    enter at all."""
    hyper = dict(rc_radial=3.0, rc_angular=3.0)
    m2 = _random_species_model(("W", "Mo"), 41, **hyper)
    head, cR, cA = _blocks(m2)
    s = I.b2(4)
    E, F, W, U = O.energy_forces_virial(m2, s.pos, s.box, s.pbc, types=s.types)
    pure = I.small_box((4, 4, 4))
    for centre, other in ((0, 1), (1, 0)):
        m1 = _assemble(("W",), head, cR[centre, other][None, None], cA[centre, other][None, None],
                       W_MODEL.scaler, **hyper)
        _, _, _, U1 = O.energy_forces_virial(m1, pure.pos, pure.box, pure.pbc)
        np.testing.assert_allclose(U[s.types == centre], U1[0], rtol=1e-12)
    # the diagonal blocks are inert here
    cR2, cA2 = cR.copy(), cA.copy()
    cR2[0, 0] = cR2[1, 1] = 0.0
    cA2[0, 0] = cA2[1, 1] = 0.0
    m3 = _assemble(("W", "Mo"), head, cR2, cA2, W_MODEL.scaler, **hyper)
    E3 = O.energy_forces_virial(m3, s.pos, s.box, s.pbc, types=s.types)[0]
    assert E3 == pytest.approx(E, rel=1e-13)
    assert np.max(np.abs(F)) < 1e-11


def test_zero_cross_blocks_give_independent_sublattices():
    """With c^{01} = c^{10} = 0 and no pair inside the ZBL range, the species
    interact only with their own kind: the energy is the sum of the two
    sub-lattices computed alone (one-species models with blocks (0, 0) and
    (1, 1)), and so are the forces."""
    m2 = _random_species_model(("W", "Mo"), 51)
    head, cR, cA = _blocks(m2)
    cR[0, 1] = cR[1, 0] = 0.0
    cA[0, 1] = cA[1, 0] = 0.0
    m2 = _assemble(("W", "Mo"), head, cR, cA, W_MODEL.scaler)
    s = I.alloy(I.small_box((6, 6, 6), sigma=0.05, seed=52), [0.4, 0.6], seed=53)
    E, F, W, U = O.energy_forces_virial(m2, s.pos, s.box, s.pbc, types=s.types)
    Esum = 0.0
    for t in (0, 1):
        sel = s.types == t
        m1 = _assemble(("W",), head, cR[t, t][None, None], cA[t, t][None, None], W_MODEL.scaler)
        Et, Ft, Wt, Ut = O.energy_forces_virial(m1, s.pos[sel], s.box, s.pbc)
        Esum += Et
        np.testing.assert_allclose(F[sel], Ft, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(U[sel], Ut, rtol=1e-12)
    assert E == pytest.approx(Esum, rel=1e-13)


def test_relabelling_species_is_a_symmetry():
    """Swapping the labels of the atoms together with the coefficient blocks,
    Z and masses leaves energy, forces and virial unchanged."""
    m = _random_species_model(("W", "Mo"), 61)
    head, cR, cA = _blocks(m)
    sw = _assemble(("Mo", "W"), head, cR[::-1, ::-1], cA[::-1, ::-1], W_MODEL.scaler)
    s = I.alloy(I.small_box((4, 4, 4), sigma=0.12, seed=62), [0.5, 0.5], seed=63)
    s.pos[5] = s.pos[9] + np.array([0.5, -0.6, 0.4])
    E, F, W, U = O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=s.types)
    E2, F2, W2, U2 = O.energy_forces_virial(sw, s.pos, s.box, s.pbc, types=1 - s.types)
    assert E2 == pytest.approx(E, rel=1e-13)
    np.testing.assert_allclose(F2, F, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(W2, W, rtol=1e-11, atol=1e-11)


def test_mixed_dimer_is_the_mixed_zbl_term():
    """With every NEP coefficient zero the network sees q = 0 at every atom, so
    the separation dependence of a W-Mo dimer is the ZBL pair term of Z = 74
    and 42 alone; as r -> 0, r U -> k Z_i Z_j phi(0) (Coulomb limit, Eq. 2-3),
    42/74 of the W-W value."""
    m = _random_species_model(("W", "Mo"), 71)
    head, cR, cA = _blocks(m)
    m0 = _assemble(("W", "Mo"), head, 0 * cR, 0 * cA, W_MODEL.scaler)
    box = np.array([40.0, 40, 40])
    far = np.array([[5.0, 5, 5], [25.0, 25, 25]])
    Einf = O.energy_forces_virial(m0, far, box, [0, 0, 0], types=[0, 1])[0]
    for r in (0.4, 1.0, 1.5, 1.9):
        pos = np.array([[10.0, 10, 10], [10.0 + r, 10, 10]])
        E, F, _, _ = O.energy_forces_virial(m0, pos, box, [0, 0, 0], types=[0, 1])
        u, du = O.zbl(r, 74.0, 42.0)
        assert E - Einf == pytest.approx(u, rel=1e-12)
        np.testing.assert_allclose(F[1], [-du, 0, 0], rtol=1e-12)
    k = 14.39964547
    phi0 = 0.32825 + 0.09219 + 0.58110
    r = 1e-6
    assert r * O.zbl(r, 74.0, 42.0)[0] == pytest.approx(k * 74 * 42 * phi0, rel=1e-4)
    assert O.zbl(r, 74.0, 42.0)[0] / O.zbl(r, 74.0, 74.0)[0] == pytest.approx(42 / 74, rel=1e-4)


def test_forces_finite_difference_four_species():
    """Random W-Mo-Ta-Nb box with a close pair of unlike species: F = -dE/dx."""
    m = _random_species_model(("W", "Mo", "Ta", "Nb"), 81)
    s = I.alloy(I.small_box((3, 3, 3), a=3.23, sigma=0.12, seed=82), [0.25] * 4, seed=83)
    s.pos[1] = s.pos[0] + np.array([0.6, 0.5, 0.45])
    assert s.types[0] != s.types[1]
    E, F, W, U = O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=s.types, use_grid=False)
    h = 1e-6
    for i in (0, 1, 13):
        for a in range(3):
            p, q = s.pos.copy(), s.pos.copy()
            p[i, a] += h
            q[i, a] -= h
            fd = -(O.energy_forces_virial(m, p, s.box, s.pbc, types=s.types, use_grid=False)[0]
                   - O.energy_forces_virial(m, q, s.box, s.pbc, types=s.types,
                                            use_grid=False)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    np.testing.assert_allclose(F.sum(axis=0), 0, atol=1e-9)


def test_site_gradient_finite_difference_mixed_neighbours():
    m = _random_species_model(("W", "Mo", "Ta"), 91)
    rng = np.random.default_rng(92)
    u = rng.normal(size=(7, 3))
    d = u / np.linalg.norm(u, axis=1, keepdims=True) * rng.uniform(1.5, 3.9, 7)[:, None]
    tn = rng.integers(0, 3, 7)
    U, q, gR, gA = O.site(m, d, d, ti=2, tR=tn, tA=tn)
    h = 1e-6
    for sidx in (0, 3, 6):
        for a in range(3):
            dp, dm = d.copy(), d.copy()
            dp[sidx, a] += h
            dm[sidx, a] -= h
            fd = (O.site(m, dp, dp, 2, tn, tn)[0] - O.site(m, dm, dm, 2, tn, tn)[0]) / (2 * h)
            assert gR[sidx, a] + gA[sidx, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # the centre's species selects the blocks: another centre species changes U
    assert abs(O.site(m, d, d, 0, tn, tn)[0] - U) > 1e-6


def test_nve_two_masses_conserves_momentum_and_energy():
    """W-Mo NVE with per-species masses: total momentum sum m_i v_i stays zero
    (Newton's third law, exact up to rounding) and the total energy drift
    shrinks as dt^2; using one mass for both species would break both."""
    m = I.nep_model(301, species=("W", "Mo"))
    s = I.alloy(I.small_box((3, 3, 3), sigma=0.05, seed=101), [0.5, 0.5], seed=102)
    masses = np.array(m.masses)[s.types]
    s.vel = I.maxwell_boltzmann(np.random.default_rng(103), s.n, 600.0, masses)
    p0 = (masses[:, None] * s.vel).sum(axis=0)
    assert np.max(np.abs(p0)) < 1e-12
    drift = []
    ke0 = 0.5 * np.sum(masses[:, None] * s.vel ** 2) / I.EV_PER_AMU_A2_FS2
    E0 = O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=s.types, use_grid=False)[0]
    for dt in (1.0, 0.5):
        n = int(round(30 / dt))
        p, v, F, th = O.md(m, s.pos, s.vel, s.box, s.pbc, m.masses, dt, n, types=s.types,
                           use_grid=False)
        mom = (masses[:, None] * v).sum(axis=0)
        assert np.max(np.abs(mom)) < 1e-10 * np.sum(masses) * np.max(np.abs(s.vel))
        drift.append(np.max(np.abs(th[:, 2] + th[:, 3] - (E0 + ke0))))
    assert 2.5 < drift[0] / drift[1] < 6.0, drift
    assert drift[1] < 1e-2 * ke0


def test_species_out_of_range_is_rejected():
    m = I.nep_model(301, species=("W", "Mo"))
    s = I.small_box((3, 3, 3))
    t = np.zeros(s.n, np.int32)
    t[4] = 2
    with pytest.raises(RuntimeError):
        O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=t)
    t[4] = -1
    with pytest.raises(RuntimeError):
        O.energy_forces_virial(m, s.pos, s.box, s.pbc, types=t)
