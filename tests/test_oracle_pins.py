"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, independent library routines, invariances, finite differences,
brute force).  CPU only."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

MODEL = I.nep_model(1)


def _rng(seed=0):
    return np.random.default_rng(seed)


# --- one-dimensional building blocks -----------------------------------------

def test_cutoff_closed_form():
    rc = 6.0
    assert O.cutoff(0.0, rc)[0] == pytest.approx(1.0, abs=1e-15)
    assert O.cutoff(rc / 2, rc)[0] == pytest.approx(0.5, abs=1e-15)
    assert O.cutoff(rc, rc) == (0.0, 0.0)
    assert O.cutoff(7.0, rc) == (0.0, 0.0)
    # C1 at rc: value and slope vanish from below
    fc, dfc = O.cutoff(rc - 1e-7, rc)
    assert abs(fc) < 1e-12 and abs(dfc) < 1e-6
    for r in (0.3, 1.7, 3.3, 5.9):
        h = 1e-6
        fd = (O.cutoff(r + h, rc)[0] - O.cutoff(r - h, rc)[0]) / (2 * h)
        assert O.cutoff(r, rc)[1] == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_chebyshev_is_cos_k_theta():
    for theta in np.linspace(0.05, math.pi - 0.05, 11):
        T, dT = O.chebyshev(math.cos(theta), 9)
        for k in range(9):
            assert T[k] == pytest.approx(math.cos(k * theta), abs=1e-13)
            # dT_k/dx = k sin(k theta) / sin(theta)
            assert dT[k] == pytest.approx(k * math.sin(k * theta) / math.sin(theta), abs=1e-11)


def test_basis_special_points():
    rc, K = 4.0, 9
    f, _ = O.basis(0.0, rc, K)          # x = 1: T_k(1) = 1, f_c(0) = 1
    np.testing.assert_allclose(f, np.ones(K), atol=1e-15)
    r0 = rc * (1 - 1 / math.sqrt(2))    # x = 0: T_k(0) = cos(k pi / 2)
    f, _ = O.basis(r0, rc, K)
    fc = O.cutoff(r0, rc)[0]
    np.testing.assert_allclose(f, [0.5 * (math.cos(k * math.pi / 2) + 1) * fc for k in range(K)],
                               atol=1e-14)
    f, df = O.basis(rc, rc, K)
    assert np.all(f == 0) and np.all(df == 0)
    for r in (0.7, 2.2, 3.9):
        h = 1e-6
        fd = (O.basis(r + h, rc, K)[0] - O.basis(r - h, rc, K)[0]) / (2 * h)
        np.testing.assert_allclose(O.basis(r, rc, K)[1], fd, rtol=1e-6, atol=1e-9)


def test_legendre_matches_numpy():
    for x in np.linspace(-1, 1, 17):
        P, dP = O.legendre(x, 6)
        for l in range(7):
            c = np.zeros(l + 1)
            c[l] = 1
            assert P[l] == pytest.approx(npleg.legval(x, c), abs=1e-14)
            assert dP[l] == pytest.approx(npleg.legval(x, npleg.legder(c)), abs=1e-12)


# --- ZBL (Eq. 2-4) -----------------------------------------------------------

def _coulomb_ev_angstrom():
    e = 1.602176634e-19
    eps0 = 8.8541878128e-12
    return e * e / (4 * math.pi * eps0) / e * 1e10   # J m -> eV A


def test_zbl_small_r_limit_and_screening_length():
    """r U(r) -> k Z^2 phi(0) with phi(0) the sum of the printed coefficients
    (Eq. 3), and its slope at 0 is -k Z^2 sum(c_i b_i)/a with a of Eq. 4."""
    Z = 74.0
    k = _coulomb_ev_angstrom() * Z * Z
    phi0 = 0.32825 + 0.09219 + 0.58110
    cb = 0.32825 * 2.54931 + 0.09219 * 0.29182 + 0.58110 * 0.59231
    a = 0.46848 / (2 * Z ** 0.23)
    r1, r2 = 1e-6, 2e-6
    y1 = r1 * O.zbl(r1, Z, Z)[0] / k
    y2 = r2 * O.zbl(r2, Z, Z)[0] / k
    assert y1 == pytest.approx(phi0, rel=1e-4)
    slope = (y2 - y1) / (r2 - r1)
    assert slope == pytest.approx(-cb / a, rel=1e-3)


def test_zbl_tersoff_switch():
    """Switch is 1 below 1 A, (1 + cos(pi (r-1)))/2 between 1 and 2 A, 0 above
    (Sec. II.A): compare with the same pair term with the switch moved away."""
    Z = 74.0
    for r, s in ((0.5, 1.0), (1.0, 1.0), (1.25, 0.5 + 0.5 * math.cos(math.pi / 4)),
                 (1.5, 0.5), (1.75, 0.5 + 0.5 * math.cos(3 * math.pi / 4))):
        u_sw = O.zbl(r, Z, Z, 1.0, 2.0)[0]
        u_free = O.zbl(r, Z, Z, 10.0, 11.0)[0]
        assert u_sw / u_free == pytest.approx(s, rel=1e-12)
    assert O.zbl(2.0, Z, Z) == (0.0, 0.0)
    assert O.zbl(2.741, Z, Z) == (0.0, 0.0)   # bcc W nearest neighbour
    # C1 at both switch radii
    for rs in (1.0, 2.0):
        dl = O.zbl(rs - 1e-7, Z, Z)[1]
        dr = O.zbl(rs + 1e-7, Z, Z)[1]
        assert dl == pytest.approx(dr, rel=1e-4, abs=1e-4)
    for r in (0.3, 0.8, 1.2, 1.6, 1.95):
        h = 1e-7
        fd = (O.zbl(r + h, Z, Z)[0] - O.zbl(r - h, Z, Z)[0]) / (2 * h)
        assert O.zbl(r, Z, Z)[1] == pytest.approx(fd, rel=1e-6)


def test_dimer_energy_is_zbl_pair_term():
    """With the NEP network switched off (all weights zero) a dimer's energy is
    one ZBL pair term (the 1/2 of Eq. 1 counts each pair once), and the force
    is -dU_ZBL/dr along the bond."""
    m = I.nep_model(1)
    m.params = np.zeros_like(m.params)
    for r in (0.4, 1.0, 1.5, 1.9):
        pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        E, F, W, U = O.energy_forces_virial(m, pos, np.array([30.0, 30, 30]), [0, 0, 0],
                                            use_grid=False)
        u, du = O.zbl(r)
        assert E == pytest.approx(u, rel=1e-12)
        np.testing.assert_allclose(U, [u / 2, u / 2], rtol=1e-12)
        np.testing.assert_allclose(F[1], [-du, 0, 0], rtol=1e-12)
        np.testing.assert_allclose(F[0], [du, 0, 0], rtol=1e-12)


# --- descriptor ----------------------------------------------------------------

def _random_env(n, rmin=1.2, rmax=3.95, seed=0):
    rng = _rng(seed)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = rng.uniform(rmin, rmax, n)
    return u * r[:, None]


def _gA(model, r):
    nA, KA = model.n_max_angular + 1, model.basis_size_angular + 1
    H, D = model.n_hidden, model.dim
    off = H * D + 2 * H + 1 + (model.n_max_radial + 1) * (model.basis_size_radial + 1)
    cA = model.params[off:off + nA * KA].reshape(nA, KA)
    return np.array([cA @ O.basis(x, model.rc_angular, KA)[0] for x in r])  # (M, nA)


def test_angular_descriptor_addition_theorem_scipy():
    """q_nl (Legendre double sum) equals 4 pi/(2l+1) sum_m |sum_j g_n Y_lm|^2
    with scipy's spherical harmonics."""
    from scipy import special
    d = _random_env(9)
    U, q, _, _ = O.site(MODEL, d, d)
    r = np.linalg.norm(d, axis=1)
    g = _gA(MODEL, r)
    theta = np.arccos(d[:, 2] / r)
    phi = np.arctan2(d[:, 1], d[:, 0])
    nR, nA = 5, 5
    for l in range(1, 5):
        for n in range(nA):
            tot = 0.0
            for mm in range(-l, l + 1):
                if hasattr(special, "sph_harm_y"):
                    Y = special.sph_harm_y(l, mm, theta, phi)
                else:
                    Y = special.sph_harm(mm, l, phi, theta)
                tot += abs(np.sum(g[:, n] * Y)) ** 2
            tot *= 4 * math.pi / (2 * l + 1)
            assert q[nR + (l - 1) * nA + n] == pytest.approx(tot, rel=1e-11, abs=1e-14)


def test_angular_l1_l2_closed_forms_and_fourbody():
    d = _random_env(11, seed=3)
    U, q, _, _ = O.site(MODEL, d, d)
    r = np.linalg.norm(d, axis=1)
    u = d / r[:, None]
    g = _gA(MODEL, r)
    nR, nA = 5, 5
    for n in range(nA):
        v = (g[:, n, None] * u).sum(axis=0)
        assert q[nR + n] == pytest.approx(v @ v, rel=1e-12)                 # l = 1
        T = np.einsum("j,ja,jb->ab", g[:, n], u, u) - g[:, n].sum() * np.eye(3) / 3
        assert q[nR + nA + n] == pytest.approx(1.5 * np.trace(T @ T), rel=1e-12)  # l = 2
        q4 = q[nR + 4 * nA + n]
        assert q4 == pytest.approx(3 * np.linalg.det(T), rel=1e-10, abs=1e-15)
        assert q4 == pytest.approx(O.fourbody_triple(g[:, n], u), rel=1e-10, abs=1e-15)


def test_radial_descriptor_single_neighbour():
    nR, KR = 5, 9
    H, D = MODEL.n_hidden, MODEL.dim
    cR = MODEL.params[H * D + 2 * H + 1:H * D + 2 * H + 1 + nR * KR].reshape(nR, KR)
    for r in (2.0, 3.5, 5.5):
        _, q, _, _ = O.site(MODEL, [[0, 0, r]], np.zeros((0, 3)))
        f = O.basis(r, 6.0, KR)[0]
        np.testing.assert_allclose(q[:nR], cR @ f, rtol=1e-13)
        # the angular part is empty without angular neighbours
        assert np.all(q[nR:] == 0)


def test_network_matches_numpy():
    d = _random_env(12, seed=5)
    dR = np.vstack([d, _random_env(30, 4.0, 5.99, seed=6)])
    U, q, _, _ = O.site(MODEL, dR, d)
    H, D = MODEL.n_hidden, MODEL.dim
    p = MODEL.params
    w0 = p[:H * D].reshape(H, D)
    b0 = p[H * D:H * D + H]
    w1 = p[H * D + H:H * D + 2 * H]
    b1 = p[H * D + 2 * H]
    ref = w1 @ np.tanh(w0 @ (MODEL.scaler * q) - b0) - b1
    assert U == pytest.approx(ref, rel=1e-13)


def test_network_special_weights_dimer_closed_form():
    """A network that reads only the radial descriptor: w0[mu, nu(mu)] = a_mu
    with nu(mu) = (mu + 2) mod n_R for the first n_R neurons and 0 elsewhere,
    so the site energy of each atom of a dimer at r (outside the ZBL range,
    one neighbour) is sum_mu w1_mu tanh(a_mu s_nu q_nu(r) - b0_mu)
    + sum_rest w1 tanh(-b0) - b1
    with q(r) = c_R f(r) (the pinned radial basis).  E = 2 U_site, U_site per
    atom, and F = -dE/dr (central differences of that closed form).  Catches a
    missing descriptor scaler, a sign of b0 or b1, a transposed w0."""
    H, D = MODEL.n_hidden, MODEL.dim
    nR, KR = 5, 9
    p = MODEL.params.copy()
    w0 = np.zeros((H, D))
    a = np.array([0.7, -1.3, 0.4, 2.1, -0.9])
    nu = (np.arange(nR) + 2) % nR
    for mu in range(nR):
        w0[mu, nu[mu]] = a[mu]
    b0 = np.linspace(-0.6, 0.8, H)
    w1 = np.linspace(0.9, -0.5, H)
    b1 = 0.37
    p[:H * D] = w0.ravel()
    p[H * D:H * D + H] = b0
    p[H * D + H:H * D + 2 * H] = w1
    p[H * D + 2 * H] = b1
    cR = p[H * D + 2 * H + 1:H * D + 2 * H + 1 + nR * KR].reshape(nR, KR)
    s = np.asarray(MODEL.scaler)

    def U_closed(r):
        q = cR @ O.basis(r, 6.0, KR)[0]
        h = -b0.copy()
        h[:nR] += a * s[nu] * q[nu]
        return float(w1 @ np.tanh(h) - b1)

    box = [40.0, 40.0, 40.0]
    for r in (2.6, 3.7, 5.2):
        pos = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0 + r]])
        E, F, W, U = O.energy_forces_virial(MODEL, pos, box, [0, 0, 0], params=p)
        u = U_closed(r)
        np.testing.assert_allclose(U, [u, u], rtol=1e-12, atol=1e-12)
        assert E == pytest.approx(2 * u, rel=1e-12, abs=1e-12)
        h = 1e-5
        dEdr = 2 * (U_closed(r + h) - U_closed(r - h)) / (2 * h)
        np.testing.assert_allclose(F[1], [0.0, 0.0, -dEdr], atol=1e-7)
        np.testing.assert_allclose(F[0], -F[1], atol=1e-12)


def test_site_invariances():
    d = _random_env(10, seed=7)
    dR = np.vstack([d, _random_env(25, 4.0, 5.99, seed=8)])
    U, q, gR, gA = O.site(MODEL, dR, d)
    Rm = Rotation.random(random_state=4).as_matrix()
    U2, q2, gR2, gA2 = O.site(MODEL, dR @ Rm.T, d @ Rm.T)
    assert U2 == pytest.approx(U, rel=1e-12)
    np.testing.assert_allclose(q2, q, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(gA2, gA @ Rm.T, rtol=1e-9, atol=1e-12)    # covariant
    perm = _rng(1).permutation(len(d))
    U3, q3, _, gA3 = O.site(MODEL, dR, d[perm])
    assert U3 == pytest.approx(U, rel=1e-12)
    np.testing.assert_allclose(gA3, gA[perm], rtol=1e-10, atol=1e-13)


def test_site_gradient_finite_difference():
    d = _random_env(8, seed=9)
    dR = np.vstack([d, _random_env(12, 4.0, 5.99, seed=10)])
    U, q, gR, gA = O.site(MODEL, dR, d)
    h = 1e-6
    # angular neighbour s moves in both lists (it is also a radial neighbour)
    for s in range(len(d)):
        for a in range(3):
            dp, dm = dR.copy(), dR.copy()
            ap, am = d.copy(), d.copy()
            dp[s, a] += h; ap[s, a] += h
            dm[s, a] -= h; am[s, a] -= h
            fd = (O.site(MODEL, dp, ap)[0] - O.site(MODEL, dm, am)[0]) / (2 * h)
            assert gR[s, a] + gA[s, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for s in range(len(d), len(dR)):
        for a in range(3):
            dp, dm = dR.copy(), dR.copy()
            dp[s, a] += h
            dm[s, a] -= h
            fd = (O.site(MODEL, dp, d)[0] - O.site(MODEL, dm, d)[0]) / (2 * h)
            assert gR[s, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# --- neighbours ------------------------------------------------------------------

def test_bcc_shell_counts_and_distances():
    s = I.small_box((6, 6, 6))
    a = I.A_W
    cnt6, dist = O.neighbor_counts(s.pos, s.box, s.pbc, 6.0, mode=0, maxn=58)
    cnt4, _ = O.neighbor_counts(s.pos, s.box, s.pbc, 4.0, mode=0)
    assert set(cnt6.tolist()) == {58} and set(cnt4.tolist()) == {14}
    shells = [(a * math.sqrt(3) / 2, 8), (a, 6), (a * math.sqrt(2), 12),
              (a * math.sqrt(11) / 2, 24), (a * math.sqrt(3), 8)]
    expect = np.concatenate([[r] * k for r, k in shells])
    np.testing.assert_allclose(dist[0], expect, rtol=1e-12)


def test_cell_grid_matches_brute_force():
    s = I.c1()
    for rc in (6.0, 4.0, 2.0):
        cb, db = O.neighbor_counts(s.pos, s.box, s.pbc, rc, mode=0, maxn=80)
        cg, dg = O.neighbor_counts(s.pos, s.box, s.pbc, rc, mode=1, maxn=80)
        np.testing.assert_array_equal(cb, cg)
        np.testing.assert_allclose(db, dg, rtol=0, atol=1e-12)
    # open z with a slab
    t = I.displaced(I.c5(ncell=6, vacuum=5.0), 0.05, 1)
    cb, _ = O.neighbor_counts(t.pos, t.box, t.pbc, 6.0, mode=0)
    cg, _ = O.neighbor_counts(t.pos, t.box, t.pbc, 6.0, mode=1)
    np.testing.assert_array_equal(cb, cg)
    assert cb.min() < 58 and cb.max() == 58  # surfaces have fewer neighbours


# --- energy, forces, virial --------------------------------------------------------

def test_perfect_lattice_zero_force_equal_sites():
    s = I.small_box((5, 5, 5))
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)
    assert np.max(np.abs(F)) < 1e-11
    np.testing.assert_allclose(U, U[0], rtol=1e-12)
    assert np.max(np.abs(W - np.diag(np.diag(W)))) < 1e-9    # cubic symmetry
    assert W[0, 0] == pytest.approx(W[1, 1], rel=1e-10)


def test_forces_finite_difference_small_periodic_box():
    """54-atom box (L = 9.5 A < 2 rc): images and self-images matter."""
    s = I.small_box((3, 3, 3), sigma=0.15, seed=2)
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    h = 1e-5
    for i in (0, 7, 31):
        for a in range(3):
            p, m = s.pos.copy(), s.pos.copy()
            p[i, a] += h
            m[i, a] -= h
            fd = -(O.energy_forces_virial(MODEL, p, s.box, s.pbc, use_grid=False)[0]
                   - O.energy_forces_virial(MODEL, m, s.box, s.pbc, use_grid=False)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    np.testing.assert_allclose(F.sum(axis=0), 0, atol=1e-10)


def test_forces_finite_difference_with_zbl_close_pairs():
    s = I.small_box((4, 4, 4), sigma=0.02, seed=3)
    s.pos[1] = s.pos[0] + np.array([0.6, 0.5, 0.4])     # ~0.88 A pair
    s.pos[2] = s.pos[0] + np.array([-1.1, 0.6, 0.3])    # ~1.29 A, in the switch
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)
    h = 1e-6
    for i in (0, 1, 2, 5):
        for a in range(3):
            p, m = s.pos.copy(), s.pos.copy()
            p[i, a] += h
            m[i, a] -= h
            fd = -(O.energy_forces_virial(MODEL, p, s.box, s.pbc)[0]
                   - O.energy_forces_virial(MODEL, m, s.box, s.pbc)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_images_extensivity():
    """A 54-atom periodic box (smaller than 2 r_c) replicated 2x2x2 has 8x the
    energy and the same per-atom forces: checks image enumeration."""
    s = I.small_box((3, 3, 3), sigma=0.12, seed=5)
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    reps = [np.array([i, j, k]) for i in range(2) for j in range(2) for k in range(2)]
    big = np.vstack([s.pos + rr * s.box for rr in reps])
    E8, F8, W8, U8 = O.energy_forces_virial(MODEL, big, 2 * s.box, s.pbc, use_grid=True)
    assert E8 == pytest.approx(8 * E, rel=1e-12)
    np.testing.assert_allclose(F8[:len(F)], F, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(W8, 8 * W, rtol=1e-10, atol=1e-9)


def test_virial_strain_derivative_periodic_diagonal():
    s = I.small_box((4, 4, 4), sigma=0.1, seed=6)
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)
    h = 1e-6
    for a in range(3):
        sc = np.ones(3)
        sc[a] = 1 + h
        Ep = O.energy_forces_virial(MODEL, s.pos * sc, s.box * sc, s.pbc)[0]
        sc[a] = 1 - h
        Em = O.energy_forces_virial(MODEL, s.pos * sc, s.box * sc, s.pbc)[0]
        assert W[a, a] == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6, abs=1e-6)


def test_virial_open_cluster_full_tensor():
    s = I.small_box((3, 3, 3), sigma=0.1, seed=8, pbc=(0, 0, 0))
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    np.testing.assert_allclose(W, np.einsum("ia,ib->ab", F, s.pos), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(W, W.T, rtol=1e-9, atol=1e-9)
    h = 1e-6
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3))
            eps[a, b] = h
            Ep = O.energy_forces_virial(MODEL, s.pos @ (np.eye(3) + eps).T, s.box, s.pbc,
                                        use_grid=False)[0]
            Em = O.energy_forces_virial(MODEL, s.pos @ (np.eye(3) - eps).T, s.box, s.pbc,
                                        use_grid=False)[0]
            assert W[a, b] == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6, abs=1e-7)


def test_translation_rotation_permutation_invariance():
    s = I.small_box((3, 3, 3), sigma=0.1, seed=9, pbc=(0, 0, 0))
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    Rm = Rotation.random(random_state=2).as_matrix()
    pos2 = s.pos @ Rm.T + np.array([3.3, -1.2, 7.7])
    E2, F2, _, _ = O.energy_forces_virial(MODEL, pos2, s.box, s.pbc, use_grid=False)
    assert E2 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F @ Rm.T, rtol=1e-9, atol=1e-11)
    perm = _rng(3).permutation(s.n)
    E3, F3, _, _ = O.energy_forces_virial(MODEL, s.pos[perm], s.box, s.pbc, use_grid=False)
    assert E3 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F3, F[perm], rtol=1e-10, atol=1e-12)
    # periodic translation
    t = I.small_box((4, 4, 4), sigma=0.1, seed=10)
    Et, Ft, _, _ = O.energy_forces_virial(MODEL, t.pos, t.box, t.pbc)
    Et2, Ft2, _, _ = O.energy_forces_virial(MODEL, t.pos + np.array([5.0, -3.0, 11.0]),
                                            t.box, t.pbc)
    assert Et2 == pytest.approx(Et, rel=1e-12)
    np.testing.assert_allclose(Ft2, Ft, rtol=1e-9, atol=1e-11)


def test_grid_equals_brute_force_c1():
    s = I.c1()
    E1, F1, W1, U1 = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=True)
    E0, F0, W0, U0 = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    assert E1 == pytest.approx(E0, rel=1e-13)
    np.testing.assert_allclose(F1, F0, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(W1, W0, rtol=1e-11, atol=1e-10)


def test_forces_subset_matches_full():
    s = I.displaced(I.c5(ncell=6, vacuum=5.0), 0.05, 2)
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)
    idx = np.array([0, 5, 100, 333, s.n - 1])
    Fs, Us = O.forces_subset(MODEL, s.pos, s.box, s.pbc, idx)
    np.testing.assert_allclose(Fs, F[idx], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Us, U[idx], rtol=1e-13)
    t = I.small_box((3, 3, 3), sigma=0.1, seed=11)   # small box: images
    E, F, W, U = O.energy_forces_virial(MODEL, t.pos, t.box, t.pbc, use_grid=False)
    Fs, Us = O.forces_subset(MODEL, t.pos, t.box, t.pbc, np.arange(t.n))
    np.testing.assert_allclose(Fs, F, rtol=1e-10, atol=1e-12)


def test_force_scales_dimers_triangle_and_linearity():
    """Rounding-error scales of each atom: the pair-term magnitude sum S is |F|
    for a symmetric dimer (NEP only at 3 A), Z is |F| with the network off at
    1.2 A (ZBL only); S + Z >= |F_i| for every atom of a disordered periodic
    box (triangle inequality); S is linear in the output weights w1 while the
    network scales follow their closed forms (W = S max_mu sum |w0 s q| for
    the dimer, SU linear in w1, TU = sum |w1 t| + |b1|); the subset routine
    gives the same values."""
    box = np.array([30.0, 30.0, 30.0])
    pos = np.array([[10.0, 10.0, 10.0], [13.0, 10.0, 10.0]])
    E, F, W, U = O.energy_forces_virial(MODEL, pos, box, [0, 0, 0], use_grid=False)
    sc = O.force_scales(MODEL, pos, box, [0, 0, 0], use_grid=False)
    np.testing.assert_allclose(sc[:, 0], np.linalg.norm(F, axis=1), rtol=1e-12)
    assert np.all(sc[:, 1] == 0)
    # network scales of one site from its descriptor (closed forms)
    H, D = MODEL.n_hidden, MODEL.dim
    P = MODEL.params
    w0 = P[:H * D].reshape(H, D) * MODEL.scaler[None, :]
    b0, w1, b1 = P[H * D:H * D + H], P[H * D + H:H * D + 2 * H], P[H * D + 2 * H]
    q = O.descriptors(MODEL, pos, box, [0, 0, 0], use_grid=False)[0]
    habs = np.abs(w0 * q[None, :]).sum(1)
    t = np.tanh(w0 @ q - b0)
    # W: both terms of atom 0's force come from sites with one radial neighbour
    np.testing.assert_allclose(sc[0, 2], sc[0, 0] * habs.max(), rtol=1e-12)
    np.testing.assert_allclose(sc[0, 3], np.sum(np.abs(w1 * (1 - t * t)) * habs), rtol=1e-12)
    np.testing.assert_allclose(sc[0, 4], np.sum(np.abs(w1 * t)) + abs(b1), rtol=1e-12)
    m = I.nep_model(1)
    m.params = np.zeros_like(m.params)
    pos[1, 0] = 11.2
    E, F, W, U = O.energy_forces_virial(m, pos, box, [0, 0, 0], use_grid=False)
    sc = O.force_scales(m, pos, box, [0, 0, 0], use_grid=False)
    assert np.all(sc[:, 0] == 0)
    np.testing.assert_allclose(sc[:, 1], abs(O.zbl(1.2)[1]), rtol=1e-12)
    np.testing.assert_allclose(sc[:, 1], np.linalg.norm(F, axis=1), rtol=1e-12)
    s = I.c3(ncell=6, fraction=0.05, radius=4.0, seed=5)
    E, F, W, U = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)
    sc = O.force_scales(MODEL, s.pos, s.box, s.pbc)
    assert np.all(sc[:, 0] + sc[:, 1] >= np.linalg.norm(F, axis=1) * (1 - 1e-12))
    assert np.any(sc[:, 1] > 0) and np.all(sc[:, 0] > 0)
    assert np.all(sc[:, 2] > 0) and np.all(sc[:, 4] > 0)
    m = I.nep_model(1)
    m.params = MODEL.params.copy()
    m.params[H * D + H:H * D + 2 * H] *= -2.5     # w1
    sc2 = O.force_scales(m, s.pos, s.box, s.pbc)
    np.testing.assert_allclose(sc2[:, 0], 2.5 * sc[:, 0], rtol=1e-10)
    np.testing.assert_allclose(sc2[:, 1], sc[:, 1], rtol=1e-12)
    np.testing.assert_allclose(sc2[:, 2], 2.5 * sc[:, 2], rtol=1e-10)
    np.testing.assert_allclose(sc2[:, 3], 2.5 * sc[:, 3], rtol=1e-10)
    idx = np.array([0, 7, s.n // 2, s.n - 1])
    Fs, Us, scs = O.forces_subset(MODEL, s.pos, s.box, s.pbc, idx, scales=True)
    np.testing.assert_allclose(scs, sc[idx], rtol=1e-11)


# --- MD ---------------------------------------------------------------------------

def _tiny_md_system():
    s = I.small_box((3, 3, 3), sigma=0.05, seed=12)
    s.vel = I.maxwell_boltzmann(_rng(13), s.n, 300.0)
    return s


def test_nve_drift_scales_as_dt_squared():
    s = _tiny_md_system()
    drift = []
    for dt in (1.0, 0.5):
        nsteps = int(round(40 / dt))
        E0 = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)[0]
        ke0 = 0.5 * s.mass * np.sum(s.vel ** 2) / I.EV_PER_AMU_A2_FS2
        _, _, _, th = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, dt, nsteps, use_grid=False)
        etot = th[:, 2] + th[:, 3]
        drift.append(np.max(np.abs(etot - (E0 + ke0))))
    ratio = drift[0] / drift[1]
    assert 2.5 < ratio < 6.0, (drift, ratio)
    # and small against the kinetic energy (a wrong unit in the kick would not be)
    ke0 = 0.5 * s.mass * np.sum(s.vel ** 2) / I.EV_PER_AMU_A2_FS2
    assert drift[1] < 1e-2 * ke0


def test_md_time_reversible():
    s = _tiny_md_system()
    p1, v1, F1, _ = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 20, use_grid=False)
    p2, v2, _, _ = O.md(MODEL, p1, -v1, s.box, s.pbc, s.mass, 1.0, 20, forces=F1,
                        use_grid=False)
    dp = p2 - s.pos
    dp -= s.box * np.round(dp / s.box)
    assert np.max(np.abs(dp)) < 1e-9
    np.testing.assert_allclose(-v2, s.vel, atol=1e-11)


def test_variable_timestep_bounds_displacement():
    s = _tiny_md_system()
    s.vel[0] = [0.3, 0.2, -0.1]      # a fast atom (A/fs)
    d_max = 0.01
    p_prev = s.pos.copy()
    v = s.vel.copy()
    F = None
    for _ in range(5):
        p_new, v, F, th = O.md(MODEL, p_prev, v, s.box, s.pbc, s.mass, 1.0, 1, d_max=d_max,
                               forces=F, use_grid=False)
        dp = p_new - p_prev
        dp -= s.box * np.round(dp / s.box)
        assert th[0, 1] <= 1.0
        # the time step is set from the speeds before the step
        assert np.max(np.linalg.norm(dp, axis=1)) < 1.05 * d_max
        p_prev = p_new
