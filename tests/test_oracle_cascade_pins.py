"""Pins of the oracle's cascade-protocol pieces (Sec. II.B): the Nose-Hoover
chain thermostat on a group of atoms, the Berendsen barostat of the NPT
equilibration and the PKA launch, against facts that hold by construction:
reduction to NVE, the extended energy as a constant of the motion (error
shrinking as dt^2), canonical mean temperature, pressure relaxation, affine
box scaling and the kinetic energy of the launched atom.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

MODEL = I.nep_model(1)


def _system(ncell=3, T=300.0, seed=12):
    s = I.small_box((ncell, ncell, ncell), sigma=0.05, seed=seed)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(seed + 1), s.n, T)
    return s


def _border(s, width):
    """Atoms within `width` of a face of the box (the paper's 3 a0 shell)."""
    lo = np.min(np.stack([s.pos, s.box - s.pos]), axis=0)
    return (np.min(lo, axis=1) < width).astype(np.uint8)


def test_without_thermostat_and_barostat_is_nve():
    s = _system()
    p, v, F, th = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 15, use_grid=False)
    p2, v2, F2, th2, box = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 15,
                                    use_grid=False)
    np.testing.assert_array_equal(p, p2)
    np.testing.assert_array_equal(v, v2)
    np.testing.assert_array_equal(th[:, :4], th2[:, :4])
    np.testing.assert_array_equal(box, s.box)


@pytest.mark.parametrize("chain", [1, 4])
def test_nhc_extended_energy_is_conserved(chain):
    """PE + KE + E_NHC is a constant of the motion of the Nose-Hoover chain;
    its error shrinks as dt^2 (ratio 2.5-6 for dt 1 -> 0.5 fs) and is small
    against the kinetic energy.  A wrong force term G_j, scale or xi update
    breaks it.  The thermostat acts on the border shell only."""
    s = _system(ncell=4, T=300.0)
    grp = _border(s, 3.0)
    assert 0 < grp.sum() < s.n
    th_cfg = dict(T=900.0, tau=20.0, chain=chain, group=grp)
    E0 = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc)[0]
    ke0 = 0.5 * s.mass * np.sum(s.vel ** 2) / I.EV_PER_AMU_A2_FS2
    drift = []
    for dt in (1.0, 0.5):
        n = int(round(60 / dt))
        _, _, _, th, _ = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, dt, n,
                                  thermostat=th_cfg)
        H = th[:, 2] + th[:, 3] + th[:, 4]
        drift.append(np.max(np.abs(H - (E0 + ke0))))
        assert np.max(np.abs(th[:, 4])) > 10 * drift[-1]      # the thermostat did work
    assert 2.5 < drift[0] / drift[1] < 6.0, drift
    assert drift[1] < 1e-2 * ke0


@pytest.mark.parametrize("chain", [1, 4])
def test_nhc_mean_temperature_is_the_target(chain):
    """Canonical sampling: from 100 K, a thermostat on all 250 atoms (tau =
    20 fs) brings the mean temperature of the second half of an 800-step run to
    the 600 K target (within 5%: the temperature of 250 atoms fluctuates by
    ~5% and the window spans ~20 thermostat periods).  For one thermostat
    (chain 1) the long-time mean of 2 K - N_f kT is exactly zero (it is
    Q_1 dv_1/dt).  The crystal is taken at 0.91 a, near the random model's
    zero-pressure volume, where the bcc lattice is stable (at a it is not,
    and releases heat faster than a 20 fs thermostat removes it)."""
    s = I.small_box((5, 5, 5), a=0.91 * I.A_W, sigma=0.05, seed=20)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(21), s.n, 100.0)
    _, _, _, th, _ = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 800,
                              thermostat=dict(T=600.0, tau=20.0, chain=chain))
    T = 2 * th[400:, 3] / ((3 * s.n) * I.KB_EV)
    assert abs(T.mean() / 600.0 - 1) < 0.05, T.mean()


def test_barostat_off_and_affine_scaling():
    s = _system(ncell=4)
    # beta = 0: no coupling, box and trajectory of NVE
    p, v, F, th = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 5, use_grid=False)
    p2, v2, F2, th2, box = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 5,
                                    use_grid=False, barostat=dict(p0=0.0, tau=100.0, beta=0.0))
    np.testing.assert_array_equal(box, s.box)
    np.testing.assert_allclose(p2, p, rtol=0, atol=1e-12)
    # one coupled step: every coordinate of a periodic dimension scales by the
    # box ratio of that dimension; velocities are not scaled
    p1, v1, _, _, _ = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 1, use_grid=False)
    p3, v3, _, _, b3 = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 1,
                                use_grid=False, barostat=dict(p0=0.0, tau=100.0, beta=0.002))
    mu = b3 / s.box
    assert np.all(np.abs(mu - 1) > 1e-6)
    np.testing.assert_allclose(p3, p1 * mu[None, :], rtol=1e-14)
    np.testing.assert_array_equal(v3, v1)


def test_barostat_relaxes_the_pressure():
    """The random model is under about -37 GPa at the W lattice constant; with
    p0 = 0, tau_p = 50 fs and beta = 0.002 / GPa the box shrinks and the
    pressure relaxes to within a quarter of its start in 300 steps.  An open
    dimension keeps its extent."""
    s = _system(ncell=5, T=300.0, seed=3)

    def pressure(pos, vel, box):
        E, F, W, U = O.energy_forces_virial(MODEL, pos, box, s.pbc)
        k = np.sum(s.mass * vel ** 2, axis=0) / I.EV_PER_AMU_A2_FS2
        return (k + np.diag(W)) / np.prod(box) * O.EV_A3_GPA

    P0 = pressure(s.pos, s.vel, s.box)
    assert np.all(P0 < -20)
    p, v, F, th, box = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 300,
                                barostat=dict(p0=0.0, tau=50.0, beta=0.002))
    P1 = pressure(p, v, box)
    assert np.all(np.abs(P1) < 0.25 * np.abs(P0)), (P0, P1)
    assert np.all(box < s.box)
    # open z: only x and y couple
    s2 = s.copy()
    s2.pbc = np.array([1, 1, 0], np.int32)
    _, _, _, th2, box2 = O.md_ext(MODEL, s2.pos, s2.vel, s2.box, s2.pbc, s2.mass, 1.0, 20,
                                  barostat=dict(p0=0.0, tau=50.0, beta=0.002))
    assert box2[2] == s2.box[2] and box2[0] < s2.box[0]


def test_pka_launch():
    """The PKA gets exactly E_PKA of kinetic energy along <135>; the chosen atom
    is the nearest to the point (minimum image), lowest index on ties."""
    e = 1000.0
    v = O.pka_velocity(e, I.MASS_W, [1, 3, 5])
    assert 0.5 * I.MASS_W * v @ v / I.EV_PER_AMU_A2_FS2 == pytest.approx(e, rel=1e-14)
    np.testing.assert_allclose(np.cross(v, [1, 3, 5]), 0, atol=1e-12)
    assert np.all(v > 0)
    s = I.small_box((4, 4, 4))
    c = 0.5 * s.box
    i = O.pka_atom(s.pos, s.box, s.pbc, c)
    np.testing.assert_allclose(s.pos[i], c, atol=1e-12)           # the body-centre site
    j = O.pka_atom(s.pos, s.box, s.pbc, s.box - 0.1)              # wraps to the origin corner
    assert j == 0
    two = np.array([[1.0, 0, 0], [3.0, 0, 0]])
    assert O.pka_atom(two, [10.0, 10, 10], [1, 1, 1], [2.0, 0, 0]) == 0
