"""GPU parity of the cascade-protocol pieces (Sec. II.B) through the C ABI
against the oracle's extended MD: the Nose-Hoover chain on the 3 a0 border
shell, the Berendsen barostat of the NPT equilibration, and the PKA launch
along <135> with the variable time step."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MODEL = I.nep_model(1)


def _border(s, width):
    lo = np.min(np.stack([s.pos, s.box - s.pos]), axis=0)
    return (np.min(lo, axis=1) < width).astype(np.uint8)


def _state(N, s, d_max=0.0):
    return N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                     d_max=d_max)


def _min_image(d, box, pbc):
    return d - np.where(np.asarray(pbc) > 0, box * np.round(d / box), 0.0)


def _system(ncell=8, a=I.A_W, T=300.0, seed=51):
    s = I.small_box((ncell,) * 3, a=a, sigma=0.05, seed=seed)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(seed + 1), s.n, T)
    return s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nhc_border_thermostat_matches_oracle(precision):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = _system()
    grp = _border(s, 3 * I.A_W)
    assert 0 < grp.sum() < s.n
    m = N.NEP(MODEL, precision)
    m.set_option(N.NEP_OPT_GRAPH_CHUNK, 7)
    m.set_thermostat(900.0, tau=20.0, chain=4,
                     group=torch.tensor(grp, dtype=torch.uint8, device="cuda"))
    st = _state(N, s)
    m.md(st, 40)
    p, v, F, th, _ = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 40,
                              thermostat=dict(T=900.0, tau=20.0, chain=4, group=grp))
    dp = np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc))
    if precision == "fp64":
        assert dp.max() < 1e-9
        assert st.thermostat_energy == pytest.approx(th[-1, 4], abs=1e-8)
        assert st.kinetic_energy == pytest.approx(th[-1, 3], abs=1e-8)
    else:
        assert dp.max() < 2e-5
        assert abs(st.thermostat_energy - th[-1, 4]) / s.n < 2e-6
        assert abs(st.kinetic_energy - th[-1, 3]) / s.n < 2e-6
    assert abs(th[-1, 4]) > 1e-3        # the thermostat did work
    m.close()


def test_thermostat_all_atoms_chain_one_and_continuation():
    """Chain length 1 on every atom, run as 15 + 15 steps in two calls (the
    chain state persists) against 30 oracle steps."""
    from paper_2305_08140_gb300 import nepzbl as N
    s = _system(ncell=6, seed=53)
    m = N.NEP(MODEL, "fp64")
    m.set_thermostat(600.0, tau=30.0, chain=1)
    st = _state(N, s)
    m.md(st, 15)
    m.md(st, 15)
    p, v, F, th, _ = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 30,
                              thermostat=dict(T=600.0, tau=30.0, chain=1))
    assert np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc)).max() < 1e-9
    assert st.thermostat_energy == pytest.approx(th[-1, 4], abs=1e-8)
    # switching it off gives NVE again
    m.set_thermostat(None)
    m.md(st, 3)
    assert st.thermostat_energy == 0.0
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_barostat_matches_oracle(precision):
    """NPT (Berendsen barostat + Nose-Hoover chain on all atoms) from the
    random model's tensile state at a: the box shrinks step by step exactly
    as in the oracle; one open dimension keeps its extent."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = _system(ncell=7, seed=55)
    s.pbc = np.array([1, 1, 0], np.int32)
    m = N.NEP(MODEL, precision)
    m.set_barostat(0.0, tau=50.0, compressibility=0.002)
    m.set_thermostat(300.0, tau=50.0, chain=4)
    st = _state(N, s)
    m.md(st, 25)
    p, v, F, th, box = O.md_ext(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 25,
                                thermostat=dict(T=300.0, tau=50.0, chain=4),
                                barostat=dict(p0=0.0, tau=50.0, beta=0.002))
    assert np.all(box[:2] < s.box[:2]) and box[2] == s.box[2]
    xg = st.xyz.cpu().numpy().T
    if precision == "fp64":
        np.testing.assert_allclose(st.box, box, rtol=1e-12)
        assert np.abs(_min_image(xg - p, box, s.pbc)).max() < 1e-9
    else:
        np.testing.assert_allclose(st.box, box, rtol=1e-8)
        assert np.abs(_min_image(xg - p, box, s.pbc)).max() < 2e-5
    m.close()


def test_pka_launch_and_cascade_start_fp64():
    """The start of a cascade: border thermostat at 300 K, a 1 keV PKA at the
    box centre along <135>, variable time step (0.01 A per step, dt <= 1 fs):
    the chosen atom, its velocity and 30 steps against the oracle."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = _system(ncell=8, seed=57)
    grp = _border(s, 3 * I.A_W)
    m = N.NEP(MODEL, "fp64")
    m.set_thermostat(300.0, tau=100.0, chain=4,
                     group=torch.tensor(grp, dtype=torch.uint8, device="cuda"))
    st = _state(N, s, d_max=0.01)
    centre = 0.5 * s.box
    atom = m.pka(st, centre, 1000.0, (1, 3, 5))
    assert atom == O.pka_atom(s.pos, s.box, s.pbc, centre)
    v0 = s.vel.copy()
    v0[atom] = O.pka_velocity(1000.0, I.MASS_W, (1, 3, 5))
    vg = st.vel.cpu().numpy().T
    np.testing.assert_allclose(vg[atom], v0[atom], rtol=1e-14)
    np.testing.assert_array_equal(np.delete(vg, atom, 0), np.delete(s.vel, atom, 0))
    m.md(st, 30)
    p, v, F, th, _ = O.md_ext(MODEL, s.pos, v0, s.box, s.pbc, s.mass, 1.0, 30, d_max=0.01,
                              thermostat=dict(T=300.0, tau=100.0, chain=4, group=grp))
    assert st.time == pytest.approx(th[:, 1].sum(), rel=1e-9)
    assert np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc)).max() < 1e-8
    m.close()


def test_cascade_argument_errors():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    m = N.NEP(MODEL, "fp32")
    with pytest.raises(N.NepError):
        m.set_thermostat(300.0, tau=0.0)
    with pytest.raises(N.NepError):
        m.set_thermostat(300.0, tau=10.0, chain=9)
    with pytest.raises(N.NepError):
        m.set_thermostat(300.0, tau=10.0, group=torch.ones(5, dtype=torch.uint8))   # host
    with pytest.raises(N.NepError):
        m.set_barostat(0.0, tau=-1.0)
    s = _system(ncell=6, seed=59)
    st = _state(N, s)
    with pytest.raises(N.NepError):
        m.pka(st, (1.0, 1.0, 1.0), 100.0, (0.0, 0.0, 0.0))
    m.close()
