"""GPU parity in triclinic cells (rows of H are the cell vectors): skewed and
rotated cells, an open dimension, MD with the fractional wrap and with a
Verlet skin, against the oracle's brute-force images."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

from gpu_common import (F32_E_PER_ATOM, F32_F, F32_U, F32_W_PER_ATOM, F64_E_PER_ATOM, F64_F,
                        F64_U, F64_W_PER_ATOM)

pytestmark = pytest.mark.gpu

MODEL = I.nep_model(1)


def _parity(s, precision):
    from paper_2305_08140_gb300 import nepzbl as N
    nep = N.NEP(MODEL, precision)
    E, F, W, U = nep.compute(N.to_device_soa(s.pos), s.box, s.pbc, site_energy=True)
    nep.close()
    F = F.cpu().numpy().T
    U = U.cpu().numpy()
    Eo, Fo, Wo, Uo = O.energy_forces_virial(MODEL, s.pos, s.box, s.pbc, use_grid=False)
    if precision == "fp32":
        tf, te, tu, tw = F32_F, F32_E_PER_ATOM, F32_U, F32_W_PER_ATOM
    else:
        tf, te, tu, tw = F64_F, F64_E_PER_ATOM, F64_U, F64_W_PER_ATOM
    assert np.max(np.abs(F - Fo)) <= tf, np.max(np.abs(F - Fo))
    assert abs(E - Eo) / s.n <= te
    assert np.max(np.abs(U - Uo)) <= tu
    assert np.max(np.abs(W - Wo)) / s.n <= tw


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_skewed_cell(precision):
    _parity(I.triclinic(), precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rotated_orthorhombic_cell(precision):
    """An orthorhombic crystal in a general orientation (every entry of H
    nonzero)."""
    s = I.small_box((7, 7, 8), sigma=0.05, seed=82)
    R = Rotation.random(random_state=83).as_matrix()
    t = I.Structure(s.pos @ R.T, np.diag(s.box) @ R.T, s.pbc, s.types)
    _parity(t, precision)


def test_skewed_cell_with_open_dimension():
    s = I.triclinic(ncell=7, shear=2.0, seed=84, pbc=(1, 1, 0))
    _parity(s, "fp64")


def _frac_min_image(d, H, pbc):
    return O.min_image(d, H, pbc)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_skewed_cell(precision):
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.triclinic(seed=85)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(86), s.n, 600.0)
    m = N.NEP(MODEL, precision)
    m.set_option(N.NEP_OPT_GRAPH_CHUNK, 7)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    m.md(st, 30)
    p, v, F, th = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 30, use_grid=False)
    xg = st.xyz.cpu().numpy().T
    frac = xg @ np.linalg.inv(s.box)
    assert np.all(frac >= 0) and np.all(frac < 1)
    dp = np.abs(_frac_min_image(xg - p, s.box, s.pbc))
    if precision == "fp64":
        assert dp.max() < 1e-9
        assert st.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)
    else:
        assert dp.max() < 2e-5
        assert abs(st.potential_energy - th[-1, 2]) / s.n < 2e-6
    m.close()


def test_md_skewed_cell_with_verlet_skin_fp32():
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.triclinic(seed=87)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(88), s.n, 900.0)
    m = N.NEP(MODEL, "fp32")
    m.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, 500)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    m.md(st, 40)
    assert m.stats()["list_builds_skin"] < 40
    p, v, F, th = O.md(MODEL, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 40, use_grid=False)
    dp = np.abs(_frac_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc))
    assert dp.max() < 2e-5
    m.close()


def test_triclinic_errors():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.triclinic(seed=89)
    m = N.NEP(MODEL, "fp32")
    with pytest.raises(N.NepError):      # left-handed cell: det H < 0
        m.compute(N.to_device_soa(s.pos), s.box[[1, 0, 2]], s.pbc)
    m.set_barostat(0.0, tau=100.0, compressibility=0.002)
    st = N.MDState(N.to_device_soa(s.pos), torch.zeros((3, s.n), dtype=torch.float64,
                                                       device="cuda"), s.box, s.pbc)
    with pytest.raises(N.NepError) as e:
        m.md(st, 2)
    assert e.value.code == N.NEP_ERR_UNSUPPORTED
    m.close()
