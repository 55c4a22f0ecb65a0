"""GPU parity of the multi-species path: W-Mo and W-Mo-Ta-Nb models (pair
coefficients per ordered species pair, mixed-Z ZBL, per-species masses)
through the C ABI against the FP64 oracle, element by element."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

from gpu_common import (F32_E_PER_ATOM, F32_F, F32_U, F32_W_PER_ATOM, F64_E_PER_ATOM, F64_F,
                        F64_U, F64_W_PER_ATOM, check_forces, check_sites, force_bound,
                        site_bound)

pytestmark = pytest.mark.gpu

WMO = ("W", "Mo")
HEA = ("W", "Mo", "Ta", "Nb")
SEEDS = {WMO: 301, HEA: 401}
_NEP = {}


def _model(species):
    return I.nep_model(SEEDS[species], species=species)


def _nep(species, precision):
    from paper_2305_08140_gb300 import nepzbl as N
    key = (species, precision)
    if key not in _NEP:
        _NEP[key] = N.NEP(_model(species), precision)
    return _NEP[key]


def _types_dev(s):
    import torch
    return torch.tensor(s.types, dtype=torch.int32, device="cuda")


def _parity(s, species, precision, scaled=False):
    from paper_2305_08140_gb300 import nepzbl as N
    E, F, W, U = _nep(species, precision).compute(N.to_device_soa(s.pos), s.box, s.pbc,
                                                  types=_types_dev(s), site_energy=True)
    F = F.cpu().numpy().T
    U = U.cpu().numpy()
    Eo, Fo, Wo, Uo = O.energy_forces_virial(_model(species), s.pos, s.box, s.pbc, types=s.types)
    if precision == "fp32":
        te, tw = F32_E_PER_ATOM, F32_W_PER_ATOM
    else:
        te, tw = F64_E_PER_ATOM, F64_W_PER_ATOM
    sc = O.force_scales(_model(species), s.pos, s.box, s.pbc, types=s.types) if scaled else None
    check_forces(F, Fo, force_bound(precision, sc))
    assert abs(E - Eo) / s.n <= te, (E, Eo)
    check_sites(U, Uo, site_bound(precision, Uo, sc))
    assert np.max(np.abs(W - Wo)) / s.n <= tw, (W, Wo)
    return E, F, Eo, Fo


def _wmo_box(ncell=(10, 10, 10), seed=301, sigma=0.08, close=True):
    s = I.alloy(I.small_box(ncell, sigma=sigma, seed=seed), [0.5, 0.5], seed=seed + 1)
    if close:
        # unlike-species pairs inside the ZBL range and its switch
        s.pos[1] = s.pos[0] + np.array([0.55, 0.45, 0.4])
        s.pos[3] = s.pos[2] + np.array([-0.9, 0.7, 0.5])
        s.types[0], s.types[1], s.types[2], s.types[3] = 0, 1, 1, 0
    return s


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_w_mo_alloy_2000_atoms(precision):
    _parity(_wmo_box(), WMO, precision, scaled=True)
    if precision == "fp32":
        # the several-species angular state in Tensor Memory (its close-pair
        # variant on the tiles holding the unlike close pairs)
        st = _nep(WMO, precision).stats()
        assert st["angular_state_in_tmem"] == 1 and st["angular_tiles_register"] == 0, st


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_hea_four_species_ragged(precision):
    # 7 x 7 x 8 cells: 784 atoms, 6 full tiles and a ragged one
    s = I.alloy(I.small_box((7, 7, 8), a=3.23, sigma=0.1, seed=311), [0.25] * 4, seed=312)
    _parity(s, HEA, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_b2_ordered_and_open_slab(precision):
    s = I.b2(8)
    s.pos += np.random.default_rng(313).normal(0.0, 0.05, s.pos.shape)
    s.pbc = np.array([1, 0, 1], np.int32)
    _parity(s, WMO, precision)


def test_hea_128000_atoms_fp32():
    """The full W-Mo-Ta-Nb box (40^3 cells) against the oracle's full
    evaluation."""
    _parity(I.hea(), HEA, "fp32")


def test_one_species_model_equals_identical_blocks():
    """A two-species model whose blocks all equal the W model's (and Z = 74
    twice) reproduces the one-species library result on a mixed labelling
    (the two paths run different kernels)."""
    from paper_2305_08140_gb300 import nepzbl as N
    w = I.nep_model(1)
    head = w.params[:30 * 30 + 61]
    cR = w.params[961:961 + 45]
    cA = w.params[961 + 45:]
    m2 = I.NepModel(species=("W", "W"))
    m2.params = np.concatenate([head, np.tile(cR, 4), np.tile(cA, 4)])
    m2.scaler = w.scaler
    s = _wmo_box(seed=321, close=False)
    x = N.to_device_soa(s.pos)
    # FP32: the two paths sum the radial basis in different orders (per
    # neighbour species, or inside the neighbour search)
    for prec, tol, tol_e in (("fp32", 2e-6, 2e-8), ("fp64", 1e-10, 1e-12)):
        a = N.NEP(w, prec)
        b = N.NEP(m2, prec)
        E1, F1, W1, _ = a.compute(x, s.box, s.pbc)
        E2, F2, W2, _ = b.compute(x, s.box, s.pbc, types=_types_dev(s))
        assert abs(E1 - E2) / s.n < tol_e
        assert float((F1 - F2).abs().max()) < tol
        a.close()
        b.close()


def _min_image(d, box, pbc):
    return d - np.where(np.asarray(pbc) > 0, box * np.round(d / box), 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_two_masses_matches_oracle(precision):
    from paper_2305_08140_gb300 import nepzbl as N
    s = _wmo_box(ncell=(8, 8, 8), seed=331, sigma=0.05, close=False)
    model = _model(WMO)
    masses = np.array(model.masses)[s.types]
    s.vel = I.maxwell_boltzmann(np.random.default_rng(332), s.n, 600.0, masses)
    m = N.NEP(model, precision)
    m.set_option(N.NEP_OPT_GRAPH_CHUNK, 7)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                   types=_types_dev(s))
    m.md(st, 50)
    p, v, F, th = O.md(model, s.pos, s.vel, s.box, s.pbc, model.masses, 1.0, 50, types=s.types)
    dp = np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc))
    vg = st.vel.cpu().numpy().T
    if precision == "fp64":
        assert dp.max() < 1e-9
        assert np.abs(vg - v).max() < 1e-10
        assert st.kinetic_energy == pytest.approx(th[-1, 3], abs=1e-8)
        assert st.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)
    else:
        assert dp.max() < 2e-5
        assert abs(st.kinetic_energy - th[-1, 3]) / s.n < 2e-6
        assert abs(st.potential_energy - th[-1, 2]) / s.n < 2e-6
    # total momentum stays zero with the per-species masses
    mom = (masses[:, None] * vg).sum(axis=0)
    assert np.max(np.abs(mom)) < 1e-6 * np.sum(masses) * np.abs(s.vel).max()
    m.close()


def test_md_hea_with_verlet_skin_fp32():
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.hea(ncell=10)
    model = _model(HEA)
    m = N.NEP(model, "fp32")
    m.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, 500)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                   types=_types_dev(s))
    m.md(st, 40)
    assert m.stats()["list_builds_skin"] < 40
    p, v, F, th = O.md(model, s.pos, s.vel, s.box, s.pbc, model.masses, 1.0, 40, types=s.types)
    assert np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc)).max() < 2e-5
    assert abs(st.potential_energy - th[-1, 2]) / s.n < 2e-6
    m.close()


def test_species_index_out_of_range_is_an_error():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = _wmo_box(close=False)
    t = _types_dev(s)
    t[17] = 2
    with pytest.raises(N.NepError) as e:
        _nep(WMO, "fp32").compute(N.to_device_soa(s.pos), s.box, s.pbc, types=t)
    assert e.value.code == N.NEP_ERR_INVALID_ARG
    t[17] = -1
    with pytest.raises(N.NepError):
        _nep(WMO, "fp64").compute(N.to_device_soa(s.pos), s.box, s.pbc, types=t)
    # a one-species model rejects index 1 as well
    one = N.NEP(I.nep_model(1), "fp32")
    with pytest.raises(N.NepError):
        one.compute(N.to_device_soa(s.pos), s.box, s.pbc, types=_types_dev(s))
    one.close()
    # the context stays usable
    E, _, _, _ = _nep(WMO, "fp32").compute(N.to_device_soa(s.pos), s.box, s.pbc,
                                           types=_types_dev(s))
    assert np.isfinite(E)


def test_set_params_two_species():
    from paper_2305_08140_gb300 import nepzbl as N
    s = _wmo_box(ncell=(6, 6, 6), seed=341, close=False)
    model = _model(WMO)
    m = N.NEP(model, "fp64")
    theta = model.params * 0.8
    m.set_params(theta)
    E, F, W, U = m.compute(N.to_device_soa(s.pos), s.box, s.pbc, types=_types_dev(s))
    m2 = _model(WMO)
    m2.params = theta
    Eo, Fo, Wo, Uo = O.energy_forces_virial(m2, s.pos, s.box, s.pbc, types=s.types)
    assert E == pytest.approx(Eo, rel=1e-12)
    np.testing.assert_allclose(F.cpu().numpy().T, Fo, atol=1e-9)
    m.close()


def test_batch_species_index_out_of_range():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    m = _nep(WMO, "fp32")
    b = N.Batch(I.c4(2))
    b.types[3] = 2
    with pytest.raises(N.NepError) as e:
        m.batch_forward(b)
    assert e.value.code == N.NEP_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# Batched (training) path with several species
# ---------------------------------------------------------------------------

def _one_species(structs):
    return [I.Structure(t.pos, t.box, t.pbc, np.zeros_like(t.types)) for t in structs]


def _alloy_configs(k, seed):
    out = []
    for c, s in enumerate([s for s in I.c4(64, seed=seed) if s.n <= 128][:k]):
        out.append(I.alloy(s, [0.5, 0.5], seed=seed + 100 + c))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_forward_two_species(precision):
    from oracle import training as T
    from paper_2305_08140_gb300 import nepzbl as N
    structs = _alloy_configs(8, 401)
    model = _model(WMO)
    nep = N.NEP(model, precision)
    b = N.Batch(structs)
    E, F, W = nep.batch_forward(b, virials=True)
    Eo, Fo, Wo = T.evaluate(model, structs)
    E, F, W = E.cpu().numpy(), F.cpu().numpy().T, W.cpu().numpy()
    tf, te, tw = (1e-4, 1e-6, 2e-5) if precision == "fp32" else (1e-9, 1e-11, 1e-10)
    for c, s in enumerate(structs):
        a, z = b.offsets[c], b.offsets[c + 1]
        assert abs(E[c] - Eo[c]) / s.n <= te
        assert np.max(np.abs(F[a:z] - Fo[c])) <= tf
        assert np.max(np.abs(W[c] - Wo[c])) / s.n <= tw
    nep.close()


def test_batch_loss_gradient_two_species_all_parameters_fd():
    """All 961 + 90 x 4 = 1,321 parameters of the W-Mo model (FP64 path):
    energy + force + virial mean-square loss against central differences of
    the oracle's loss."""
    import torch
    from oracle import training as T
    from paper_2305_08140_gb300 import nepzbl as N
    structs = _alloy_configs(3, 402)
    model = _model(WMO)
    # targets: the W-only seed-101 model on the same positions (any fixed numbers)
    Et, Ft, Wt = T.evaluate(I.nep_model(101), _one_species(structs))
    W6t = T.virial6(Wt)
    hv = np.array([1, 0, 1], np.uint8)
    nep = N.NEP(model, "fp64")
    b = N.Batch(structs)
    dev = dict(dtype=torch.float64, device="cuda")
    L, g, E, F = nep.batch_loss_grad(b, torch.tensor(Et, **dev),
                                     torch.tensor(np.concatenate(Ft).T.copy(), **dev),
                                     W_target=torch.tensor(W6t, **dev), has_virial=hv,
                                     w_virial=0.1)
    Nn = [s.n for s in structs]

    def loss(theta):
        E_, F_, W_ = T.evaluate(model, structs, theta)
        return T.mse_loss(E_, F_, T.virial6(W_), Et, Ft, W6t, Nn, hv, 1.0, 1.0, 0.1)[0]

    assert L == pytest.approx(loss(model.params), rel=1e-10)
    g = g.cpu().numpy()
    assert g.shape == (model.n_params,)
    th = model.params
    fd = np.zeros(len(th))
    for k in range(len(th)):
        h = 1e-6 * max(1.0, abs(th[k]))
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        fd[k] = (loss(tp) - loss(tm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))
    nep.close()


def test_population_loss_four_species():
    import torch
    from oracle import training as T
    from paper_2305_08140_gb300 import nepzbl as N
    structs = [I.alloy(s, [0.25] * 4, seed=410 + c) for c, s in
               enumerate([s for s in I.c4(64, seed=403) if s.n <= 128][:4])]
    model = _model(HEA)
    Et, Ft, Wt = T.evaluate(I.nep_model(101), _one_species(structs))
    W6t = T.virial6(Wt)
    hv = np.ones(len(structs), np.uint8)
    weights = {"energy": 1.0, "force": 1.0, "virial": 0.1, "l1": 0.05, "l2": 0.05}
    rng = np.random.default_rng(404)
    thetas = model.params[None, :] + 0.05 * rng.normal(size=(3, model.n_params))
    dev = dict(dtype=torch.float64, device="cuda")
    for prec, rel in (("fp64", 1e-10), ("fp32", 2e-5)):
        nep = N.NEP(model, prec)
        b = N.Batch(structs)
        L = N.population_loss(nep, b, torch.tensor(thetas, **dev), torch.tensor(Et, **dev),
                              torch.tensor(np.concatenate(Ft).T.copy(), **dev),
                              torch.tensor(W6t, **dev), hv, weights).cpu().numpy()
        Nn = [s.n for s in structs]
        for k in range(len(thetas)):
            E_, F_, W_ = T.evaluate(model, structs, thetas[k])
            d = T.nep_loss(thetas[k], T.rmse_terms(E_, F_, T.virial6(W_), Et, Ft, W6t, Nn, hv),
                           weights)
            ref = [d[t] for t in ("total", "l1", "l2", "energy", "force", "virial")]
            np.testing.assert_allclose(L[k], ref, rtol=rel, atol=1e-12)
        nep.close()
