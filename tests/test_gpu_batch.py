"""Batched small periodic configurations (the training-style workload): energies
and forces against the oracle, and the hand-written parameter gradient of an
energy+force loss (force term included) against central finite differences of
the FP64 oracle's loss."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TARGET_SEED = 101


def _oracle_EF(model, structs):
    E, F = [], []
    for s in structs:
        e, f, _, _ = O.energy_forces_virial(model, s.pos, s.box, s.pbc)
        E.append(e)
        F.append(f)
    return np.array(E), F


def _oracle_loss(model, theta, structs, Et, Ft, we=1.0, wf=1.0):
    m = I.nep_model(model.seed)
    m.params = theta
    E, F = _oracle_EF(m, structs)
    N = np.array([s.n for s in structs])
    Fall = np.concatenate(F)
    Ftall = np.concatenate(Ft)
    return we * np.mean(((E - Et) / N) ** 2) + wf * np.mean((Fall - Ftall) ** 2)


def _targets(structs):
    return _oracle_EF(I.nep_model(TARGET_SEED), structs)


def _fd_grad(model, structs, Et, Ft, idx, we=1.0, wf=1.0):
    theta = model.params.copy()
    g = np.zeros(len(idx))
    for t, k in enumerate(idx):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        g[t] = (_oracle_loss(model, tp, structs, Et, Ft, we, wf)
                - _oracle_loss(model, tm, structs, Et, Ft, we, wf)) / (2 * h)
    return g


def _gpu(structs, precision="fp32", seed=1):
    from paper_2305_08140_gb300 import nepzbl as N
    nep = N.NEP(I.nep_model(seed), precision)
    return nep, N.Batch(structs)


def _targets_dev(Et, Ft):
    import torch
    return (torch.tensor(Et, dtype=torch.float64, device="cuda"),
            torch.tensor(np.concatenate(Ft).T.copy(), dtype=torch.float64, device="cuda"))


def _small_configs(k, seed=4):
    return [s for s in I.c4(64, seed=seed) if s.n <= 128][:k]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_forward_matches_oracle_all_512(precision):
    """The full 512-configuration batch (~116k atoms, one persistent launch):
    every configuration's energy and virial and every atom's force against the
    oracle, element by element."""
    structs = I.c4()
    assert len(structs) == 512
    nep, b = _gpu(structs, precision)
    E, F, W = nep.batch_forward(b, virials=True)
    E = E.cpu().numpy()
    F = F.cpu().numpy().T
    W = W.cpu().numpy()
    tf = 1e-4 if precision == "fp32" else 1e-9
    te = 1e-6 if precision == "fp32" else 1e-11
    tw = 2e-5 if precision == "fp32" else 1e-10
    worst = [0.0, 0.0, 0.0]
    for c, s in enumerate(structs):
        Eo, Fo, Wo, _ = O.energy_forces_virial(I.nep_model(1), s.pos, s.box, s.pbc)
        a, z = b.offsets[c], b.offsets[c + 1]
        de, df, dw = abs(E[c] - Eo) / s.n, np.max(np.abs(F[a:z] - Fo)), np.max(np.abs(W[c] - Wo)) / s.n
        worst = [max(worst[0], de), max(worst[1], df), max(worst[2], dw)]
        assert de <= te, (c, E[c], Eo)
        assert df <= tf, (c, df)
        assert dw <= tw, (c, W[c], Wo)
    print(f"512 configurations: max |dE|/N {worst[0]:.2e}, max |dF| {worst[1]:.2e}, "
          f"max |dW|/N {worst[2]:.2e}")
    nep.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_gradient_all_parameters_fd(precision):
    """All 1051 parameters on a small batch.  FP64 path: every component within
    1e-6 relative (plus 1e-9 of the largest); FP32 path: relative 2-norm error
    <= 1e-5."""
    structs = _small_configs(4)
    Et, Ft = _targets(structs)
    model = I.nep_model(1)
    nep, b = _gpu(structs, precision)
    Etd, Ftd = _targets_dev(Et, Ft)
    L, g, E, F = nep.batch_loss_grad(b, Etd, Ftd)
    g = g.cpu().numpy()
    Lo = _oracle_loss(model, model.params, structs, Et, Ft)
    assert L == pytest.approx(Lo, rel=1e-10 if precision == "fp64" else 1e-5)
    fd = _fd_grad(model, structs, Et, Ft, np.arange(len(model.params)))
    if precision == "fp64":
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))
    else:
        assert np.linalg.norm(g - fd) / np.linalg.norm(fd) <= 1e-5
    nep.close()


def test_c4_512_configurations_loss_and_sampled_gradient():
    """The full 512-configuration batch (~110k atoms) in one persistent launch;
    loss against the oracle, gradient components sampled from every parameter
    block against central finite differences of the oracle's loss."""
    structs = I.c4()
    Et, Ft = _targets(structs)
    model = I.nep_model(1)
    nep, b = _gpu(structs, "fp32")
    Etd, Ftd = _targets_dev(Et, Ft)
    L, g, E, F = nep.batch_loss_grad(b, Etd, Ftd)
    g = g.cpu().numpy()
    Lo = _oracle_loss(model, model.params, structs, Et, Ft)
    assert L == pytest.approx(Lo, rel=1e-5)
    # the fused launch's own energies and forces, every configuration
    Eo, Fo = _oracle_EF(model, structs)
    E = E.cpu().numpy()
    F = F.cpu().numpy().T
    for c, s in enumerate(structs):
        a, z = b.offsets[c], b.offsets[c + 1]
        assert abs(E[c] - Eo[c]) / s.n <= 1e-6, (c, E[c], Eo[c])
        assert np.max(np.abs(F[a:z] - Fo[c])) <= 1e-4, c
    rng = np.random.default_rng(7)
    H, D = 30, 30
    idx = np.concatenate([rng.choice(H * D, 6, replace=False), H * D + rng.choice(30, 3),
                          H * D + 30 + rng.choice(30, 3), [H * D + 60],
                          H * D + 61 + rng.choice(45, 4), H * D + 106 + rng.choice(45, 4)])
    fd = _fd_grad(model, structs, Et, Ft, idx)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(g[idx] - fd)) <= 1e-5 * scale, (g[idx], fd)
    nep.close()


def test_backward_arbitrary_upstream_gradients():
    """nep_batch_backward with random dL/dE, dL/dF equals the FD derivative of
    the linear functional sum_s c_s E_s + sum_i d_i . F_i (oracle)."""
    import torch
    structs = _small_configs(3, seed=9)
    nep, b = _gpu(structs, "fp64")
    rng = np.random.default_rng(11)
    c = rng.normal(size=len(structs))
    d = [rng.normal(size=(s.n, 3)) for s in structs]
    g = nep.batch_backward(b, torch.tensor(c, device="cuda"),
                           torch.tensor(np.concatenate(d).T.copy(), device="cuda")).cpu().numpy()
    model = I.nep_model(1)

    def functional(theta):
        m = I.nep_model(1)
        m.params = theta
        E, F = _oracle_EF(m, structs)
        return float(c @ E + sum(np.sum(di * fi) for di, fi in zip(d, F)))

    idx = np.concatenate([np.arange(0, 900, 97), np.arange(900, 1051, 13)])
    th = model.params
    for k in idx:
        h = 1e-6 * max(1.0, abs(th[k]))
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        fdk = (functional(tp) - functional(tm)) / (2 * h)
        assert g[k] == pytest.approx(fdk, rel=1e-6, abs=1e-9 * max(1.0, np.max(np.abs(g))))
    nep.close()


def test_autograd_function_matches_fused_loss():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs = _small_configs(4, seed=12)
    Et, Ft = _targets(structs)
    nep, b = _gpu(structs, "fp32")
    Etd, Ftd = _targets_dev(Et, Ft)
    L_fused, g_fused, _, _ = nep.batch_loss_grad(b, Etd, Ftd)
    fn = N.energy_forces_function()
    theta = torch.tensor(I.nep_model(1).params, dtype=torch.float64, requires_grad=True)
    E, F = fn.apply(theta, nep, b)
    Ns = torch.tensor([s.n for s in structs], dtype=torch.float64, device="cuda")
    loss = torch.mean(((E - Etd) / Ns) ** 2) + torch.mean((F - Ftd) ** 2)
    loss.backward()
    assert loss.item() == pytest.approx(L_fused, rel=1e-12)
    g = theta.grad.numpy()
    gf = g_fused.cpu().numpy()
    assert np.linalg.norm(g - gf) / np.linalg.norm(gf) <= 1e-6
    nep.close()


def test_set_params_changes_the_model():
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.small_box((6, 6, 6), sigma=0.1, seed=13)
    nep = N.NEP(I.nep_model(1), "fp64")
    theta = I.nep_model(1).params * 0.7
    nep.set_params(theta)
    E, F, W, U = nep.compute(N.to_device_soa(s.pos), s.box, s.pbc)
    m = I.nep_model(1)
    m.params = theta
    Eo, Fo, Wo, Uo = O.energy_forces_virial(m, s.pos, s.box, s.pbc)
    assert E == pytest.approx(Eo, rel=1e-12)
    np.testing.assert_allclose(F.cpu().numpy().T, Fo, atol=1e-9)
    nep.close()


def test_autotune_and_overflow_growth():
    structs = _small_configs(6, seed=14)
    Et, Ft = _targets(structs)
    nep, b = _gpu(structs, "fp32")
    Etd, Ftd = _targets_dev(Et, Ft)
    L0, g0, _, _ = nep.batch_loss_grad(b, Etd, Ftd)
    bt, per = nep.batch_autotune(b, Etd, Ftd)
    assert bt in (64, 128, 256) and per in (1, 2, 4)
    L1, g1, _, _ = nep.batch_loss_grad(b, Etd, Ftd)
    assert L1 == pytest.approx(L0, rel=1e-12)
    np.testing.assert_allclose(g1.cpu().numpy(), g0.cpu().numpy(), rtol=1e-5,
                               atol=1e-7 * float(g0.abs().max()))
    nep.close()


# ---------------------------------------------------------------------------
# Virials: per-configuration virial, virial loss term and its gradient
# ---------------------------------------------------------------------------

def _oracle_W(model, structs):
    from oracle import training as T
    return T.evaluate(model, structs)[2]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_virials_match_oracle(precision):
    structs = I.c4(24, seed=21)
    nep, b = _gpu(structs, precision)
    E, F, W = nep.batch_forward(b, virials=True)
    Wo = _oracle_W(I.nep_model(1), structs)
    W = W.cpu().numpy()
    tw = 2e-5 if precision == "fp32" else 1e-10
    for c, s in enumerate(structs):
        assert np.max(np.abs(W[c] - Wo[c])) / s.n <= tw, (c, W[c], Wo[c])
    nep.close()


def _virial_targets(structs, seed=22):
    """Seed-101 model virials (six components) as targets, with a mask."""
    from oracle import training as T
    W6 = T.virial6(_oracle_W(I.nep_model(TARGET_SEED), structs))
    hv = np.random.default_rng(seed).integers(0, 2, len(structs)).astype(np.uint8)
    hv[0] = 1
    return W6, hv


def _oracle_mse(model, theta, structs, Et, Ft, W6t, hv, we, wf, wv):
    from oracle import training as T
    E, F, W = T.evaluate(model, structs, theta)
    N = [s.n for s in structs]
    return T.mse_loss(E, F, T.virial6(W), Et, Ft, W6t, N, hv, we, wf, wv)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_loss_with_virial_term_gradient_all_parameters_fd(precision):
    """Energy + force + virial mean-square loss on a small batch with some
    configurations lacking a virial target: loss terms against the oracle,
    all 1051 gradient components against central differences of the oracle's
    loss."""
    import torch
    structs = _small_configs(4, seed=23)
    Et, Ft = _targets(structs)
    W6t, hv = _virial_targets(structs)
    model = I.nep_model(1)
    nep, b = _gpu(structs, precision)
    Etd, Ftd = _targets_dev(Et, Ft)
    Wtd = torch.tensor(W6t, dtype=torch.float64, device="cuda")
    we, wf, wv = 1.0, 1.0, 0.1
    L, g, E, F = nep.batch_loss_grad(b, Etd, Ftd, we, wf, W_target=Wtd, has_virial=hv, w_virial=wv)
    Lo, le, lf, lv = _oracle_mse(model, None, structs, Et, Ft, W6t, hv, we, wf, wv)
    rel = 1e-10 if precision == "fp64" else 2e-5
    assert L == pytest.approx(Lo, rel=rel)
    assert nep.last_loss_terms["virial"] == pytest.approx(lv, rel=rel)
    assert lv > 0.01 * Lo            # the virial term matters in this test
    theta = model.params.copy()
    fd = np.zeros(len(theta))
    for k in range(len(theta)):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd[k] = (_oracle_mse(model, tp, structs, Et, Ft, W6t, hv, we, wf, wv)[0]
                 - _oracle_mse(model, tm, structs, Et, Ft, W6t, hv, we, wf, wv)[0]) / (2 * h)
    g = g.cpu().numpy()
    if precision == "fp64":
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))
    else:
        assert np.linalg.norm(g - fd) / np.linalg.norm(fd) <= 1e-5
    nep.close()


def test_backward_with_virial_upstream():
    """nep_batch_backward with random dL/dE, dL/dF and dL/dW equals the FD
    derivative of sum_s c_s E_s + sum_i d_i . F_i + sum_s G_s : W_s."""
    import torch
    from oracle import training as T
    structs = _small_configs(3, seed=24)
    nep, b = _gpu(structs, "fp64")
    rng = np.random.default_rng(25)
    c = rng.normal(size=len(structs))
    d = [rng.normal(size=(s.n, 3)) for s in structs]
    G = rng.normal(size=(len(structs), 3, 3))
    g = nep.batch_backward(b, torch.tensor(c, device="cuda"),
                           torch.tensor(np.concatenate(d).T.copy(), device="cuda"),
                           torch.tensor(G, device="cuda")).cpu().numpy()
    model = I.nep_model(1)

    def functional(theta):
        E, F, W = T.evaluate(model, structs, theta)
        return float(c @ E + sum(np.sum(di * fi) for di, fi in zip(d, F)) + np.sum(G * W))

    # five-point differences with h = 1e-4: the virial sums thousands of pair
    # terms of ~10 eV, so a 1e-6 step would leave ~1e-6 of rounding noise
    th = model.params
    for k in np.concatenate([np.arange(0, 900, 89), np.arange(900, 1051, 11)]):
        h = 1e-4 * max(1.0, abs(th[k]))
        f = []
        for m in (-2, -1, 1, 2):
            t = th.copy(); t[k] += m * h
            f.append(functional(t))
        fdk = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        assert g[k] == pytest.approx(fdk, rel=1e-7, abs=1e-9 * max(1.0, np.max(np.abs(g))))
    nep.close()


def test_autograd_function_with_virials():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    structs = _small_configs(4, seed=26)
    Et, Ft = _targets(structs)
    W6t, hv = _virial_targets(structs, seed=27)
    nep, b = _gpu(structs, "fp64")
    Etd, Ftd = _targets_dev(Et, Ft)
    Wtd = torch.tensor(W6t, dtype=torch.float64, device="cuda")
    L_fused, g_fused, _, _ = nep.batch_loss_grad(b, Etd, Ftd, W_target=Wtd, has_virial=hv,
                                                 w_virial=0.1)
    fn = N.energy_forces_function(virials=True)
    theta = torch.tensor(I.nep_model(1).params, dtype=torch.float64, requires_grad=True)
    E, F, W = fn.apply(theta, nep, b)
    Ns = torch.tensor([s.n for s in structs], dtype=torch.float64, device="cuda")
    idx = [(0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (0, 1)]
    W6 = torch.stack([W[:, a, c] for a, c in idx], dim=1)
    m = torch.tensor(hv, dtype=torch.bool, device="cuda")
    lv = 0.1 * torch.mean(((W6 - Wtd)[m] / Ns[m, None]) ** 2)
    loss = torch.mean(((E - Etd) / Ns) ** 2) + torch.mean((F - Ftd) ** 2) + lv
    loss.backward()
    assert loss.item() == pytest.approx(L_fused, rel=1e-12)
    np.testing.assert_allclose(theta.grad.numpy(), g_fused.cpu().numpy(), rtol=1e-8,
                               atol=1e-12 * float(g_fused.abs().max()))
    nep.close()
