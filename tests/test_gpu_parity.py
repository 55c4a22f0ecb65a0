"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs, element by element."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

from gpu_common import (F32_E_PER_ATOM, F32_F, F64_F, assert_parity, check_forces, check_sites,
                        force_bound, gpu_eval, nep, oracle_eval, site_bound)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_c1_2000_atoms(precision):
    assert_parity(I.c1(), precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ragged_periodic_box(precision):
    # 6 x 6 x 7 cells: 504 atoms = 3 full tiles of 128 and a ragged one
    s = I.small_box((6, 6, 7), sigma=0.1, seed=21)
    assert_parity(s, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_open_z_slab(precision):
    s = I.displaced(I.c5(ncell=8, vacuum=10.0), 0.05, 22)
    assert_parity(s, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_close_pairs_zbl_clump(precision):
    """A small version of the close-pair stress case: ZBL pairs down to 0.3 A,
    ~7x the lattice density in the clump.  Each atom's force bound grows with
    the magnitudes of its NEP pair terms (the ZBL terms are FP64 on both
    paths); site energies per atom."""
    s = I.c3(ncell=10, fraction=0.05, radius=6.0, seed=23)
    assert_parity(s, precision, scaled=True)


def test_close_pair_list_overflow_tight_cluster():
    """FP32: more pairs inside the outer ZBL radius on one atom than the register
    kernel lists per atom (32; their FP64 displacements and ZBL terms are done
    warp-wide, later ones inline): 130 atoms moved into a 3.2 A sphere of a
    432-atom crystal (pairs down to 0.45 A, up to 40 inside 2 A on an atom),
    against the oracle with the per-atom bounds.  The virial (~6e5 eV here) is
    held to the flat per-atom bound plus the modelled rounding of every atom's
    NEP pair forces (its force bound above the flat part) times the radial
    cutoff, the longest lever arm a pair term has: the same pair forces enter
    the virial as -1/2 sum d_ij (x) f_ij."""
    from gpu_common import F32_W_PER_ATOM
    s = I.c3(ncell=6, fraction=0.3, radius=3.2, min_sep=0.45, seed=29)
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    assert (r < 2.0).sum(1).max() > 32
    E, F, W, U = gpu_eval(s, "fp32")
    Eo, Fo, Wo, Uo = oracle_eval(s)
    model = I.nep_model(1)
    sc = O.force_scales(model, s.pos, s.box, s.pbc)
    bF = force_bound("fp32", sc)
    check_forces(F, Fo, bF)
    assert abs(E - Eo) / s.n <= F32_E_PER_ATOM, (E, Eo)
    check_sites(U, Uo, site_bound("fp32", Uo, sc))
    bW = s.n * F32_W_PER_ATOM + model.rc_radial * float(np.sum(bF - F32_F))
    assert np.max(np.abs(W - Wo)) <= bW, (np.max(np.abs(W - Wo)), bW)


def test_single_atom_and_dimer():
    s = I.Structure(np.array([[3.0, 4.0, 5.0]]), np.array([20.0, 20.0, 20.0]),
                    np.array([1, 1, 1], np.int32), np.zeros(1, np.int32))
    E, F, W, U = gpu_eval(s, "fp64")
    Eo, Fo, Wo, Uo = oracle_eval(s)
    assert E == pytest.approx(Eo, abs=1e-12)
    assert np.all(F == 0)
    for r in (0.5, 1.5, 3.0, 5.0):
        d = I.Structure(np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]]),
                        np.array([20.0, 20.0, 20.0]), np.array([0, 0, 0], np.int32),
                        np.zeros(2, np.int32))
        for prec in ("fp32", "fp64"):
            assert_parity(d, prec, scaled=True)


def test_empty_system():
    from paper_2305_08140_gb300 import nepzbl as N
    import torch
    x = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    E, F, W, U = nep("fp32").compute(x, [20.0, 20.0, 20.0], [1, 1, 1])
    assert E == 0.0 and np.all(W == 0)


def test_fp32_deterministic_bitwise():
    s = I.displaced(I.small_box((8, 8, 8)), 0.08, 31)
    a = gpu_eval(s, "fp32")
    b = gpu_eval(s, "fp32")
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[3], b[3])


def test_periodic_shift_and_permutation():
    s = I.small_box((7, 7, 7), sigma=0.07, seed=32)
    E, F, W, U = gpu_eval(s, "fp32")
    t = s.copy()
    t.pos = t.pos + np.array([13.1, -7.7, 101.3])       # different cells, wrapped
    E2, F2, W2, U2 = gpu_eval(t, "fp32")
    assert abs(E2 - E) / s.n < 1e-7
    np.testing.assert_allclose(F2, F, atol=2e-5)
    perm = np.random.default_rng(3).permutation(s.n)
    t = s.copy()
    t.pos = s.pos[perm]
    E3, F3, W3, U3 = gpu_eval(t, "fp32")
    assert abs(E3 - E) / s.n < 1e-7
    np.testing.assert_allclose(F3, F[perm], atol=2e-5)


def test_capacity_grows_on_overflow():
    from paper_2305_08140_gb300 import nepzbl as N
    m = N.NEP(I.nep_model(1), "fp32")
    m.set_option(N.NEP_OPT_NBR_CAPACITY, 8)
    s = I.displaced(I.small_box((6, 6, 6)), 0.05, 33)
    E, F, W, U = m.compute(N.to_device_soa(s.pos), s.box, s.pbc, site_energy=True)
    st = m.stats()
    assert st["nbr_capacity"] >= st["max_nbr_radial"] >= 50
    E0, F0, W0, U0 = gpu_eval(s, "fp32")
    assert E == E0
    np.testing.assert_array_equal(F.cpu().numpy().T, F0)
    m.close()


def test_error_codes():
    from paper_2305_08140_gb300 import nepzbl as N
    import torch
    m = nep("fp32")
    s = I.small_box((6, 6, 6))
    x = N.to_device_soa(s.pos)
    with pytest.raises(N.NepError) as e:      # left-handed cell (det H < 0)
        m.compute(x, np.array([[0, 19.0, 0], [19.0, 1.0, 0], [0, 0, 19.0]]), [1, 1, 1])
    assert e.value.code == N.NEP_ERR_BOX
    with pytest.raises(N.NepError) as e:
        m.compute(x, [12.0, 19.0, 19.0], [1, 1, 1])          # < 3 r_c periodic
    assert e.value.code == N.NEP_ERR_BOX
    bad = x.clone()
    bad[0, 5] = float("nan")
    with pytest.raises(N.NepError) as e:
        m.compute(bad, s.box, s.pbc)
    assert e.value.code == N.NEP_ERR_NONFINITE
    # host memory where device memory is required
    import ctypes as C
    host = np.zeros(3 * s.n)
    Eo = C.c_double()
    rc = m.lib.nep_compute(m.ctx, s.n, C.c_void_p(host.ctypes.data),
                           np.diag(s.box).reshape(9).ctypes.data_as(C.POINTER(C.c_double)),
                           C.c_void_p(torch.zeros(s.n, dtype=torch.int32, device="cuda").data_ptr()),
                           (C.c_int32 * 3)(1, 1, 1), C.byref(Eo),
                           C.c_void_p(torch.zeros(3 * s.n, dtype=torch.float64,
                                                  device="cuda").data_ptr()),
                           None, None, None)
    assert rc == N.NEP_ERR_INVALID_ARG
    model = I.nep_model(1)
    model.n_hidden = 20
    model.params = model.params[:model.n_params]
    with pytest.raises(N.NepError) as e:
        N.NEP(model, "fp32")
    assert e.value.code == N.NEP_ERR_UNSUPPORTED


def test_atom_outside_open_extent():
    s = I.displaced(I.c5(ncell=6, vacuum=6.0), 0.05, 34)
    s.pos[0, 2] = -25.0          # far below the grid (sputtered atom)
    s.pos[1, 2] = s.box[2] + 40  # far above
    s.pos[2] = s.pos[1] + np.array([1.2, 0.3, 0.4])   # a close pair up there
    assert_parity(s, "fp32", scaled=True)
    assert_parity(s, "fp64", scaled=True)


# ---------------------------------------------------------------------------
# full-size workloads, sampled outputs
# ---------------------------------------------------------------------------

def _sampled(s, idx, precision="fp32", scaled=False):
    """Sampled atoms against the oracle, per atom; properties at any size."""
    E, F, W, U = gpu_eval(s, precision)
    Fo, Uo, sc = O.forces_subset(I.nep_model(1), s.pos, s.box, s.pbc, idx, scales=True)
    bound = force_bound(precision, sc if scaled else None)
    dF = np.abs(F[idx] - Fo)
    fn = np.linalg.norm(Fo, axis=1)
    rat = np.max(dF / bound, axis=1)
    w = int(np.argmax(rat))
    print(f"sampled {len(idx)}: max |dF| {dF.max():.3e}, max |dF|/bound {rat.max():.3f}, "
          f"max |dF_i|/|F_i| {np.max(np.max(dF, axis=1) / np.maximum(fn, 1e-30)):.3e}; worst atom "
          f"|F| {fn[w]:.3e} scales {sc[w]}; max |dU| {np.max(np.abs(U[idx] - Uo)):.3e}, "
          f"max |dU|/bound {np.max(np.abs(U[idx] - Uo) / site_bound(precision, Uo, sc)):.3f}")
    check_forces(F[idx], Fo, bound, "sampled")
    check_sites(U[idx], Uo, site_bound(precision, Uo, sc if scaled else None), "sampled")
    # properties at any size: E is the sum of the site energies, sum F = 0
    assert abs(E - U.sum()) / s.n < 1e-9
    if np.all(s.pbc):
        assert np.max(np.abs(F.sum(axis=0))) / s.n < 1e-9
    return E, F, W, U, Fo, sc


def test_c2_128000_atoms_full_oracle():
    s = I.displaced(I.c2(), 0.05, 41)
    assert_parity(s, "fp32")


def test_c5_8192000_atoms_sampled():
    s = I.c5()
    rng = np.random.default_rng(42)
    # random atoms plus atoms on both free surfaces
    z = s.pos[:, 2]
    surf = np.concatenate([np.argsort(z)[:40], np.argsort(z)[-40:]])
    idx = np.unique(np.concatenate([rng.choice(s.n, 120, replace=False), surf[::4]]))
    _sampled(s, idx)
    t = I.displaced(s, 0.05, 43)
    _sampled(t, idx)


def test_c3_250000_atoms_sampled():
    s = I.c3()
    moved = s.meta["moved"]
    rng = np.random.default_rng(44)
    idx = np.unique(np.concatenate([rng.choice(moved, 60, replace=False),
                                    rng.choice(s.n, 60, replace=False)]))
    # per-atom bounds from each atom's rounding-error scales (clump atoms: ~7x
    # the lattice neighbour count, pairs down to 0.3 A)
    _sampled(s, idx, scaled=True)


def test_md_graph_forces_equal_direct_evaluation_c5():
    """The graph-captured MD step (the launch configuration the bench times)
    evaluates forces bitwise equal to a direct evaluation: with a time step of
    1e-30 fs positions do not move in FP64."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.displaced(I.c5(), 0.05, 45)
    m = nep("fp32")
    x = N.to_device_soa(s.pos)
    E, F, W, U = m.compute(x.clone(), s.box, s.pbc)
    F = F.clone()
    st = N.MDState(x.clone(), torch.zeros_like(x), s.box, s.pbc, dt_max=1e-30)
    m.md(st, 2)
    # the step wraps periodic coordinates into [0, L) and changes nothing else
    L = torch.tensor(s.box, dtype=torch.float64, device=x.device)[:, None]
    per = torch.tensor(s.pbc, device=x.device)[:, None] > 0
    xw = torch.where(per, x - L * torch.floor(x / L), x)
    assert torch.equal(st.xyz, xw)
    assert torch.equal(st.forces, F)
    assert st.potential_energy == E


# ---------------------------------------------------------------------------
# MD against the oracle's velocity Verlet
# ---------------------------------------------------------------------------

def _run_md(s, precision, nsteps, dt=1.0, d_max=0.0, chunk=None):
    from paper_2305_08140_gb300 import nepzbl as N
    m = nep(precision)
    if chunk:
        m.set_option(N.NEP_OPT_GRAPH_CHUNK, chunk)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=dt,
                   d_max=d_max)
    m.md(st, nsteps)
    if chunk:
        m.set_option(N.NEP_OPT_GRAPH_CHUNK, 10)
    return st


def _min_image(d, box, pbc):
    return d - np.where(np.asarray(pbc) > 0, box * np.round(d / box), 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_c1_100_steps(precision):
    s = I.c1()
    st = _run_md(s, precision, 100, chunk=7)     # 7 + 7 + ... + 2: several graph lengths
    p, v, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 100)
    xg = st.xyz.cpu().numpy().T
    vg = st.vel.cpu().numpy().T
    dp = np.abs(_min_image(xg - p, s.box, s.pbc))
    if precision == "fp64":
        assert dp.max() < 1e-9
        assert np.abs(vg - v).max() < 1e-10
        assert st.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)
        assert st.kinetic_energy == pytest.approx(th[-1, 3], abs=1e-8)
    else:
        assert dp.max() < 2e-5
        assert abs(st.potential_energy - th[-1, 2]) / s.n < 2e-6
        assert abs(st.kinetic_energy - th[-1, 3]) / s.n < 2e-6
    assert st.step == 100 and st.time == pytest.approx(100.0)


def test_md_variable_timestep_fp64():
    s = I.c3(ncell=10, fraction=0.05, radius=6.0, seed=23)
    st = _run_md(s, "fp64", 20, dt=1.0, d_max=0.01, chunk=6)
    p, v, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 20, d_max=0.01)
    assert st.time == pytest.approx(th[:, 1].sum(), rel=1e-9)
    assert st.dt_last == pytest.approx(th[-1, 1], rel=1e-9)
    xg = st.xyz.cpu().numpy().T
    assert np.abs(_min_image(xg - p, s.box, s.pbc)).max() < 1e-8


def test_md_clump_fp32_tiles_split_between_kernels():
    """FP32 MD of a lattice holding a dense clump (pairs down to ~0.3 A): every
    step splits the tiles of 128 atoms between the plain Tensor-Memory angular
    kernel, its close-pair variant and the register kernel (tiles with more
    than 48 angular neighbours on an atom).  20 steps with variable dt
    (0.01 A per step) follow the oracle's trajectory; a second run on a fresh
    context repeats the first bitwise."""
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.c3(ncell=10, fraction=0.1, radius=6.0, seed=23)   # up to 85 angular neighbours
    runs = []
    for _ in range(2):
        m = N.NEP(I.nep_model(1), "fp32")
        m.set_option(N.NEP_OPT_GRAPH_CHUNK, 6)
        st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc,
                       dt_max=1.0, d_max=0.01)
        m.md(st, 20)
        runs.append((st.xyz.cpu().numpy().T.copy(), st.vel.cpu().numpy().T.copy(), st.time,
                     st.potential_energy, m.stats()))
        m.close()
    x1, v1, t1, e1, st1 = runs[0]
    x2, v2, t2, e2, _ = runs[1]
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and t1 == t2 and e1 == e2
    # the register kernel took the dense tiles, Tensor Memory the others
    assert 0 < st1["angular_tiles_register"] < st1["angular_tiles"], st1
    assert st1["angular_state_in_tmem"] == 1
    p, v, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 20, d_max=0.01)
    assert t1 == pytest.approx(th[:, 1].sum(), rel=1e-6)
    assert np.abs(_min_image(x1 - p, s.box, s.pbc)).max() < 1e-6


# ---------------------------------------------------------------------------
# Verlet skin: lists built with r_c + skin and reused; same trajectories
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_with_verlet_skin_matches_oracle(precision):
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.c1()
    m = N.NEP(I.nep_model(1), precision)
    m.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, 1000)
    m.set_option(N.NEP_OPT_GRAPH_CHUNK, 9)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    m.md(st, 100)
    builds = m.stats()["list_builds_skin"]
    assert 1 <= builds < 50, builds       # the lists were reused
    p, v, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 100)
    dp = np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc))
    if precision == "fp64":
        assert dp.max() < 1e-9
        assert st.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)
    else:
        assert dp.max() < 2e-5
        assert abs(st.potential_energy - th[-1, 2]) / s.n < 2e-6
    m.close()


def test_md_skin_variable_timestep_clump_fp64():
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.c3(ncell=10, fraction=0.05, radius=6.0, seed=23)
    m = N.NEP(I.nep_model(1), "fp64")
    m.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, 300)
    m.set_option(N.NEP_OPT_GRAPH_CHUNK, 7)
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                   d_max=0.01)
    m.md(st, 30)
    p, v, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 30, d_max=0.01)
    assert st.time == pytest.approx(th[:, 1].sum(), rel=1e-9)
    assert np.abs(_min_image(st.xyz.cpu().numpy().T - p, s.box, s.pbc)).max() < 1e-8
    assert m.stats()["list_builds_skin"] < 30
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_step_host_buffers(precision):
    """md_step_host with the state in (pinned and pageable) host memory: the
    same trajectory as md_step on device memory over calls of one and several
    steps -- bit for bit on the FP32 path (fixed-point force sums), to
    rounding on the FP64 path (its double atomics sum in any order) -- and
    the FP64 path also against the oracle."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.small_box((6, 6, 7), sigma=0.1, seed=31)
    s.vel = I.maxwell_boltzmann(np.random.default_rng(32), s.n, 600.0)
    m = nep(precision)
    dev = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    m.md(dev, 1)
    m.md(dev, 4)
    m.md(dev, 1)
    x = torch.tensor(np.ascontiguousarray(s.pos.T), dtype=torch.float64).pin_memory()
    v = torch.tensor(np.ascontiguousarray(s.vel.T), dtype=torch.float64)   # pageable
    host = N.MDState(x, v, s.box, s.pbc, dt_max=1.0)
    assert not host.xyz.is_cuda and not host.forces.is_cuda
    m.md_host(host, 1)
    m.md_host(host, 4)
    m.md_host(host, 1)
    assert host.step == dev.step == 6
    same = (lambda a, b, tol: np.array_equal(a, b)) if precision == "fp32" else \
        (lambda a, b, tol: np.max(np.abs(a - b)) <= tol)
    assert same(host.xyz.numpy(), dev.xyz.cpu().numpy(), 1e-12)
    assert same(host.vel.numpy(), dev.vel.cpu().numpy(), 1e-15)
    assert same(host.forces.numpy(), dev.forces.cpu().numpy(), 1e-11)
    assert same(np.array([host.potential_energy, host.kinetic_energy]),
                np.array([dev.potential_energy, dev.kinetic_energy]), 1e-10)
    if precision == "fp64":
        p, vo, F, th = O.md(I.nep_model(1), s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 6)
        assert np.abs(_min_image(host.xyz.numpy().T - p, s.box, s.pbc)).max() < 1e-9
        assert np.abs(host.forces.numpy().T - F).max() < 1e-9
        assert host.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)


def test_md_step_host_rejects_device_arrays():
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.small_box((6, 6, 6), sigma=0.05, seed=33)
    m = nep("fp32")
    dev = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    with pytest.raises(N.NepError, match="md_step_host takes host arrays"):
        m.md_host(dev, 1)


def test_angular_kernel_dispatch_both_paths():
    """FP32, one species: the angular kernel keeps its per-atom state in Tensor
    Memory except in the tiles (128 cell-ordered atoms) with an atom of more
    than 48 angular neighbours or a pair inside the outer ZBL radius, which the
    register kernel takes (the choice is made on the device, tile by tile, from
    this evaluation's neighbour pass).  A lattice and a dense clump in a
    lattice, alternately, on one context: the lattice runs wholly in Tensor
    Memory, the clump's box in both kernels; both match the oracle (the clump
    with the per-atom rounding bounds) and repeats are bitwise equal."""
    from paper_2305_08140_gb300 import nepzbl as N
    from gpu_common import F32_E_PER_ATOM, F32_F, F32_W_PER_ATOM, check_sites, site_bound
    m = N.NEP(I.nep_model(1), "fp32")
    lat = I.small_box((6, 6, 7), sigma=0.1, seed=51)
    clump = I.c3(ncell=10, fraction=0.1, radius=6.0, seed=23)   # up to 85 angular neighbours
    Eo, Fo, Wo, Uo = oracle_eval(lat)
    outs = {}
    for s in (lat, clump, lat, clump):
        E, F, W, U = m.compute(N.to_device_soa(s.pos), s.box, s.pbc, site_energy=True)
        st = m.stats()
        tiles = (s.n + 127) // 128
        assert st["angular_tiles"] == tiles
        assert st["angular_state_in_tmem"] == 1
        if s is lat:
            assert st["angular_tiles_register"] == 0
        else:
            assert 0 < st["angular_tiles_register"] < tiles, st["angular_tiles_register"]
        assert (st["max_nbr_angular"] > 48) == (s is clump)
        F = F.cpu().numpy().T
        assert np.all(np.isfinite(F))
        if s is lat:
            assert np.max(np.abs(F - Fo)) <= F32_F
            assert abs(E - Eo) / s.n <= F32_E_PER_ATOM
            check_sites(U.cpu().numpy(), Uo, site_bound("fp32", Uo))
            assert np.max(np.abs(W - Wo)) / s.n <= F32_W_PER_ATOM
        outs.setdefault(id(s), []).append((E, F))
    for s in (lat, clump):
        (E1, F1), (E2, F2) = outs[id(s)]
        assert E1 == E2 and np.array_equal(F1, F2)
    m.close()
    # the clump, its tiles split between the two kernels, against the oracle
    assert_parity(clump, "fp32", scaled=True)


@pytest.mark.parametrize("precision,skin", [("fp32", 0), ("fp64", 0), ("fp32", 500)])
def test_md_neighbour_overflow_rolls_back_and_replays(precision, skin):
    """md_step on a context whose neighbour capacity (8 slots) is far below the
    58 radial neighbours of bcc W: the first graph chunk overflows, is rolled
    back (x, v, F and the thermo block restored), the capacity grows and the
    chunk is replayed.  The trajectory equals that of a context with ample
    capacity -- bit for bit on the FP32 path (fixed-point force sums), to
    rounding on the FP64 path (double atomics) -- and, on the FP64 path, the
    oracle's velocity Verlet."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.c1()
    model = I.nep_model(1)
    ample = N.NEP(model, precision)
    tight = N.NEP(model, precision)
    tight.set_option(N.NEP_OPT_NBR_CAPACITY, 8)
    for m in (ample, tight):
        m.set_option(N.NEP_OPT_GRAPH_CHUNK, 5)
        if skin:
            m.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, skin)
    x0 = N.to_device_soa(s.pos)
    E0, F0, W0, U0 = ample.compute(x0.clone(), s.box, s.pbc)
    states = []
    for m in (ample, tight):
        st = N.MDState(x0.clone(), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                       forces=F0.clone())
        m.md(st, 12)
        states.append(st)
    a, b = states
    cap = tight.stats()["nbr_capacity"]
    assert cap >= 58 * (1.0 + skin / 6000.0) ** 3, cap   # grew past the bcc count
    assert a.step == b.step == 12 and a.time == b.time
    if precision == "fp32":
        for name in ("xyz", "vel", "forces"):
            assert torch.equal(getattr(a, name), getattr(b, name)), name
        assert a.potential_energy == b.potential_energy
        assert a.kinetic_energy == b.kinetic_energy
    else:
        for name, tol in (("xyz", 1e-12), ("vel", 1e-14), ("forces", 1e-10)):
            d = (getattr(a, name) - getattr(b, name)).abs().max().item()
            assert d <= tol, (name, d)
        p, v, F, th = O.md(model, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 12)
        xg = b.xyz.cpu().numpy().T
        assert np.abs(_min_image(xg - p, s.box, s.pbc)).max() < 1e-9
        assert b.potential_energy == pytest.approx(th[-1, 2], abs=1e-8)
    ample.close()
    tight.close()
