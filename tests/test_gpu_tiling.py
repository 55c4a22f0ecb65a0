"""Neighbour-search tiling (z slices per cell, candidate chunk width) and the
MD autotuner: every tiling finds the same pairs (it only skips candidates
beyond the list cutoff and reorders a cell's part of each list), so energies
and forces agree to rounding and the pair counts exactly; the autotuner times
the candidates on a state without changing it."""
import numpy as np
import pytest

from paper_2305_08140_gb300 import inputs as I

from gpu_common import F32_F, F64_F, oracle_eval

pytestmark = pytest.mark.gpu

TILINGS = [(1, 16), (1, 4), (2, 8), (4, 4), (4, 8), (8, 16)]


def _structures():
    return {
        "lattice": I.displaced(I.small_box((8, 8, 9)), 0.1, 81),
        "clump": I.c3(ncell=10, fraction=0.05, radius=6.0, seed=23),
        "open_z_slab": I.displaced(I.c5(ncell=8, vacuum=10.0), 0.05, 82),
    }


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["lattice", "clump", "open_z_slab"])
def test_every_tiling_finds_the_same_pairs(precision, name):
    from paper_2305_08140_gb300 import nepzbl as N
    s = _structures()[name]
    if name == "open_z_slab":
        # atoms beyond the open extent (clamped into the edge cells and slices)
        s.pos[0, 2] = -7.5
        s.pos[1, 2] = s.box[2] + 9.0
        s.pos[2] = s.pos[1] + np.array([1.1, 0.4, -0.3])
    m = N.NEP(I.nep_model(1), precision)
    ref = None
    for zs, chw in TILINGS:
        m.set_option(N.NEP_OPT_NBR_SLICES, zs)
        m.set_option(N.NEP_OPT_NBR_CHUNK, chw)
        E, F, W, U = m.compute(N.to_device_soa(s.pos), s.box, s.pbc, site_energy=True)
        st = m.stats()
        out = (E, F.cpu().numpy().T, W, U.cpu().numpy(),
               (st["pairs_radial"], st["pairs_angular"], st["max_nbr_radial"],
                st["max_nbr_angular"]))
        if ref is None:
            ref = out
            continue
        assert out[4] == ref[4], (zs, chw, out[4], ref[4])   # the same pairs
        tol = 1e-11 if precision == "fp64" else 2e-5
        assert abs(out[0] - ref[0]) / s.n <= (1e-13 if precision == "fp64" else 1e-7)
        np.testing.assert_allclose(out[1], ref[1], rtol=0, atol=tol * max(1.0, np.abs(ref[1]).max()))
    if name == "lattice":
        Eo, Fo, Wo, Uo = oracle_eval(s)
        assert np.max(np.abs(ref[1] - Fo)) <= (F64_F if precision == "fp64" else F32_F)
    m.close()


def test_tiling_options_rejected_out_of_range():
    from paper_2305_08140_gb300 import nepzbl as N
    m = N.NEP(I.nep_model(1), "fp32")
    for opt, bad in ((N.NEP_OPT_NBR_SLICES, 3), (N.NEP_OPT_NBR_SLICES, 16),
                     (N.NEP_OPT_NBR_CHUNK, 32), (N.NEP_OPT_NBR_CHUNK, 0)):
        with pytest.raises(N.NepError) as e:
            m.set_option(opt, bad)
        assert e.value.code == N.NEP_ERR_INVALID_ARG
    m.close()


def test_md_autotune_times_candidates_and_leaves_the_state():
    """nep_md_autotune on the 128,000-atom crystal: 12 tilings and 3 graph
    chunks timed, the fastest kept; the caller's state is bitwise unchanged;
    MD afterwards matches a run with the default options to FP32 rounding."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.c2()
    m = N.NEP(I.nep_model(1), "fp32")
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0)
    x0, v0, f0 = st.xyz.clone(), st.vel.clone(), st.forces.clone()
    res = m.md_autotune(st, reps=2)
    rows, kept = res["tiling"]
    assert len(rows) == 12 and kept is not None
    assert {(r["z_slices"], r["chunk_width"]) for r in rows} == \
        {(a, b) for a in (1, 2, 4, 8) for b in (4, 8, 16)}
    assert all(r["ms"] > 0 for r in rows)
    assert kept["ms"] == min(r["ms"] for r in rows)
    crows, ckept = res["graph_chunk"]
    assert [r["steps_per_graph"] for r in crows] == [10, 25, 50]
    assert ckept["ms"] == min(r["ms"] for r in crows)
    assert m.stats()["graph_chunk"] == ckept["steps_per_graph"]
    assert torch.equal(st.xyz, x0) and torch.equal(st.vel, v0) and torch.equal(st.forces, f0)
    assert st.step == 0
    m.md(st, 20)
    d = N.NEP(I.nep_model(1), "fp32")
    sd = N.MDState(x0.clone(), v0.clone(), s.box, s.pbc, dt_max=1.0)
    d.md(sd, 20)
    assert (st.xyz - sd.xyz).abs().max().item() < 1e-5
    assert abs(st.potential_energy - sd.potential_energy) / s.n < 1e-6
    m.close()
    d.close()
