"""Checkpoint files of an MD state on the host (no GPU): every field survives
the round trip, and a checkpoint is refused for another model -- a change of
any part of the potential (parameters, scaler, cutoffs, ZBL radii, species,
sizes) is detected."""
import copy

import numpy as np
import pytest

from paper_2305_08140_gb300 import inputs as I


def test_checkpoint_round_trip_on_host(tmp_path):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.small_box((6, 6, 7), sigma=0.1, seed=71)
    rng = np.random.default_rng(72)
    x = torch.tensor(s.pos.T.copy())
    v = torch.tensor(rng.normal(size=(3, s.n)))
    F = torch.tensor(rng.normal(size=(3, s.n)))
    types = torch.tensor(rng.integers(0, 2, s.n), dtype=torch.int32)
    box = np.array([[s.box[0], 0.0, 0.0], [0.5, s.box[1], 0.0], [0.0, 0.3, s.box[2]]])
    st = N.MDState(x, v, box, [1, 1, 0], dt_max=0.75, d_max=0.01, types=types, forces=F)
    st.c.time, st.c.step, st.c.dt_last = 12.5, 17, 0.625
    model = I.nep_model(1)
    path = str(tmp_path / "c.npz")
    N.save_checkpoint(path, st, model=model)
    r = N.load_checkpoint(path, device="cpu", model=model)
    for name in ("xyz", "vel", "forces", "types"):
        assert torch.equal(getattr(r, name), getattr(st, name)), name
    assert list(r.c.box) == list(st.c.box) and list(r.c.pbc) == [1, 1, 0]
    assert (r.c.dt_max, r.c.d_max, r.time, r.step, r.dt_last, r.c.forces_valid) == \
        (0.75, 0.01, 12.5, 17, 0.625, 1)
    # the struct points at the loaded tensors
    assert r.c.xyz == r.xyz.data_ptr() and r.c.forces == r.forces.data_ptr()
    N.load_checkpoint(path, device="cpu", model=copy.deepcopy(model))   # equal model: accepted
    N.load_checkpoint(path, device="cpu")          # no model given: not checked
    path2 = str(tmp_path / "nohash.npz")
    N.save_checkpoint(path2, st)
    with pytest.raises(ValueError):
        N.load_checkpoint(path2, device="cpu", model=model)


def _changed(model, what):
    m = copy.deepcopy(model)
    if what == "params":
        m.params = np.asarray(m.params) * (1.0 + 1e-12)
    elif what == "scaler":
        m.scaler = np.asarray(m.scaler).copy()
        m.scaler[3] *= 1.0 + 1e-12
    elif what == "species":
        m.species = ("Mo",)
    elif what == "n_hidden":
        m.n_hidden = 20
    else:
        setattr(m, what, getattr(m, what) + 1e-9)
    return m


@pytest.mark.parametrize("what", ["params", "scaler", "rc_radial", "rc_angular", "zbl_r_inner",
                                  "zbl_r_outer", "species", "n_hidden"])
def test_checkpoint_refused_for_another_model(tmp_path, what):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    s = I.small_box((6, 6, 6), sigma=0.05, seed=73)
    st = N.MDState(torch.tensor(s.pos.T.copy()), torch.zeros((3, s.n), dtype=torch.float64),
                   s.box, s.pbc)
    model = I.nep_model(1)
    path = str(tmp_path / "c.npz")
    N.save_checkpoint(path, st, model=model)
    with pytest.raises(ValueError, match="another model"):
        N.load_checkpoint(path, device="cpu", model=_changed(model, what))
