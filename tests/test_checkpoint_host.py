"""Checkpoint files of an MD state on the host (no GPU): every field survives
the round trip, and a checkpoint is refused for other model parameters."""
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
    params = I.nep_model(1).params
    path = str(tmp_path / "c.npz")
    N.save_checkpoint(path, st, params=params)
    r = N.load_checkpoint(path, device="cpu", params=params)
    for name in ("xyz", "vel", "forces", "types"):
        assert torch.equal(getattr(r, name), getattr(st, name)), name
    assert list(r.c.box) == list(st.c.box) and list(r.c.pbc) == [1, 1, 0]
    assert (r.c.dt_max, r.c.d_max, r.time, r.step, r.dt_last, r.c.forces_valid) == \
        (0.75, 0.01, 12.5, 17, 0.625, 1)
    # the struct points at the loaded tensors
    assert r.c.xyz == r.xyz.data_ptr() and r.c.forces == r.forces.data_ptr()
    other = np.asarray(params) * (1.0 + 1e-12)
    with pytest.raises(ValueError):
        N.load_checkpoint(path, device="cpu", params=other)
    N.load_checkpoint(path, device="cpu")          # no parameters given: not checked
    path2 = str(tmp_path / "nohash.npz")
    N.save_checkpoint(path2, st)
    with pytest.raises(ValueError):
        N.load_checkpoint(path2, device="cpu", params=params)
