"""Checkpoint and resume of an MD state (binding level, numpy .npz): a run
resumed from a checkpoint in a fresh context continues bit for bit like the
uninterrupted run (FP32 path: fixed-point force sums, deterministic kernels),
with a fixed and with a variable time step; a checkpoint written with another
model is refused."""
import numpy as np
import pytest

from paper_2305_08140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d_max", [0.0, 0.01])
def test_resume_is_bitwise_equal(tmp_path, d_max):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    model = I.nep_model(1)
    s = I.c1()
    a = N.NEP(model, "fp32")
    st = N.MDState(N.to_device_soa(s.pos), N.to_device_soa(s.vel), s.box, s.pbc, dt_max=1.0,
                   d_max=d_max)
    a.md(st, 7)
    path = str(tmp_path / "state.npz")
    N.save_checkpoint(path, st, model=model)
    a.md(st, 9)
    a.close()
    b = N.NEP(model, "fp32")
    r = N.load_checkpoint(path, model=model)
    assert r.step == 7 and r.c.forces_valid == 1
    b.md(r, 9)
    assert r.step == st.step == 16 and r.time == st.time
    for name in ("xyz", "vel", "forces"):
        assert torch.equal(getattr(r, name), getattr(st, name)), name
    assert r.potential_energy == st.potential_energy
    assert r.kinetic_energy == st.kinetic_energy
    other = I.nep_model(1)
    other.params = np.asarray(model.params) * (1.0 + 1e-12)
    with pytest.raises(ValueError):
        N.load_checkpoint(path, model=other)
    b.close()
