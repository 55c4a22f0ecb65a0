"""nep_compute_static: the force evaluation for callers that cannot allocate
GPU memory when they need forces (a plugin in a host program that owns all
device memory through its own pool or budget).  Its scratch is a fixed device
array inside the library.  Called through the C ABI and compared with
nep_compute, on two calls in a row (the array keeps the previous call's
contents, so the second call checks that what must start at zero is
cleared)."""
import ctypes as C

import numpy as np
import pytest

from paper_2305_08140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the FP32 tolerances of the parity tests
F_TOL = 1e-4
E_TOL_PER_ATOM = 1e-6
W_TOL_PER_ATOM = 2e-5
U_TOL = 2e-6


def _params_struct(model):
    from paper_2305_08140_gb300 import nepzbl as N
    keep = (np.ascontiguousarray(model.params, dtype=np.float64),
            np.ascontiguousarray(model.scaler, dtype=np.float64))
    p = N.NepParams()
    p.n_types = 1
    p.z[0] = int(model.zs[0])
    p.mass[0] = I.MASS_W
    p.rc_radial, p.rc_angular = model.rc_radial, model.rc_angular
    p.zbl_r_inner, p.zbl_r_outer = model.zbl_r_inner, model.zbl_r_outer
    p.n_max_radial, p.n_max_angular = model.n_max_radial, model.n_max_angular
    p.basis_size_radial, p.basis_size_angular = model.basis_size_radial, model.basis_size_angular
    p.l_max, p.use_4body, p.n_hidden = model.l_max, model.use_4body, model.n_hidden
    p.params = keep[0].ctypes.data_as(C.POINTER(C.c_double))
    p.n_params = len(keep[0])
    p.q_scaler = keep[1].ctypes.data_as(C.POINTER(C.c_double))
    return p, keep


def _static_eval(lib, p, s):
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    x = N.to_device_soa(s.pos)
    types = torch.zeros(s.n, dtype=torch.int32, device="cuda")
    F = torch.full((3, s.n), float("nan"), dtype=torch.float64, device="cuda")
    U = torch.empty(s.n, dtype=torch.float64, device="cuda")
    box = np.ascontiguousarray(np.diag(s.box).reshape(9))
    E = C.c_double()
    W = (C.c_double * 9)()
    rc = lib.nep_compute_static(C.byref(p), s.n, C.c_void_p(x.data_ptr()),
                                box.ctypes.data_as(C.POINTER(C.c_double)),
                                C.c_void_p(types.data_ptr()), (C.c_int32 * 3)(*s.pbc),
                                C.byref(E), C.c_void_p(F.data_ptr()), W, C.c_void_p(U.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.nep_last_error(None).decode()
    return E.value, F.cpu().numpy().T, np.array(W[:]).reshape(3, 3), U.cpu().numpy()


def test_static_scratch_matches_nep_compute_twice():
    from paper_2305_08140_gb300 import nepzbl as N
    lib = N.load()
    model = I.nep_model(1)
    p, keep = _params_struct(model)
    ref = N.NEP(model, "fp32")
    cases = [I.small_box((6, 6, 7), sigma=0.1, seed=61),      # 504 atoms, periodic
             I.displaced(I.c5(ncell=8, vacuum=10.0), 0.05, 62)]  # 1024 atoms, open z
    for s in cases:
        E0, F0, W0, U0 = ref.compute(N.to_device_soa(s.pos), s.box, s.pbc, site_energy=True)
        F0 = F0.cpu().numpy().T
        U0 = U0.cpu().numpy()
        for _ in range(2):
            E, F, W, U = _static_eval(lib, p, s)
            assert np.all(np.isfinite(F))
            assert np.max(np.abs(F - F0)) <= F_TOL
            assert abs(E - E0) / s.n <= E_TOL_PER_ATOM
            assert np.max(np.abs(W - W0)) / s.n <= W_TOL_PER_ATOM
            assert np.max(np.abs(U - U0)) <= U_TOL
    ref.close()


def test_static_scratch_rejects_too_many_atoms():
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    lib = N.load()
    p, keep = _params_struct(I.nep_model(1))
    n = 8193
    dummy = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    types = torch.zeros(n, dtype=torch.int32, device="cuda")
    box = np.ascontiguousarray(np.diag([100.0, 100.0, 100.0]).reshape(9))
    E = C.c_double()
    rc = lib.nep_compute_static(C.byref(p), n, C.c_void_p(dummy.data_ptr()),
                                box.ctypes.data_as(C.POINTER(C.c_double)),
                                C.c_void_p(types.data_ptr()), (C.c_int32 * 3)(1, 1, 1),
                                C.byref(E), C.c_void_p(dummy.data_ptr()), None, None, None)
    assert rc == N.NEP_ERR_INVALID_ARG
    assert "8192" in lib.nep_last_error(None).decode()


def test_static_scratch_rejects_host_site_energy():
    """A host array passed as site_energy is refused before any GPU work (the
    kernels would store to it): NEP_ERR_INVALID_ARG, naming the argument.  No
    kernel runs on the bad pointer, and a valid call afterwards still works."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    lib = N.load()
    model = I.nep_model(1)
    p, keep = _params_struct(model)
    s = I.small_box((6, 6, 7), sigma=0.1, seed=63)
    x = N.to_device_soa(s.pos)
    types = torch.zeros(s.n, dtype=torch.int32, device="cuda")
    F = torch.zeros((3, s.n), dtype=torch.float64, device="cuda")
    U_host = np.zeros(s.n)
    box = np.ascontiguousarray(np.diag(s.box).reshape(9))
    E = C.c_double()
    rc = lib.nep_compute_static(C.byref(p), s.n, C.c_void_p(x.data_ptr()),
                                box.ctypes.data_as(C.POINTER(C.c_double)),
                                C.c_void_p(types.data_ptr()), (C.c_int32 * 3)(*s.pbc),
                                C.byref(E), C.c_void_p(F.data_ptr()), None,
                                C.c_void_p(U_host.ctypes.data),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == N.NEP_ERR_INVALID_ARG
    assert "site_energy" in lib.nep_last_error(None).decode()
    assert np.all(U_host == 0.0)
    E1, F1, W1, U1 = _static_eval(lib, p, s)
    assert np.all(np.isfinite(F1)) and np.isfinite(E1)
