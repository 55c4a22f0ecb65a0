"""Shared helpers of the GPU tests: run the CUDA library and the oracle on the
same seeded structure and compare."""
import numpy as np

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

# Tolerances.  FP32 path (spec bounds): max |dF| <= 1e-4 eV/A and
# |dE|/N <= 1e-6 eV.  Site energies: FP32 rounding of a 30-term tanh network
# whose inputs carry ~1e-7 relative error -> 2e-6 eV per atom.  Virial: the sum
# of ~60 FP32 pair terms f (x) d per atom -> 2e-5 eV per atom.
F32_F = 1e-4
F32_E_PER_ATOM = 1e-6
F32_U = 2e-6
F32_W_PER_ATOM = 2e-5
# FP64 path: same arithmetic as the oracle up to summation order.
F64_F = 1e-9
F64_E_PER_ATOM = 1e-11
F64_U = 1e-10
F64_W_PER_ATOM = 1e-10

_NEP = {}


def nep(precision="fp32", seed=1):
    from paper_2305_08140_gb300 import nepzbl as N
    key = (precision, seed)
    if key not in _NEP:
        _NEP[key] = N.NEP(I.nep_model(seed), precision)
    return _NEP[key]


def gpu_eval(s, precision="fp32", site=True, seed=1):
    from paper_2305_08140_gb300 import nepzbl as N
    x = N.to_device_soa(s.pos)
    E, F, W, U = nep(precision, seed).compute(x, s.box, s.pbc, site_energy=site)
    F = F.cpu().numpy().T.copy()
    return E, F, W, (U.cpu().numpy() if U is not None else None)


def oracle_eval(s, seed=1):
    return O.energy_forces_virial(I.nep_model(seed), s.pos, s.box, s.pbc)


def assert_parity(s, precision="fp32", seed=1, rel_force=0.0):
    """Element-by-element comparison of E, F, W and U_i."""
    E, F, W, U = gpu_eval(s, precision, seed=seed)
    Eo, Fo, Wo, Uo = oracle_eval(s, seed)
    n = s.n
    if precision == "fp32":
        tf, te, tu, tw = F32_F, F32_E_PER_ATOM, F32_U, F32_W_PER_ATOM
    else:
        tf, te, tu, tw = F64_F, F64_E_PER_ATOM, F64_U, F64_W_PER_ATOM
    dF = np.abs(F - Fo)
    bound = tf + rel_force * np.linalg.norm(Fo, axis=1, keepdims=True)
    worst = np.unravel_index(np.argmax(dF - bound), dF.shape)
    assert np.all(dF <= bound), (f"max |dF| {dF.max():.3e} at {worst}: gpu {F[worst]} "
                                 f"oracle {Fo[worst]}")
    assert abs(E - Eo) / n <= te, (E, Eo, abs(E - Eo) / n)
    assert np.max(np.abs(U - Uo)) <= tu + rel_force * np.max(np.abs(Uo)), np.max(np.abs(U - Uo))
    assert np.max(np.abs(W - Wo)) / n <= tw, (W, Wo)
    return E, F, W, U, Eo, Fo, Wo, Uo
