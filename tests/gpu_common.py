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

# Per-atom bounds where the benchmark spec's tolerances cannot be reached by
# construction (close pairs, clumps with ~7x the lattice neighbour count),
# from a first-order model of the FP32 rounding with u = 2^-24 and each atom's
# rounding-error scales from the oracle (oracle.force_scales; columns S, Z, W,
# SU, TU):
#   |dF_i| <= 1e-4 + u (C_PAIR S_i + C_NET W_i) + 2^-40 Z_i
#   |dU_i| <= 2e-6 + 1e-9 |U_i| + u (SU_i + C_SUM TU_i)
# * Each NEP pair term g_p (S_i = sum |g_p|) carries C_PAIR = 256 u relative
#   error from its own evaluation: its displacement (cell-relative FP32
#   coordinates, <= 2.1e-6 A absolute; pairs closer than 2 A come from FP64
#   positions) is <= 18 u relative at r >= 2 A, amplified <= 8x by the term's
#   dependence on it (harmonics of degree <= 4 over r, radial basis) = 144 u;
#   cutoff, Chebyshev recurrence, harmonics and the contraction ~32 u; FP32
#   rounding of the adjoint entries ~32 u: 208 u, rounded up to 256 u.
# * The descriptor sums of a site with M radial neighbours carry relative
#   rounding ~sqrt(M) u (accumulation of M FP32 terms), so each
#   pre-activation h_mu moves by up to sqrt(M) u sum_nu |w0 s q| and the
#   adjoint factor 1 - t^2 by a relative 2 |t dh| <= 2 |dh|: a pair term of
#   site k carries a further 2 sqrt(M_k) max_mu sum_nu |w0 s q_k| u of its
#   magnitude (W_i sums |g_p| times that conditioning, C_NET = 2).
# * The ZBL terms are FP64 on both paths; rounding them to the 2^-32 eV/A
#   fixed-point grid is ~2^-33 absolute per term (covered by 2^-40 Z_i + 1e-4).
# * U_i: the same pre-activation shifts move U by <= sqrt(M) u sum_mu |w1 (1 -
#   t^2)| sum_nu |w0 s q| (SU_i), the 30-term output sum adds C_SUM = 32 u of
#   its terms' magnitude (TU_i); the ZBL half-sums are FP64 (1e-9 |U_i|).
U32 = 2.0 ** -24
C_PAIR = 256.0
C_NET = 2.0
C_SUM = 32.0
F64_REL_SCALE = 1e-12   # FP64 path: relative to S_i + Z_i
U_REL64 = 1e-12

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


def force_bound(precision, sc=None):
    """Per-atom bound on |dF_i| (N, 1): the flat tolerance, plus, with the
    oracle's rounding-error scales ``sc`` (N, 5), the model above."""
    flat = F32_F if precision == "fp32" else F64_F
    if sc is None:
        return np.array([[flat]])
    S, Z, W = sc[:, 0], sc[:, 1], sc[:, 2]
    if precision == "fp32":
        b = flat + U32 * (C_PAIR * S + C_NET * W) + 2.0 ** -40 * Z
    else:
        b = flat + F64_REL_SCALE * (S + Z)
    return b[:, None]


def site_bound(precision, Uo, sc=None):
    """Per-atom bound on |dU_i|: flat, plus the model above with ``sc``."""
    if precision == "fp32":
        b = F32_U + 1e-9 * np.abs(Uo)
        if sc is not None:
            b = b + U32 * (sc[:, 3] + C_SUM * sc[:, 4])
        return b
    return F64_U + U_REL64 * np.abs(Uo)


def check_forces(F, Fo, bound, label=""):
    dF = np.abs(F - Fo)
    worst = np.unravel_index(np.argmax(dF - bound), dF.shape)
    assert np.all(dF <= bound), (f"{label} max |dF| {dF.max():.3e}, worst excess at {worst}: "
                                 f"gpu {F[worst]} oracle {Fo[worst]} bound {bound[worst[0], 0]:.3e}")


def check_sites(U, Uo, bound, label=""):
    dU = np.abs(U - Uo)
    worst = int(np.argmax(dU - bound))
    assert np.all(dU <= bound), (f"{label} |dU| {dU[worst]:.3e} at atom {worst}: gpu {U[worst]} "
                                 f"oracle {Uo[worst]} bound {bound[worst]:.3e}")


def assert_parity(s, precision="fp32", seed=1, scaled=False):
    """Element-by-element comparison of E, F, W and U_i.  ``scaled``: each
    atom's bounds follow the rounding model above (close pairs, clumps);
    otherwise the flat spec bounds."""
    E, F, W, U = gpu_eval(s, precision, seed=seed)
    Eo, Fo, Wo, Uo = oracle_eval(s, seed)
    n = s.n
    if precision == "fp32":
        te, tw = F32_E_PER_ATOM, F32_W_PER_ATOM
    else:
        te, tw = F64_E_PER_ATOM, F64_W_PER_ATOM
    sc = O.force_scales(I.nep_model(seed), s.pos, s.box, s.pbc) if scaled else None
    check_forces(F, Fo, force_bound(precision, sc))
    assert abs(E - Eo) / n <= te, (E, Eo, abs(E - Eo) / n)
    check_sites(U, Uo, site_bound(precision, Uo, sc))
    assert np.max(np.abs(W - Wo)) / n <= tw, (W, Wo)
    return E, F, W, U, Eo, Fo, Wo, Uo
