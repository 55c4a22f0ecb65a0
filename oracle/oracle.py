"""Python access to the FP64 CPU oracle (``nep_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``,
by the bench's CPU-baseline leg and by ``make_scaler.py``.  It never imports
the CUDA package; it reads only the seeded inputs module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libnep_oracle.so")
SRC = os.path.join(HERE, "nep_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/lib/."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(LIBDIR, exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_energy_forces_virial.argtypes = [ip, dp, dp, dp, C.c_int, dp, ip, dp, ip,
                                               C.c_int, dp, dp, dp, dp]
        L.orc_descriptors.argtypes = [ip, dp, dp, dp, C.c_int, dp, ip, dp, ip, C.c_int, dp]
        L.orc_forces_subset.argtypes = [ip, dp, dp, dp, C.c_int, dp, ip, dp, ip, C.c_int,
                                        C.POINTER(C.c_int64), dp, dp]
        L.orc_forces_subset_scales.argtypes = [ip, dp, dp, dp, C.c_int, dp, ip, dp, ip, C.c_int,
                                               C.POINTER(C.c_int64), dp, dp, dp]
        L.orc_force_scales.argtypes = [ip, dp, dp, dp, C.c_int, dp, ip, dp, ip, C.c_int, dp]
        L.orc_md.argtypes = [ip, dp, dp, dp, C.c_int, dp, dp, dp, C.c_int, ip, dp, ip,
                             dp, C.c_double, C.c_double, C.c_int, C.c_int, dp]
        L.orc_md_ext.argtypes = [ip, dp, dp, dp, C.c_int, dp, dp, dp, C.c_int, ip, dp, ip,
                                 dp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(C.c_uint8), dp, dp]
        L.orc_site.argtypes = [ip, dp, dp, dp, C.c_int, C.c_int, dp, ip, C.c_int, dp, ip,
                               dp, dp, dp, dp]
        L.orc_neighbor_counts.argtypes = [C.c_int, dp, dp, ip, C.c_double, C.c_int, ip,
                                          C.c_int, dp]
        L.orc_cutoff.argtypes = [C.c_double, C.c_double, dp, dp]
        L.orc_chebyshev.argtypes = [C.c_double, C.c_int, dp, dp]
        L.orc_basis.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp]
        L.orc_legendre.argtypes = [C.c_double, C.c_int, dp, dp]
        L.orc_zbl.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                              dp, dp]
        L.orc_fourbody_triple.argtypes = [C.c_int, dp, dp]
        L.orc_fourbody_triple.restype = C.c_double
        L.orc_n_params.argtypes = [ip]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _hp(model):
    ihp = np.array([model.n_max_radial + 1, model.n_max_angular + 1,
                    model.basis_size_radial + 1, model.basis_size_angular + 1,
                    model.l_max, model.use_4body, model.n_hidden, model.n_types],
                   dtype=np.int32)
    dhp = np.array([model.rc_radial, model.rc_angular, model.zbl_r_inner, model.zbl_r_outer,
                    *[float(z) for z in model.zs]], dtype=np.float64)
    return ihp, dhp


def _types(types, n):
    if types is None:
        return np.zeros(max(n, 1), np.int32)
    t = np.ascontiguousarray(types, dtype=np.int32)
    if t.shape != (n,):
        raise ValueError("types must have one entry per atom")
    return t if n > 0 else np.zeros(1, np.int32)


def _masses(model, mass):
    m = np.atleast_1d(np.asarray(mass, dtype=np.float64))
    if m.size == 1:
        m = np.full(model.n_types, float(m[0]))
    if m.size != model.n_types:
        raise ValueError("one mass per species")
    return np.ascontiguousarray(m)


# 1 eV/amu in A^2/fs^2 (CODATA e and u)
EV_PER_AMU = 1.602176634e-19 / 1.66053906660e-27 * 1e-10


def _box9(box):
    """Row-major 3x3 cell H from box lengths (3,) or a (3, 3) matrix."""
    b = np.asarray(box, dtype=np.float64)
    if b.shape == (3,):
        b = np.diag(b)
    return np.ascontiguousarray(b.reshape(9))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def energy_forces_virial(model, pos, box, pbc, use_grid=True, params=None, types=None):
    """E, F (N,3), W (3,3), U_site (N) of one system (``types``: species per
    atom, default all 0)."""
    ihp, dhp = _hp(model)
    p = _f64(model.params if params is None else params)
    s = _f64(model.scaler)
    pos = _f64(pos)
    n = pos.shape[0]
    t = _types(types, n)
    box = _box9(box)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    E = np.zeros(1)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    U = np.zeros(n)
    _check(lib().orc_energy_forces_virial(_i(ihp), _d(dhp), _d(p), _d(s), n, _d(pos), _i(t),
                                          _d(box), _i(pbc), int(use_grid), _d(E), _d(F), _d(W),
                                          _d(U)),
           "energy_forces_virial")
    return float(E[0]), F, W.reshape(3, 3), U


def descriptors(model, pos, box, pbc, use_grid=True, types=None):
    """Unscaled descriptors (N, D)."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler if model.scaler is not None else np.ones(model.dim))
    pos = _f64(pos)
    n = pos.shape[0]
    t = _types(types, n)
    q = np.zeros((n, model.dim))
    _check(lib().orc_descriptors(_i(ihp), _d(dhp), _d(p), _d(s), n, _d(pos), _i(t),
                                 _d(_box9(box)), _i(np.ascontiguousarray(pbc, dtype=np.int32)),
                                 int(use_grid), _d(q)), "descriptors")
    return q


# columns of the rounding-error scales (orc_force_scales in nep_oracle.c)
SCALE_COLUMNS = ("S", "Z", "W", "SU", "TU")


def forces_subset(model, pos, box, pbc, idx, types=None, scales=False):
    """Forces (len(idx), 3) and site energies (len(idx)) of the listed atoms;
    with ``scales`` also their rounding-error scales (len(idx), 5), columns
    SCALE_COLUMNS (see force_scales)."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler)
    pos = _f64(pos)
    t = _types(types, pos.shape[0])
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((len(idx), 3))
    U = np.zeros(len(idx))
    sc = np.zeros((max(len(idx), 1), 5))
    _check(lib().orc_forces_subset_scales(
        _i(ihp), _d(dhp), _d(p), _d(s), pos.shape[0], _d(pos), _i(t), _d(_box9(box)),
        _i(np.ascontiguousarray(pbc, dtype=np.int32)), len(idx),
        idx.ctypes.data_as(C.POINTER(C.c_int64)), _d(F), _d(U), _d(sc)), "forces_subset")
    return (F, U, sc[:len(idx)]) if scales else (F, U)


def force_scales(model, pos, box, pbc, types=None, use_grid=True):
    """Rounding-error scales of every atom, (N, 5), columns SCALE_COLUMNS:
    S, the sum of the magnitudes |dU_i/dd_ij| of the NEP pair terms that enter
    its force; Z, the same over the ZBL pair terms; W, the NEP terms'
    magnitudes each weighted by sqrt(M_k) max_mu sum_nu |w0_{mu nu} s_nu
    q_{k nu}| of the atom k whose site energy it differentiates (M_k radial
    neighbours); SU, sqrt(M_i) sum_mu |w1_mu (1 - t_mu^2)| sum_nu |w0 s q_i|;
    TU, sum_mu |w1_mu t_mu| + |b1|."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler)
    pos = _f64(pos)
    n = pos.shape[0]
    t = _types(types, n)
    sc = np.zeros((max(n, 1), 5))
    _check(lib().orc_force_scales(_i(ihp), _d(dhp), _d(p), _d(s), n, _d(pos), _i(t),
                                  _d(_box9(box)), _i(np.ascontiguousarray(pbc, dtype=np.int32)),
                                  int(use_grid), _d(sc)), "force_scales")
    return sc[:n]


def site(model, dR, dA, ti=0, tR=None, tA=None):
    """U^NEP, q (unscaled), dU/dd for radial and angular neighbour lists of one
    atom of species ``ti`` (neighbour species ``tR``, ``tA``, default 0)."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler)
    dR = _f64(np.reshape(dR, (-1, 3)))
    dA = _f64(np.reshape(dA, (-1, 3)))
    tR = _types(tR, dR.shape[0])
    tA = _types(tA, dA.shape[0])
    U = np.zeros(1)
    q = np.zeros(model.dim)
    gR = np.zeros_like(dR)
    gA = np.zeros_like(dA)
    _check(lib().orc_site(_i(ihp), _d(dhp), _d(p), _d(s), int(ti), dR.shape[0], _d(dR), _i(tR),
                          dA.shape[0], _d(dA), _i(tA), _d(U), _d(q), _d(gR), _d(gA)), "site")
    return float(U[0]), q, gR, gA


def md(model, pos, vel, box, pbc, mass, dt_max, nsteps, d_max=0.0, forces=None,
       use_grid=True, types=None):
    """Velocity-Verlet NVE; returns (pos, vel, forces, thermo[nsteps, 4]).
    ``mass``: one value, or one per species."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler)
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    n = pos.shape[0]
    t = _types(types, n)
    F = np.zeros((n, 3)) if forces is None else _f64(forces).copy()
    thermo = np.zeros((nsteps, 4))
    _check(lib().orc_md(_i(ihp), _d(dhp), _d(p), _d(s), n, _d(pos), _d(vel), _d(F),
                        0 if forces is None else 1, _i(t), _d(_box9(box)),
                        _i(np.ascontiguousarray(pbc, dtype=np.int32)), _d(_masses(model, mass)),
                        float(dt_max), float(d_max), int(nsteps), int(use_grid), _d(thermo)),
           "md")
    return pos, vel, F, thermo


def neighbor_counts(pos, box, pbc, rc, mode=0, maxn=0):
    """Per-atom neighbour counts within rc (mode 0 brute force, 1 cell grid)
    and, if maxn > 0, the sorted neighbour distances (N, maxn)."""
    pos = _f64(pos)
    n = pos.shape[0]
    counts = np.zeros(n, np.int32)
    dist = np.zeros((n, max(maxn, 1)))
    _check(lib().orc_neighbor_counts(n, _d(pos), _d(_box9(box)),
                                     _i(np.ascontiguousarray(pbc, dtype=np.int32)), float(rc),
                                     int(mode), _i(counts), int(maxn),
                                     _d(dist) if maxn > 0 else None), "neighbor_counts")
    return counts, (dist if maxn > 0 else None)


def cutoff(r, rc):
    fc, dfc = np.zeros(1), np.zeros(1)
    lib().orc_cutoff(float(r), float(rc), _d(fc), _d(dfc))
    return float(fc[0]), float(dfc[0])


def chebyshev(x, K):
    T, dT = np.zeros(K), np.zeros(K)
    lib().orc_chebyshev(float(x), int(K), _d(T), _d(dT))
    return T, dT


def basis(r, rc, K):
    f, df = np.zeros(K), np.zeros(K)
    lib().orc_basis(float(r), float(rc), int(K), _d(f), _d(df))
    return f, df


def legendre(x, lmax):
    P, dP = np.zeros(lmax + 1), np.zeros(lmax + 1)
    lib().orc_legendre(float(x), int(lmax), _d(P), _d(dP))
    return P, dP


def zbl(r, Zi=74.0, Zj=74.0, r1=1.0, r2=2.0):
    U, dU = np.zeros(1), np.zeros(1)
    lib().orc_zbl(float(r), float(Zi), float(Zj), float(r1), float(r2), _d(U), _d(dU))
    return float(U[0]), float(dU[0])


def fourbody_triple(g, u):
    g = _f64(g)
    u = _f64(np.reshape(u, (-1, 3)))
    return float(lib().orc_fourbody_triple(len(g), _d(g), _d(u)))


# 1 eV/A^3 in GPa (CODATA e)
EV_A3_GPA = 160.21766208


def md_ext(model, pos, vel, box, pbc, mass, dt_max, nsteps, d_max=0.0, forces=None,
           use_grid=True, types=None, thermostat=None, barostat=None):
    """Velocity Verlet with a Nose-Hoover chain thermostat on a group and a
    Berendsen barostat (``orc_md_ext``).  thermostat = dict(T (K), tau (fs),
    chain, group (N bools) or None); barostat = dict(p0 (GPa), tau (fs), beta
    (1/GPa)).  Returns (pos, vel, forces, thermo[nsteps, 8], box)."""
    ihp, dhp = _hp(model)
    p = _f64(model.params)
    s = _f64(model.scaler)
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    diag = np.asarray(box).shape == (3,)
    box = _box9(box).copy()
    n = pos.shape[0]
    t = _types(types, n)
    F = np.zeros((n, 3)) if forces is None else _f64(forces).copy()
    thermo = np.zeros((nsteps, 8))
    ext = np.zeros(6)
    group = None
    if thermostat is not None:
        ext[0], ext[1], ext[2] = thermostat["T"], thermostat["tau"], thermostat.get("chain", 4)
        if thermostat.get("group") is not None:
            group = np.ascontiguousarray(thermostat["group"], dtype=np.uint8)
    if barostat is not None:
        ext[3] = barostat["p0"] / EV_A3_GPA
        ext[4] = barostat["tau"]
        ext[5] = barostat["beta"] * EV_A3_GPA
    _check(lib().orc_md_ext(_i(ihp), _d(dhp), _d(p), _d(s), n, _d(pos), _d(vel), _d(F),
                            0 if forces is None else 1, _i(t), _d(box),
                            _i(np.ascontiguousarray(pbc, dtype=np.int32)), _d(_masses(model, mass)),
                            float(dt_max), float(d_max), int(nsteps), int(use_grid),
                            1 if thermostat is not None else 0,
                            group.ctypes.data_as(C.POINTER(C.c_uint8)) if group is not None
                            else None, _d(ext), _d(thermo)), "md_ext")
    box = box.reshape(3, 3)
    return pos, vel, F, thermo, (np.diag(box).copy() if diag else box)


def min_image(d, box, pbc):
    """Displacements (M, 3) reduced to the nearest image along each periodic
    lattice direction (fractional rounding)."""
    H = _box9(box).reshape(3, 3)
    d = np.array(d, dtype=np.float64, copy=True)
    f = d @ np.linalg.inv(H)
    per = np.asarray(pbc) > 0
    f[:, per] -= np.round(f[:, per])
    return f @ H


def pka_atom(pos, box, pbc, point):
    """Index of the atom nearest to ``point`` (minimum image in periodic
    dimensions; ties to the lowest index)."""
    d = np.asarray(pos, dtype=np.float64) - np.asarray(point, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    per = np.asarray(pbc) > 0
    if box.shape == (3,):
        d[:, per] -= box[per] * np.round(d[:, per] / box[per])
    else:
        d = min_image(d, box, pbc)
    return int(np.argmin(np.einsum("ij,ij->i", d, d)))


def pka_velocity(energy_ev, mass_amu, direction):
    """Velocity (A/fs) of kinetic energy ``energy_ev`` along ``direction``."""
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    return np.sqrt(2.0 * energy_ev / mass_amu * EV_PER_AMU) * u
