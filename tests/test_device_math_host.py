"""CPU tests of the CUDA path's per-pair math (nep_math.cuh compiled for the
host): the addition theorem of its real harmonics, their gradients, the
Chebyshev recurrence and the l = 2 <-> 4-body tensor map.  These check the
library's own building blocks (not the oracle)."""
import ctypes as C
import math
import os
import subprocess

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "nep_math_host.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("nepmath") / "libnep_math_host.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, SRC])
    L = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    L.h_harmonics.argtypes = [C.c_double] * 3 + [dp]
    L.h_harmonics_grad_dot.argtypes = [C.c_double] * 3 + [dp, dp]
    L.h_fourbody.argtypes = [dp, dp]
    L.h_fourbody.restype = C.c_double
    L.h_cheb9.argtypes = [C.c_double, C.c_double, dp, dp, dp]
    return L


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def Y(lib, v):
    out = np.zeros(24)
    lib.h_harmonics(*[float(t) for t in v], _p(out))
    return out


L_OF = np.array([1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)


def test_addition_theorem(lib):
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        v = rng.normal(size=3); v /= np.linalg.norm(v)
        yu, yv = Y(lib, u), Y(lib, v)
        c = u @ v
        for l in range(1, 5):
            coef = np.zeros(l + 1); coef[l] = 1
            assert np.sum(yu[L_OF == l] * yv[L_OF == l]) == pytest.approx(npleg.legval(c, coef),
                                                                        abs=1e-13)


def test_homogeneous_and_gradient(lib):
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=3) * 2.0
        r = np.linalg.norm(d)
        # homogeneity: R_lm(d) = r^l Y_lm(d/r)
        np.testing.assert_allclose(Y(lib, d), r ** L_OF * Y(lib, d / r), rtol=1e-12, atol=1e-12)
        G = rng.normal(size=24)
        v = np.zeros(3)
        lib.h_harmonics_grad_dot(*[float(t) for t in d], _p(G), _p(v))
        h = 1e-6
        fd = np.zeros(3)
        for a in range(3):
            e = np.zeros(3); e[a] = h
            fd[a] = (G @ Y(lib, d + e) - G @ Y(lib, d - e)) / (2 * h)
        np.testing.assert_allclose(v, fd, rtol=1e-7, atol=1e-8)


def test_fourbody_map(lib):
    rng = np.random.default_rng(2)
    u = rng.normal(size=(7, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    g = rng.normal(size=7)
    A2 = np.array([g @ np.array([Y(lib, x)[3 + m] for x in u]) for m in range(5)])
    T = np.einsum("j,ja,jb->ab", g, u, u) - g.sum() * np.eye(3) / 3
    dq = np.zeros(5)
    q4 = lib.h_fourbody(_p(A2), _p(dq))
    assert q4 == pytest.approx(np.trace(T @ T @ T), rel=1e-12)
    h = 1e-6
    for m in range(5):
        e = np.zeros(5); e[m] = h
        fd = (lib.h_fourbody(_p(A2 + e), None) - lib.h_fourbody(_p(A2 - e), None)) / (2 * h)
        assert dq[m] == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_chebyshev_basis(lib):
    rc = 4.0
    for r in (0.2, 1.3, 2.9, 3.8):
        T, dT, o = np.zeros(9), np.zeros(9), np.zeros(3)
        lib.h_cheb9(r, 1 / rc, _p(T), _p(dT), _p(o))
        x = 2 * (r / rc - 1) ** 2 - 1
        th = math.acos(x)
        np.testing.assert_allclose(T, [math.cos(k * th) for k in range(9)], atol=1e-13)
        np.testing.assert_allclose(dT, [k * math.sin(k * th) / math.sin(th) for k in range(9)],
                                   atol=1e-11)
        assert o[0] == pytest.approx(0.5 * (1 + math.cos(math.pi * r / rc)), abs=1e-15)
        assert o[1] == pytest.approx(-0.5 * math.pi / rc * math.sin(math.pi * r / rc), abs=1e-15)
        assert o[2] == pytest.approx(4 * (r / rc - 1) / rc, abs=1e-15)


def test_fp32_cutoff_polynomial(lib):
    """The FP32 sin/cos(pi x) used for the cutoff is within 3e-7 of the exact
    values on [0, 1] (FP32 rounding of the Horner evaluation)."""
    lib.h_cutoff_f.argtypes = [C.c_float, C.POINTER(C.c_float)]
    out = np.zeros(2, np.float32)
    worst = 0.0
    for x in np.linspace(0.0, 1.0, 2001):
        lib.h_cutoff_f(float(x), out.ctypes.data_as(C.POINTER(C.c_float)))
        xf = float(np.float32(x))
        worst = max(worst, abs(out[0] - math.sin(math.pi * xf)), abs(out[1] - math.cos(math.pi * xf)))
    assert worst < 3e-7, worst


def test_harmonics_directional_derivative(lib):
    lib.h_harmonics_dir.argtypes = [C.POINTER(C.c_double)] * 3
    rng = np.random.default_rng(5)
    for _ in range(10):
        u = rng.normal(size=3)
        w = rng.normal(size=3)
        D = np.zeros(24)
        lib.h_harmonics_dir(_p(u), _p(w), _p(D))
        h = 1e-6
        fd = (Y(lib, u + h * w) - Y(lib, u - h * w)) / (2 * h)
        np.testing.assert_allclose(D, fd, rtol=1e-7, atol=1e-8)


def test_fourbody_hessian_vector_product(lib):
    lib.h_fourbody_hvp.argtypes = [C.POINTER(C.c_double)] * 3
    rng = np.random.default_rng(6)
    A2 = rng.normal(size=5)
    Ad = rng.normal(size=5)
    out = np.zeros(5)
    lib.h_fourbody_hvp(_p(A2), _p(Ad), _p(out))
    h = 1e-6
    gp, gm = np.zeros(5), np.zeros(5)
    lib.h_fourbody(_p(A2 + h * Ad), _p(gp))
    lib.h_fourbody(_p(A2 - h * Ad), _p(gm))
    np.testing.assert_allclose(out, (gp - gm) / (2 * h), rtol=1e-7, atol=1e-9)


def test_grouped_harmonics_equal_the_full_forms(lib):
    """The three 8-index groups of harmonics and of the gradient contraction
    (used when coefficients stream in group by group) give exactly the full
    harmonics and the full contraction, and the contraction is the gradient
    of sum_lm G_lm R_lm (central differences)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        u = rng.normal(size=3)
        G = rng.normal(size=24)
        Yg, vg = np.zeros(24), np.zeros(3)
        lib.h_harmonics_groups(_p(u), _p(G), _p(Yg), _p(vg))
        np.testing.assert_allclose(Yg, Y(lib, u), rtol=1e-14, atol=1e-14)
        v = np.zeros(3)
        lib.h_harmonics_grad_dot(*[float(t) for t in u], _p(G), _p(v))
        np.testing.assert_allclose(vg, v, rtol=1e-13, atol=1e-13)
        h = 1e-6
        fd = np.array([(G @ Y(lib, u + h * e) - G @ Y(lib, u - h * e)) / (2 * h)
                       for e in np.eye(3)])
        np.testing.assert_allclose(vg, fd, rtol=1e-7, atol=1e-7)
