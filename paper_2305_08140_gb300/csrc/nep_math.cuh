// nep_math.cuh -- per-pair building blocks of the NEP descriptor on the GPU.
//
// Host+device so the same code is unit-tested on the CPU.  Sizes are fixed at
// compile time (registers): K Chebyshev basis functions, angular orders
// l = 1..4 (24 real harmonics).
//
// Radial basis (NEP descriptor, Sec. II.A "Chebyshev"):
//   f_c(r)  = (1 + cos(pi r / rc)) / 2             (r < rc)
//   x       = 2 (r/rc - 1)^2 - 1
//   f_k(r)  = (T_k(x) + 1) / 2 * f_c(r)
//   g_n(r)  = sum_k c_nk f_k(r) = f_c(r) * (C_n + sum_k h_nk T_k(x)),
//             with h_nk = c_nk / 2 and C_n = sum_k h_nk.
// Angular part (Sec. II.A "Legendre"): by the addition theorem
//   P_l(u.v) = sum_m Y_lm(u) Y_lm(v)
// for the Schmidt semi-normalised real harmonics Y_lm written here as
// homogeneous polynomials R_lm of degree l (Y_lm(u) = R_lm(u) on |u| = 1), so
// the Legendre double sum of one atom is q_nl = sum_m A_nlm^2 with
// A_nlm = sum_j g_n(r_ij) Y_lm(u_ij).
// Index of (l, m) in the 24-vector: l = 1: 0..2, l = 2: 3..7, l = 3: 8..14,
// l = 4: 15..23; inside each l: m = 0, then (cos, sin) for m = 1..l.
#pragma once

#if defined(__CUDACC__)
#define NEP_HD __host__ __device__ __forceinline__
#else
#define NEP_HD inline
#endif

#include <math.h>

namespace nepm {

constexpr int NLM = 24;   // real harmonics for l = 1..4

NEP_HD float nep_sqrt(float x) { return sqrtf(x); }
NEP_HD double nep_sqrt(double x) { return sqrt(x); }

// sin(pi x), cos(pi x)
NEP_HD void nep_sincospi(float x, float* s, float* c)
{
#if defined(__CUDA_ARCH__)
    sincospif(x, s, c);
#else
    *s = (float)sin(M_PI * (double)x);
    *c = (float)cos(M_PI * (double)x);
#endif
}
NEP_HD void nep_sincospi(double x, double* s, double* c)
{
#if defined(__CUDA_ARCH__)
    sincospi(x, s, c);
#else
    *s = sin(M_PI * x);
    *c = cos(M_PI * x);
#endif
}

NEP_HD float nep_rsqrt(float x)
{
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
NEP_HD double nep_rsqrt(double x) { return 1.0 / sqrt(x); }

// sin(pi x) and cos(pi x) for x in [0, 1].  FP32: with theta = pi (x - 1/2)
// in [-pi/2, pi/2], cos(pi x) = -sin(theta) and sin(pi x) = cos(theta), each
// from its Taylor series (sin to theta^13, cos to theta^14; truncation below
// 7e-10 on the interval), evaluated by Horner in theta^2.  FP64: sincospi.
NEP_HD void cutoff_sincospi(float x, float* s, float* c)
{
    const float th = 3.14159265358979f * (x - 0.5f);
    const float u = th * th;
    float sn = 1.6059043836821613e-10f;            // 1/13!
    sn = sn * u - 2.505210838544172e-08f;          // 1/11!
    sn = sn * u + 2.7557319223985893e-06f;         // 1/9!
    sn = sn * u - 1.984126984126984e-04f;          // 1/7!
    sn = sn * u + 8.333333333333333e-03f;          // 1/5!
    sn = sn * u - 1.6666666666666666e-01f;         // 1/3!
    sn = (sn * u + 1.0f) * th;
    float cs = -1.1470745597729725e-11f;           // 1/14!
    cs = cs * u + 2.08767569878681e-09f;           // 1/12!
    cs = cs * u - 2.755731922398589e-07f;          // 1/10!
    cs = cs * u + 2.48015873015873e-05f;           // 1/8!
    cs = cs * u - 1.388888888888889e-03f;          // 1/6!
    cs = cs * u + 4.1666666666666664e-02f;         // 1/4!
    cs = cs * u - 0.5f;                            // 1/2!
    cs = cs * u + 1.0f;
    *c = -sn;
    *s = cs;
}
NEP_HD void cutoff_sincospi(double x, double* s, double* c) { nep_sincospi(x, s, c); }

// Chebyshev values T_0..T_{K-1} at x = 2 (r/rc - 1)^2 - 1, the cutoff f_c and,
// when DERIV, dT_k/dx, dx/dr and df_c/dr.  Requires r < rc.
template <int K, bool DERIV, typename R>
NEP_HD void cheb(R r, R inv_rc, R* T, R* dT, R& fc, R& dfc, R& dxdr)
{
    R t = r * inv_rc - R(1);
    R x = R(2) * t * t - R(1);
    R s, c;
    cutoff_sincospi(r * inv_rc, &s, &c);
    fc = R(0.5) * (R(1) + c);
    T[0] = R(1);
    T[1] = x;
#pragma unroll
    for (int k = 2; k < K; ++k) T[k] = R(2) * x * T[k - 1] - T[k - 2];
    if (DERIV) {
        dfc = R(-0.5) * R(M_PI) * inv_rc * s;
        dxdr = R(4) * t * inv_rc;
        dT[0] = R(0);
        dT[1] = R(1);
#pragma unroll
        for (int k = 2; k < K; ++k) dT[k] = R(2) * T[k - 1] + R(2) * x * dT[k - 1] - dT[k - 2];
    }
}

// Real Schmidt harmonics R_lm at u (homogeneous polynomials; u need not be a
// unit vector, then the values are R_lm(u) = |u|^l Y_lm(u/|u|)), in two
// parts: l = 1, 2 (Y[0..7]) and l = 3, 4 (Y[8..23]), so that a caller can
// consume the first part before forming the second.
template <typename R>
NEP_HD void harmonics_l12(R x, R y, R z, R* Y)
{
    const R s3 = R(1.7320508075688772);
    R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
    R xy = x * y, xmy = x2 - y2;
    // l = 1
    Y[0] = z; Y[1] = x; Y[2] = y;
    // l = 2
    Y[3] = z2 - R(0.5) * rho2;
    Y[4] = s3 * x * z;
    Y[5] = s3 * y * z;
    Y[6] = R(0.5) * s3 * xmy;
    Y[7] = s3 * xy;
}

// l = 3, 4: writes Y[8..23]
template <typename R>
NEP_HD void harmonics_l34(R x, R y, R z, R* Y)
{
    const R s6_4 = R(0.6123724356957945), s15 = R(3.872983346207417),
            s15_2 = R(1.9364916731037085), s10_4 = R(0.7905694150420949),
            s5_4 = R(0.5590169943749475), s5_2 = R(1.118033988749895),
            s70_4 = R(2.091650066335189), s35_8 = R(0.739509972887452),
            s35_2 = R(2.958039891549808);
    R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
    R xy = x * y, xmy = x2 - y2;
    // l = 3
    R a3 = R(4) * z2 - rho2;
    Y[8] = z * (z2 - R(1.5) * rho2);
    Y[9] = s6_4 * x * a3;
    Y[10] = s6_4 * y * a3;
    Y[11] = s15_2 * z * xmy;
    Y[12] = s15 * xy * z;
    R c3 = x * (x2 - R(3) * y2), s3m = y * (R(3) * x2 - y2);
    Y[13] = s10_4 * c3;
    Y[14] = s10_4 * s3m;
    // l = 4
    R a4 = R(4) * z2 - R(3) * rho2, b4 = R(6) * z2 - rho2;
    Y[15] = z2 * z2 - R(3) * z2 * rho2 + R(0.375) * rho2 * rho2;
    Y[16] = s10_4 * x * z * a4;
    Y[17] = s10_4 * y * z * a4;
    Y[18] = s5_4 * b4 * xmy;
    Y[19] = s5_2 * b4 * xy;
    Y[20] = s70_4 * z * c3;
    Y[21] = s70_4 * z * s3m;
    Y[22] = s35_8 * (xmy * xmy - R(4) * x2 * y2);
    Y[23] = s35_2 * xy * xmy;
}

template <typename R>
NEP_HD void harmonics(R x, R y, R z, R* Y)
{
    harmonics_l12(x, y, z, Y);
    harmonics_l34(x, y, z, Y);
}

// V = sum_lm G[lm] grad R_lm (u), the gradients of the homogeneous
// polynomials above evaluated at u.
template <typename R>
NEP_HD void harmonics_grad_dot(R x, R y, R z, const R* G, R& vx, R& vy, R& vz)
{
    const R s3 = R(1.7320508075688772), s6_4 = R(0.6123724356957945),
            s15 = R(3.872983346207417), s15_2 = R(1.9364916731037085),
            s10_4 = R(0.7905694150420949), s5 = R(2.23606797749979),
            s5_2 = R(1.118033988749895), s70_4 = R(2.091650066335189),
            s35_2 = R(2.958039891549808);
    R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
    R xy = x * y, xz = x * z, yz = y * z, xmy = x2 - y2, xyz = xy * z;
    // l = 1
    vx = G[1];
    vy = G[2];
    vz = G[0];
    // l = 2
    vx += -x * G[3] + s3 * (z * G[4] + x * G[6] + y * G[7]);
    vy += -y * G[3] + s3 * (z * G[5] - y * G[6] + x * G[7]);
    vz += R(2) * z * G[3] + s3 * (x * G[4] + y * G[5]);
    // l = 3
    vx += R(-3) * xz * G[8] + s6_4 * (R(4) * z2 - R(3) * x2 - y2) * G[9] -
          s6_4 * R(2) * xy * G[10] + s15 * (xz * G[11] + yz * G[12]) +
          s10_4 * R(3) * (xmy * G[13] + R(2) * xy * G[14]);
    vy += R(-3) * yz * G[8] - s6_4 * R(2) * xy * G[9] +
          s6_4 * (R(4) * z2 - x2 - R(3) * y2) * G[10] + s15 * (-yz * G[11] + xz * G[12]) +
          s10_4 * R(3) * (R(-2) * xy * G[13] + xmy * G[14]);
    vz += (R(3) * z2 - R(1.5) * rho2) * G[8] + s6_4 * R(8) * (xz * G[9] + yz * G[10]) +
          s15_2 * xmy * G[11] + s15 * xy * G[12];
    // l = 4
    R c3 = x * (x2 - R(3) * y2), s3m = y * (R(3) * x2 - y2);
    R t15 = R(1.5) * rho2 - R(6) * z2;
    vx += x * t15 * G[15] +
          s10_4 * (z * (R(4) * z2 - R(9) * x2 - R(3) * y2) * G[16] - R(6) * xyz * G[17]) +
          s5 * x * (R(3) * z2 - x2) * G[18] + s5_2 * y * (R(6) * z2 - R(3) * x2 - y2) * G[19] +
          s70_4 * (R(3) * z * xmy * G[20] + R(6) * xyz * G[21]) +
          s35_2 * (c3 * G[22] + s3m * G[23]);
    vy += y * t15 * G[15] +
          s10_4 * (R(-6) * xyz * G[16] + z * (R(4) * z2 - R(3) * x2 - R(9) * y2) * G[17]) -
          s5 * y * (R(3) * z2 - y2) * G[18] + s5_2 * x * (R(6) * z2 - x2 - R(3) * y2) * G[19] +
          s70_4 * (R(-6) * xyz * G[20] + R(3) * z * xmy * G[21]) +
          s35_2 * (-s3m * G[22] + c3 * G[23]);
    vz += (R(4) * z2 * z - R(6) * z * rho2) * G[15] +
          s10_4 * R(3) * (R(4) * z2 - rho2) * (x * G[16] + y * G[17]) +
          R(3) * s5 * z * xmy * G[18] + R(6) * s5 * xyz * G[19] +
          s70_4 * (c3 * G[20] + s3m * G[21]);
}

// The harmonics and their gradient contraction in three groups of 8 indices
// (group 0: lm 0-7 = l 1, 2; group 1: lm 8-15 = l 3 and the first l = 4;
// group 2: lm 16-23), for callers that stream coefficients group by group:
// harmonics_group<GR> writes Y[0..7] = R_lm for lm = 8 GR + 0..7, and
// harmonics_grad_dot_group<GR> adds sum over the group's lm of Gg[lm - 8 GR]
// grad R_lm(u) to v.  Summed over the three groups they equal harmonics and
// harmonics_grad_dot (the same terms).
template <int GR, typename R>
NEP_HD void harmonics_group(R x, R y, R z, R* Y)
{
    if constexpr (GR == 0) {
        harmonics_l12(x, y, z, Y);
    } else {
        const R s6_4 = R(0.6123724356957945), s15 = R(3.872983346207417),
                s15_2 = R(1.9364916731037085), s10_4 = R(0.7905694150420949),
                s5_4 = R(0.5590169943749475), s5_2 = R(1.118033988749895),
                s70_4 = R(2.091650066335189), s35_8 = R(0.739509972887452),
                s35_2 = R(2.958039891549808);
        R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
        R xy = x * y, xmy = x2 - y2;
        R c3 = x * (x2 - R(3) * y2), s3m = y * (R(3) * x2 - y2);
        if constexpr (GR == 1) {   // as harmonics_l34, Y[8..15]
            R a3 = R(4) * z2 - rho2;
            Y[0] = z * (z2 - R(1.5) * rho2);
            Y[1] = s6_4 * x * a3;
            Y[2] = s6_4 * y * a3;
            Y[3] = s15_2 * z * xmy;
            Y[4] = s15 * xy * z;
            Y[5] = s10_4 * c3;
            Y[6] = s10_4 * s3m;
            Y[7] = z2 * z2 - R(3) * z2 * rho2 + R(0.375) * rho2 * rho2;
        } else {                   // Y[16..23]
            R a4 = R(4) * z2 - R(3) * rho2, b4 = R(6) * z2 - rho2;
            Y[0] = s10_4 * x * z * a4;
            Y[1] = s10_4 * y * z * a4;
            Y[2] = s5_4 * b4 * xmy;
            Y[3] = s5_2 * b4 * xy;
            Y[4] = s70_4 * z * c3;
            Y[5] = s70_4 * z * s3m;
            Y[6] = s35_8 * (xmy * xmy - R(4) * x2 * y2);
            Y[7] = s35_2 * xy * xmy;
        }
    }
}

template <int GR, typename R>
NEP_HD void harmonics_grad_dot_group(R x, R y, R z, const R* Gg, R& vx, R& vy, R& vz)
{
    const R s3 = R(1.7320508075688772), s6_4 = R(0.6123724356957945),
            s15 = R(3.872983346207417), s15_2 = R(1.9364916731037085),
            s10_4 = R(0.7905694150420949), s5 = R(2.23606797749979),
            s5_2 = R(1.118033988749895), s70_4 = R(2.091650066335189),
            s35_2 = R(2.958039891549808);
    R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
    R xy = x * y, xz = x * z, yz = y * z, xmy = x2 - y2, xyz = xy * z;
    if constexpr (GR == 0) {
        const R* G = Gg;   // lm 0..7
        vx += G[1];
        vy += G[2];
        vz += G[0];
        vx += -x * G[3] + s3 * (z * G[4] + x * G[6] + y * G[7]);
        vy += -y * G[3] + s3 * (z * G[5] - y * G[6] + x * G[7]);
        vz += R(2) * z * G[3] + s3 * (x * G[4] + y * G[5]);
    } else if constexpr (GR == 1) {
        const R* G = Gg - 8;   // lm 8..15
        vx += R(-3) * xz * G[8] + s6_4 * (R(4) * z2 - R(3) * x2 - y2) * G[9] -
              s6_4 * R(2) * xy * G[10] + s15 * (xz * G[11] + yz * G[12]) +
              s10_4 * R(3) * (xmy * G[13] + R(2) * xy * G[14]);
        vy += R(-3) * yz * G[8] - s6_4 * R(2) * xy * G[9] +
              s6_4 * (R(4) * z2 - x2 - R(3) * y2) * G[10] + s15 * (-yz * G[11] + xz * G[12]) +
              s10_4 * R(3) * (R(-2) * xy * G[13] + xmy * G[14]);
        vz += (R(3) * z2 - R(1.5) * rho2) * G[8] + s6_4 * R(8) * (xz * G[9] + yz * G[10]) +
              s15_2 * xmy * G[11] + s15 * xy * G[12];
        R t15 = R(1.5) * rho2 - R(6) * z2;
        vx += x * t15 * G[15];
        vy += y * t15 * G[15];
        vz += (R(4) * z2 * z - R(6) * z * rho2) * G[15];
    } else {
        const R* G = Gg - 16;   // lm 16..23
        R c3 = x * (x2 - R(3) * y2), s3m = y * (R(3) * x2 - y2);
        vx += s10_4 * (z * (R(4) * z2 - R(9) * x2 - R(3) * y2) * G[16] - R(6) * xyz * G[17]) +
              s5 * x * (R(3) * z2 - x2) * G[18] + s5_2 * y * (R(6) * z2 - R(3) * x2 - y2) * G[19] +
              s70_4 * (R(3) * z * xmy * G[20] + R(6) * xyz * G[21]) +
              s35_2 * (c3 * G[22] + s3m * G[23]);
        vy += s10_4 * (R(-6) * xyz * G[16] + z * (R(4) * z2 - R(3) * x2 - R(9) * y2) * G[17]) -
              s5 * y * (R(3) * z2 - y2) * G[18] + s5_2 * x * (R(6) * z2 - x2 - R(3) * y2) * G[19] +
              s70_4 * (R(-6) * xyz * G[20] + R(3) * z * xmy * G[21]) +
              s35_2 * (-s3m * G[22] + c3 * G[23]);
        vz += s10_4 * R(3) * (R(4) * z2 - rho2) * (x * G[16] + y * G[17]) +
              R(3) * s5 * z * xmy * G[18] + R(6) * s5 * xyz * G[19] +
              s70_4 * (c3 * G[20] + s3m * G[21]);
    }
}

// D[lm] = grad R_lm(u) . w, the directional derivatives of the homogeneous
// polynomials above along w (each row is the gradient of harmonics_grad_dot
// dotted with w).
template <typename R>
NEP_HD void harmonics_dir(R x, R y, R z, R wx, R wy, R wz, R* Dd)
{
    const R s3 = R(1.7320508075688772), s6_4 = R(0.6123724356957945),
            s15 = R(3.872983346207417), s15_2 = R(1.9364916731037085),
            s10_4 = R(0.7905694150420949), s5 = R(2.23606797749979),
            s5_2 = R(1.118033988749895), s70_4 = R(2.091650066335189),
            s35_2 = R(2.958039891549808);
    R x2 = x * x, y2 = y * y, z2 = z * z, rho2 = x2 + y2;
    R xy = x * y, xz = x * z, yz = y * z, xmy = x2 - y2, xyz = xy * z;
    R c3 = x * (x2 - R(3) * y2), s3m = y * (R(3) * x2 - y2);
    Dd[0] = wz; Dd[1] = wx; Dd[2] = wy;
    Dd[3] = -x * wx - y * wy + R(2) * z * wz;
    Dd[4] = s3 * (z * wx + x * wz);
    Dd[5] = s3 * (z * wy + y * wz);
    Dd[6] = s3 * (x * wx - y * wy);
    Dd[7] = s3 * (y * wx + x * wy);
    Dd[8] = R(-3) * xz * wx - R(3) * yz * wy + (R(3) * z2 - R(1.5) * rho2) * wz;
    Dd[9] = s6_4 * ((R(4) * z2 - R(3) * x2 - y2) * wx - R(2) * xy * wy + R(8) * xz * wz);
    Dd[10] = s6_4 * (R(-2) * xy * wx + (R(4) * z2 - x2 - R(3) * y2) * wy + R(8) * yz * wz);
    Dd[11] = s15 * (xz * wx - yz * wy) + s15_2 * xmy * wz;
    Dd[12] = s15 * (yz * wx + xz * wy + xy * wz);
    Dd[13] = s10_4 * (R(3) * xmy * wx - R(6) * xy * wy);
    Dd[14] = s10_4 * (R(6) * xy * wx + R(3) * xmy * wy);
    R t15 = R(1.5) * rho2 - R(6) * z2;
    Dd[15] = x * t15 * wx + y * t15 * wy + (R(4) * z2 * z - R(6) * z * rho2) * wz;
    Dd[16] = s10_4 * (z * (R(4) * z2 - R(9) * x2 - R(3) * y2) * wx - R(6) * xyz * wy +
                      R(3) * x * (R(4) * z2 - rho2) * wz);
    Dd[17] = s10_4 * (R(-6) * xyz * wx + z * (R(4) * z2 - R(3) * x2 - R(9) * y2) * wy +
                      R(3) * y * (R(4) * z2 - rho2) * wz);
    Dd[18] = s5 * (x * (R(3) * z2 - x2) * wx - y * (R(3) * z2 - y2) * wy + R(3) * z * xmy * wz);
    Dd[19] = s5_2 * (y * (R(6) * z2 - R(3) * x2 - y2) * wx + x * (R(6) * z2 - x2 - R(3) * y2) * wy) +
             R(6) * s5 * xyz * wz;
    Dd[20] = s70_4 * (R(3) * z * xmy * wx - R(6) * xyz * wy + c3 * wz);
    Dd[21] = s70_4 * (R(6) * xyz * wx + R(3) * z * xmy * wy + s3m * wz);
    Dd[22] = s35_2 * (c3 * wx - s3m * wy);
    Dd[23] = s35_2 * (s3m * wx + c3 * wy);
}

// The symmetric traceless T of one channel from its l = 2 coefficients
// (order xx, yy, zz, xy, xz, yz); see fourbody() below.
template <typename R>
NEP_HD void fourbody_T(const R* A2, R* T)
{
    const R i3 = R(0.5773502691896258);
    T[0] = -A2[0] * R(1.0 / 3.0) + A2[3] * i3;
    T[1] = -A2[0] * R(1.0 / 3.0) - A2[3] * i3;
    T[2] = A2[0] * R(2.0 / 3.0);
    T[3] = A2[4] * i3;
    T[4] = A2[1] * i3;
    T[5] = A2[2] * i3;
}

// out_m = 3 <dT/dA_m, S> for a symmetric S (xx, yy, zz, xy, xz, yz): with
// S = T^2 this is d tr(T^3)/dA; with S = T T' + T' T it is the Hessian of
// tr(T^3) applied to the direction A' (T' = T(A')).
template <typename R>
NEP_HD void fourbody_map(const R* S, R* out)
{
    const R i3 = R(0.5773502691896258);
    out[0] = -S[0] - S[1] + R(2) * S[2];
    out[1] = R(6) * S[4] * i3;
    out[2] = R(6) * S[5] * i3;
    out[3] = R(3) * (S[0] - S[1]) * i3;
    out[4] = R(6) * S[3] * i3;
}

// Symmetric product P = X Y + Y X of two symmetric matrices (same order).
template <typename R>
NEP_HD void sym_anticomm(const R* X, const R* Yv, R* P)
{
    // full entries: X = [[a d e][d b f][e f c]]
    R xy_xx = X[0] * Yv[0] + X[3] * Yv[3] + X[4] * Yv[4];
    R xy_yy = X[3] * Yv[3] + X[1] * Yv[1] + X[5] * Yv[5];
    R xy_zz = X[4] * Yv[4] + X[5] * Yv[5] + X[2] * Yv[2];
    R xy_xy = X[0] * Yv[3] + X[3] * Yv[1] + X[4] * Yv[5];   // (XY)_xy
    R xy_yx = X[3] * Yv[0] + X[1] * Yv[3] + X[5] * Yv[4];   // (XY)_yx
    R xy_xz = X[0] * Yv[4] + X[3] * Yv[5] + X[4] * Yv[2];
    R xy_zx = X[4] * Yv[0] + X[5] * Yv[3] + X[2] * Yv[4];
    R xy_yz = X[3] * Yv[4] + X[1] * Yv[5] + X[5] * Yv[2];
    R xy_zy = X[4] * Yv[3] + X[5] * Yv[1] + X[2] * Yv[5];
    // (XY + YX) = XY + (XY)^T for symmetric X, Y
    P[0] = R(2) * xy_xx;
    P[1] = R(2) * xy_yy;
    P[2] = R(2) * xy_zz;
    P[3] = xy_xy + xy_yx;
    P[4] = xy_xz + xy_zx;
    P[5] = xy_yz + xy_zy;
}

// 4-body invariant of one radial channel from its l = 2 coefficients
// A2[0..4] (harmonic order R20, R21c, R21s, R22c, R22s):
// T = sum_j g_j (u u^T - I/3) is the linear image
//   Txx = -A0/3 + A3/sqrt3, Tyy = -A0/3 - A3/sqrt3, Tzz = 2 A0/3,
//   Txy = A4/sqrt3, Txz = A1/sqrt3, Tyz = A2/sqrt3,
// q4 = tr(T^3); dq4/dA2 through d tr(T^3)/dT = 3 T^2.
template <typename R>
NEP_HD R fourbody(const R* A2, R* dq4)
{
    const R i3 = R(0.5773502691896258);   // 1/sqrt(3)
    R txx = -A2[0] * R(1.0 / 3.0) + A2[3] * i3;
    R tyy = -A2[0] * R(1.0 / 3.0) - A2[3] * i3;
    R tzz = A2[0] * R(2.0 / 3.0);
    R txy = A2[4] * i3, txz = A2[1] * i3, tyz = A2[2] * i3;
    // S = T^2 (symmetric)
    R sxx = txx * txx + txy * txy + txz * txz;
    R syy = txy * txy + tyy * tyy + tyz * tyz;
    R szz = txz * txz + tyz * tyz + tzz * tzz;
    R sxy = txx * txy + txy * tyy + txz * tyz;
    R sxz = txx * txz + txy * tyz + txz * tzz;
    R syz = txy * txz + tyy * tyz + tyz * tzz;
    R q4 = sxx * txx + syy * tyy + szz * tzz + R(2) * (sxy * txy + sxz * txz + syz * tyz);
    if (dq4) {
        dq4[0] = (-sxx - syy + R(2) * szz);          // 3 * (Sxx(-1/3) + Syy(-1/3) + Szz(2/3))
        dq4[1] = R(6) * sxz * i3;
        dq4[2] = R(6) * syz * i3;
        dq4[3] = R(3) * (sxx - syy) * i3;
        dq4[4] = R(6) * sxy * i3;
    }
    return q4;
}

}  // namespace nepm
