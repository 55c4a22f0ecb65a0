// nep_batch.cuh -- many small periodic configurations in one persistent launch:
// forward (energies, forces), backward (gradient of a loss with respect to
// all model parameters, given dL/dE_s and dL/dF_i) and the fused
// energy+force loss with its gradient.
//
// One CTA takes whole configurations from an atomic work queue.  A
// configuration's positions, force accumulators and force residuals live in
// shared memory; neighbour lists (all periodic images, self-images included)
// and the per-atom backward state live in global scratch.
//
// Parameter gradient.  With e_i = dL/dF_i and eps_s = dL/dE_s, and
// F_i = -dE/dr_i,
//   dL/dtheta = sum_i d/dtheta [ eps U_i - a_i . qdot_i ],
// where a_i = dU_i/dq_i and qdot_i = sum_j (dq_i/dd_ij) . (e_j - e_i) is the
// derivative of atom i's descriptor along the residual field (the
// force-loss term is minus the parameter derivative of E's directional
// derivative along e).  Per atom this needs q, qdot (descriptor and its
// tangent), the network's value, gradient and Hessian-vector product, and two
// pair loops that contract the basis-coefficient derivatives.
// Virial term.  With W = -sum_ij (dU_i/dd_ij) (x) d_ij and G_s = dL/dW_s,
//   sum_ab G_ab dW_ab/dtheta = -d/dtheta sum_ij (dU_i/dd_ij) . (G d_ij),
// the same form as the force term, so the pair direction becomes
//   v_ij = (e_j - e_i) + G_s d_ij
// and everything downstream is unchanged.
#pragma once

#include "nep_device.cuh"

namespace nepk {

constexpr int BMAXA = 512;   // largest configuration handled by one CTA
constexpr int NP = H * D + 2 * H + 1 + NR * KR + NA * KA;   // 1051 parameters
constexpr int OFF_B0 = H * D, OFF_W1 = OFF_B0 + H, OFF_B1 = OFF_W1 + H;
constexpr int OFF_CR = OFF_B1 + 1, OFF_CA = OFF_CR + NR * KR;

// per-atom backward scratch layout (units of R)
constexpr int BS_A = 0;                // A_nlm [NA][NLM]
constexpr int BS_AD = NA * NLM;        // A-dot [NA][NLM]
constexpr int BS_Q = 2 * NA * NLM;     // q [D]
constexpr int BS_QD = BS_Q + D;        // q-dot [D]
constexpr int BS_U = BS_QD + D;        // u_mu = w1 (eps s' - s'' h-dot) [H]
constexpr int BS_V = BS_U + H;         // v_mu = w1 s' [H]
constexpr int BS_GW1 = BS_V + H;       // eps t - s' h-dot [H]
constexpr int BS_P = BS_GW1 + H;       // p = W^T u [D]
constexpr int BS_AV = BS_P + D;        // a = W^T v [D]
constexpr int BSTRIDE = BS_AV + D;

enum { MODE_FORWARD = 0, MODE_BACKWARD = 1, MODE_LOSS = 2, MODE_LISTS = 3 };

struct Batch {
    int S;                     // configurations
    int M;                     // neighbour slots per atom
    long long ntot;            // atoms in the batch
    const long long* off;      // [S + 1] first atom of each configuration
    const int* order;          // [S] processing order (largest first)
    const double* box;         // [S][3] periodic box lengths
    const double* x;           // [3][ntot] positions
    int* nbr;                  // [M][ntot] (local index << 5) | image code
    int2* cnt;                 // [ntot] (angular, radial-only) counts
    int* queue;                // work counter, zero before the launch
    int* status;               // [3] status bits, max neighbour count
    double* E;                 // [S] energies (forward, loss)
    double* F;                 // [3][ntot] forces (forward, loss)
    const double* dLdE;        // [S] (backward)
    const double* dLdF;        // [3][ntot] (backward)
    const double* Et;          // [S] target energies (loss)
    const double* Ft;          // [3][ntot] target forces (loss)
    double we, wf;             // loss weights
    double* W;                 // [S][9] virials (forward, loss), or nullptr
    const double* Wt;          // [S][6] target virials xx yy zz yz zx xy (loss), or nullptr
    const unsigned char* hv;   // [S] 1 = configuration has a virial target (loss)
    double wv, nv;             // virial weight, number of configurations with a target
    const double* dLdW;        // [S][9] (backward), or nullptr
    double* lpart;             // [S][3] energy, force and virial loss of each configuration
    double* gpart;             // [S][np] gradient of each configuration
    void* scr;                 // [ntot][BSTRIDE] backward scratch
    // several species: T types, the pair coefficient table [T * T][CSTR] (R),
    // species of every atom, and the parameter count 961 + 90 T^2
    int T;
    const void* coef;
    const int* types;
    int np;
};

// Sum of v over the CTA, in a fixed order; every thread gets the result.
template <int BT>
__device__ __forceinline__ double block_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < BT / 32; ++w) s += sh[w];
    return s;
}

// Neighbour list of local atom i: every atom j and image shift (-1, 0, 1 per
// dimension; box >= r_c^R) with r < r_c^R, j = i only at a non-zero shift.
template <typename R>
__device__ __forceinline__ void batch_neighbors(const Model<R>& P, const Batch& b, long long a0,
                                                int N, int i, const typename V4<R>::T* spos,
                                                const double* L)
{
    using P4 = typename V4<R>::T;
    const P4 pi = spos[i];
    const R Lx = (R)L[0], Ly = (R)L[1], Lz = (R)L[2];
    const int M = b.M;
    const size_t col = (size_t)(a0 + i);
    int na = 0, nro = 0, sa = 0, sro = 0;
    for (int j = 0; j < N; ++j) {
        const P4 pj = spos[j];
        const R d0x = pj.x - pi.x, d0y = pj.y - pi.y, d0z = pj.z - pi.z;
        for (int ox = -1; ox <= 1; ++ox) {
            const R dx = d0x + R(ox) * Lx;
            const R rx = dx * dx;
            if (rx >= P.rcR2) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                const R dy = d0y + R(oy) * Ly;
                const R rxy = rx + dy * dy;
                if (rxy >= P.rcR2) continue;
                for (int oz = -1; oz <= 1; ++oz) {
                    if (j == i && ox == 0 && oy == 0 && oz == 0) continue;
                    const R dz = d0z + R(oz) * Lz;
                    const R r2 = rxy + dz * dz;
                    if (r2 >= P.rcR2) continue;
                    const bool ang = r2 < P.rcA2;
                    if (sa + sro < M) {
                        const int ent = (j << 5) | ((ox + 1) * 9 + (oy + 1) * 3 + (oz + 1));
                        if (ang) b.nbr[(size_t)(sa++) * b.ntot + col] = ent;
                        else b.nbr[(size_t)(M - 1 - sro++) * b.ntot + col] = ent;
                    }
                    if (ang) ++na; else ++nro;
                }
            }
        }
    }
    b.cnt[col] = make_int2(sa, sro);
    if (na + nro > M) {
        atomicOr(b.status, ST_OVERFLOW);
        atomicMax(b.status + 1, na + nro);
    }
}

template <typename R>
struct PairGeom {
    R dx, dy, dz, r, inv_r, ux, uy, uz;
    int j;
};

template <typename R>
__device__ __forceinline__ PairGeom<R> pair_geom(int ent, const typename V4<R>::T& pi,
                                                 const typename V4<R>::T* spos,
                                                 const typename V4<R>::T* s_off)
{
    PairGeom<R> g;
    g.j = ent >> 5;
    const typename V4<R>::T pj = spos[g.j];
    const typename V4<R>::T o = s_off[ent & 31];
    g.dx = pj.x - pi.x + o.x;
    g.dy = pj.y - pi.y + o.y;
    g.dz = pj.z - pi.z + o.z;
    const R r2 = g.dx * g.dx + g.dy * g.dy + g.dz * g.dz;
    g.inv_r = nepm::nep_rsqrt(r2);
    g.r = r2 * g.inv_r;
    g.ux = g.dx * g.inv_r;
    g.uy = g.dy * g.inv_r;
    g.uz = g.dz * g.inv_r;
    return g;
}

__device__ __forceinline__ int slot_of(int s, int na, int nro, int M)
{
    return s < na ? s : M - nro + (s - na);
}

// Pair direction of the backward: v_ij = (e_j - e_i) + G d_ij.
template <typename R>
__device__ __forceinline__ void pair_dir(const PairGeom<R>& g, const R (*se)[BMAXA], R eix, R eiy,
                                         R eiz, const R* G, R& vx, R& vy, R& vz)
{
    vx = se[0][g.j] - eix + G[0] * g.dx + G[1] * g.dy + G[2] * g.dz;
    vy = se[1][g.j] - eiy + G[3] * g.dx + G[4] * g.dy + G[5] * g.dz;
    vz = se[2][g.j] - eiz + G[6] * g.dx + G[7] * g.dy + G[8] * g.dz;
}

// Forward of local atom i: descriptor, network, pair forces scattered into
// the shared accumulators; returns U_i (NEP + half ZBL).
// Pair coefficient block (t_i, t_j) with several species, nullptr otherwise.
template <typename R, bool MS>
__device__ __forceinline__ const R* pair_coef(const Batch& b, int ti, int tj)
{
    if constexpr (MS) return (const R*)b.coef + (size_t)(ti * b.T + tj) * CSTR;
    else return nullptr;
}

template <typename R>
__device__ __forceinline__ int species_at(const typename V4<R>::T& p)
{
    return (int)p.w;
}

// MS: coefficients of every pair from its species block (pair_coef); the
// radial descriptor and radial force per pair instead of through basis sums.
// atoms per R partial of the per-configuration gradient sums
constexpr int GSUM_BLK = 16;

template <typename R, bool MS = false>
__device__ __forceinline__ double batch_atom_forward(const Model<R>& P, const Batch& b,
                                                     long long a0, int i,
                                                     const typename V4<R>::T* spos,
                                                     const typename V4<R>::T* s_off,
                                                     typename Acc<R>::T (*sF)[BMAXA], bool& bad,
                                                     double (&w)[9])
{
    using A_ = Acc<R>;
    const size_t col = (size_t)(a0 + i);
    const int2 c2 = b.cnt[col];
    const int na = c2.x, nro = c2.y, tot = na + nro, M = b.M;
    const typename V4<R>::T pi = spos[i];
    const int ti = MS ? species_at<R>(pi) : 0;
    R Sb[KR];
    R A[NA][NLM];
    R qR[NR];
#pragma unroll
    for (int kk = 0; kk < KR; ++kk) Sb[kk] = R(0);
#pragma unroll
    for (int n = 0; n < NR; ++n) qR[n] = R(0);
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) A[n][lm] = R(0);
    for (int s = 0; s < tot; ++s) {
        const int ent = b.nbr[(size_t)slot_of(s, na, nro, M) * b.ntot + col];
        const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
        if constexpr (MS) {
            const R* cs = pair_coef<R, MS>(b, ti, species_at<R>(spos[g.j]));
            R T[KR], dT[KR], fc, dfc, dxdr;
            nepm::cheb<KR, false>(g.r, P.inv_rcR, T, dT, fc, dfc, dxdr);
#pragma unroll
            for (int n = 0; n < NR; ++n) {
                R a = cs[C_RAD + NR * KR + n];
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) a += cs[C_RAD + n * KR + kk] * T[kk];
                qR[n] += fc * a;
            }
            if (s < na) {
                nepm::cheb<KA, false>(g.r, P.inv_rcA, T, dT, fc, dfc, dxdr);
                R Y[NLM];
                nepm::harmonics(g.ux, g.uy, g.uz, Y);
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    R a = cs[C_ANG + NA * KA + n];
#pragma unroll
                    for (int kk = 0; kk < KA; ++kk) a += cs[C_ANG + n * KA + kk] * T[kk];
                    const R gn = fc * a;
#pragma unroll
                    for (int lm = 0; lm < NLM; ++lm) A[n][lm] += gn * Y[lm];
                }
            }
        } else {
            desc_pair<R>(P, g.dx, g.dy, g.dz, g.r, g.inv_r, s < na, Sb, A);
        }
    }
    R bR[KR], B0, aR[NR];
    R U;
    if constexpr (MS) {
        U = network_adjoint_core<R>(P, qR, A, aR);
    } else {
        radial_q<R>(P, Sb, qR);
        U = network_adjoint<R>(P, qR, A, bR, B0);
    }
    double ez = 0.0;
    typename A_::T fi[3] = {0, 0, 0};
    // this atom's NEP virial in R (the narrow FP64 pipe of this GPU made the
    // per-pair FP64 sums the launch's bottleneck); the rare ZBL pairs in FP64
    R wr[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wr[t] = R(0);
    bad |= !isfinite(U);
    for (int s = 0; s < tot; ++s) {
        const int ent = b.nbr[(size_t)slot_of(s, na, nro, M) * b.ntot + col];
        const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
        R fx, fy, fz;
        int tj = 0;
        if constexpr (MS) {
            tj = species_at<R>(spos[g.j]);
            const R* cs = pair_coef<R, MS>(b, ti, tj);
            // radial: sum_n dU/dq_n g_n'(r) along u
            R T[KR], dT[KR], fc, dfc, dxdr;
            nepm::cheb<KR, true>(g.r, P.inv_rcR, T, dT, fc, dfc, dxdr);
            R fs = R(0);
#pragma unroll
            for (int n = 0; n < NR; ++n) {
                R a = cs[C_RAD + NR * KR + n], c = R(0);
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) {
                    a += cs[C_RAD + n * KR + kk] * T[kk];
                    c += cs[C_RAD + n * KR + kk] * dT[kk];
                }
                fs += aR[n] * (dfc * a + fc * dxdr * c);
            }
            fx = fs * g.ux; fy = fs * g.uy; fz = fs * g.uz;
            if (s < na) {
                R ax, ay, az;
                force_pair_ang<R>(P, g.r, g.inv_r, g.ux, g.uy, g.uz, A, ax, ay, az, cs + C_ANG);
                fx += ax; fy += ay; fz += az;
            }
        } else {
            force_pair<R>(P, g.r, g.inv_r, g.ux, g.uy, g.uz, s < na, A, bR, B0, fx, fy, fz);
        }
        bad |= !isfinite(fx + fy + fz);
        typename A_::T cx = A_::conv(fx), cy = A_::conv(fy), cz = A_::conv(fz);
        const R fp[3] = {fx, fy, fz}, dp[3] = {g.dx, g.dy, g.dz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) wr[3 * a + c] -= fp[a] * dp[c];
        if (s < na && g.r < P.zbl_r2) {
            const double d64[3] = {(double)g.dx, (double)g.dy, (double)g.dz};
            const double r64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
            if (r64 < P.zbl_rr2) {
                double Uz, dUz;
                const int pz = MS ? ti * b.T + tj : 0;
                zbl_pair(r64, MS ? P.zbl_kp[pz] : P.zbl_k, MS ? P.zbl_inv_ap[pz] : P.zbl_inv_a,
                         P.zbl_r1, P.zbl_rr2, Uz, dUz);
                ez += 0.5 * Uz;
                const double c = 0.5 * dUz / r64;
                cx += A_::convd(c * d64[0]);
                cy += A_::convd(c * d64[1]);
                cz += A_::convd(c * d64[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int e = 0; e < 3; ++e) w[3 * a + e] -= c * d64[a] * d64[e];
            }
        }
        fi[0] += cx; fi[1] += cy; fi[2] += cz;
        A_::add(&sF[0][g.j], -cx);
        A_::add(&sF[1][g.j], -cy);
        A_::add(&sF[2][g.j], -cz);
    }
    A_::add(&sF[0][i], fi[0]);
    A_::add(&sF[1][i], fi[1]);
    A_::add(&sF[2][i], fi[2]);
#pragma unroll
    for (int t = 0; t < 9; ++t) w[t] += (double)wr[t];
    return (double)U + ez;
}

// Backward, first pass for local atom i: descriptor q, its tangent q-dot along
// the residual field, the network quantities; all into the atom's scratch row.
template <typename R, bool MS = false>
__device__ __forceinline__ void batch_atom_tangent(const Model<R>& P, const Batch& b, long long a0,
                                                   int i, double eps,
                                                   const typename V4<R>::T* spos,
                                                   const typename V4<R>::T* s_off,
                                                   const R (*se)[BMAXA], const R* G)
{
    const size_t col = (size_t)(a0 + i);
    const int2 c2 = b.cnt[col];
    const int na = c2.x, nro = c2.y, tot = na + nro, M = b.M;
    const typename V4<R>::T pi = spos[i];
    const int ti = MS ? species_at<R>(pi) : 0;
    const R eix = se[0][i], eiy = se[1][i], eiz = se[2][i];
    R* row = (R*)b.scr + col * BSTRIDE;
    R q[D], qd[D];
    // radial: q_n = sum g_n, q-dot_n = sum g'_n (u . dd)
#pragma unroll
    for (int n = 0; n < NR; ++n) { q[n] = R(0); qd[n] = R(0); }
    for (int s = 0; s < tot; ++s) {
        const int ent = b.nbr[(size_t)slot_of(s, na, nro, M) * b.ntot + col];
        const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
        R vx, vy, vz;
        pair_dir<R>(g, se, eix, eiy, eiz, G, vx, vy, vz);
        const R ud = g.ux * vx + g.uy * vy + g.uz * vz;
        R T[KR], dT[KR], fc, dfc, dxdr;
        nepm::cheb<KR, true>(g.r, P.inv_rcR, T, dT, fc, dfc, dxdr);
        const R* cs = pair_coef<R, MS>(b, ti, MS ? species_at<R>(spos[g.j]) : 0);
#pragma unroll
        for (int n = 0; n < NR; ++n) {
            R a = MS ? cs[C_RAD + NR * KR + n] : P.CR[n], c = R(0);
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) {
                const R h = MS ? cs[C_RAD + n * KR + kk] : P.hR[n * KR + kk];
                a += h * T[kk];
                c += h * dT[kk];
            }
            q[n] += fc * a;
            qd[n] += (dfc * a + fc * dxdr * c) * ud;
        }
    }
    // angular, one radial channel at a time
#pragma unroll 1
    for (int n = 0; n < NA; ++n) {
        R An[NLM], Ad[NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) { An[lm] = R(0); Ad[lm] = R(0); }
        for (int s = 0; s < na; ++s) {
            const int ent = b.nbr[(size_t)s * b.ntot + col];
            const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
            R ddx, ddy, ddz;
            pair_dir<R>(g, se, eix, eiy, eiz, G, ddx, ddy, ddz);
            const R ud = g.ux * ddx + g.uy * ddy + g.uz * ddz;
            R T[KA], dT[KA], fc, dfc, dxdr;
            nepm::cheb<KA, true>(g.r, P.inv_rcA, T, dT, fc, dfc, dxdr);
            const R* cs = pair_coef<R, MS>(b, ti, MS ? species_at<R>(spos[g.j]) : 0);
            R a = MS ? cs[C_ANG + NA * KA + n] : P.CA[n], c = R(0);
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) {
                const R h = MS ? cs[C_ANG + n * KA + kk] : P.hA[n * KA + kk];
                a += h * T[kk];
                c += h * dT[kk];
            }
            const R gn = fc * a, dgn = dfc * a + fc * dxdr * c;
            R Y[NLM], Dd[NLM];
            nepm::harmonics(g.ux, g.uy, g.uz, Y);
            nepm::harmonics_dir(g.ux, g.uy, g.uz, ddx, ddy, ddz, Dd);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) {
                const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
                An[lm] += gn * Y[lm];
                Ad[lm] += dgn * ud * Y[lm] + gn * g.inv_r * (Dd[lm] - R(l) * Y[lm] * ud);
            }
        }
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            row[BS_A + n * NLM + lm] = An[lm];
            row[BS_AD + n * NLM + lm] = Ad[lm];
        }
#pragma unroll
        for (int l = 1; l <= LM; ++l) {
            const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
            R qq = R(0), qqd = R(0);
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) {
                qq += An[lm] * An[lm];
                qqd += R(2) * An[lm] * Ad[lm];
            }
            q[NR + (l - 1) * NA + n] = qq;
            qd[NR + (l - 1) * NA + n] = qqd;
        }
        R G4[5];
        q[NR + LM * NA + n] = nepm::fourbody(&An[3], G4);
        R q4d = R(0);
#pragma unroll
        for (int t = 0; t < 5; ++t) q4d += G4[t] * Ad[3 + t];
        qd[NR + LM * NA + n] = q4d;
    }
    // network: h = W q - b0, h-dot = W q-dot
    const R e = (R)eps;
#pragma unroll 1
    for (int mu = 0; mu < H; ++mu) {
        R h = -P.b0[mu], hd = R(0);
#pragma unroll
        for (int nu = 0; nu < D; ++nu) {
            h += P.w0[mu * D + nu] * q[nu];
            hd += P.w0[mu * D + nu] * qd[nu];
        }
        const R t = tanh(h);
        const R s1 = R(1) - t * t;       // tanh'
        const R s2 = R(-2) * t * s1;     // tanh''
        row[BS_U + mu] = P.w1[mu] * (e * s1 - s2 * hd);
        row[BS_V + mu] = P.w1[mu] * s1;
        row[BS_GW1 + mu] = e * t - s1 * hd;
    }
#pragma unroll
    for (int nu = 0; nu < D; ++nu) {
        row[BS_Q + nu] = q[nu];
        row[BS_QD + nu] = qd[nu];
    }
    // p = W^T u, a = W^T v
#pragma unroll 1
    for (int nu = 0; nu < D; ++nu) {
        R pp = R(0), aa = R(0);
#pragma unroll
        for (int mu = 0; mu < H; ++mu) {
            pp += P.w0[mu * D + nu] * row[BS_U + mu];
            aa += P.w0[mu * D + nu] * row[BS_V + mu];
        }
        row[BS_P + nu] = pp;
        row[BS_AV + nu] = aa;
    }
}

// Radial basis-coefficient gradient contribution of local atom i:
// g[n][k] += p_n f_k(r) - a_n f'_k(r) (u . dd).
// With several species: only atoms of species ti_sel and their neighbours of
// species tj_sel contribute (the gradient block (ti_sel, tj_sel)).
template <typename R, bool MS = false>
__device__ __forceinline__ void batch_atom_grad_cR(const Model<R>& P, const Batch& b, long long a0,
                                                   int i, const typename V4<R>::T* spos,
                                                   const typename V4<R>::T* s_off,
                                                   const R (*se)[BMAXA], const R* G,
                                                   R (&gR)[NR * KR], int ti_sel = 0,
                                                   int tj_sel = 0)
{
    const size_t col = (size_t)(a0 + i);
    const int2 c2 = b.cnt[col];
    const int na = c2.x, nro = c2.y, tot = na + nro, M = b.M;
    const typename V4<R>::T pi = spos[i];
    if (MS && species_at<R>(pi) != ti_sel) return;
    const R eix = se[0][i], eiy = se[1][i], eiz = se[2][i];
    const R* row = (const R*)b.scr + col * BSTRIDE;
    R p[NR], a[NR];
#pragma unroll
    for (int n = 0; n < NR; ++n) { p[n] = row[BS_P + n]; a[n] = row[BS_AV + n]; }
    for (int s = 0; s < tot; ++s) {
        const int ent = b.nbr[(size_t)slot_of(s, na, nro, M) * b.ntot + col];
        if (MS && species_at<R>(spos[ent >> 5]) != tj_sel) continue;
        const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
        R vx, vy, vz;
        pair_dir<R>(g, se, eix, eiy, eiz, G, vx, vy, vz);
        const R ud = g.ux * vx + g.uy * vy + g.uz * vz;
        R T[KR], dT[KR], fc, dfc, dxdr;
        nepm::cheb<KR, true>(g.r, P.inv_rcR, T, dT, fc, dfc, dxdr);
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) {
            const R fk = R(0.5) * (T[kk] + R(1)) * fc;
            const R dfk = R(0.5) * dT[kk] * dxdr * fc + R(0.5) * (T[kk] + R(1)) * dfc;
#pragma unroll
            for (int n = 0; n < NR; ++n) gR[n * KR + kk] += p[n] * fk - a[n] * dfk * ud;
        }
    }
}

// Angular basis-coefficient gradient of channel n for local atom i.
template <typename R, bool MS = false>
__device__ __forceinline__ void batch_atom_grad_cA(const Model<R>& P, const Batch& b, long long a0,
                                                   int i, int n, const typename V4<R>::T* spos,
                                                   const typename V4<R>::T* s_off,
                                                   const R (*se)[BMAXA], const R* G,
                                                   R (&gA)[KA], int ti_sel = 0, int tj_sel = 0)
{
    const size_t col = (size_t)(a0 + i);
    const int na = b.cnt[col].x;
    const typename V4<R>::T pi = spos[i];
    if (MS && species_at<R>(pi) != ti_sel) return;
    const R eix = se[0][i], eiy = se[1][i], eiz = se[2][i];
    const R* row = (const R*)b.scr + col * BSTRIDE;
    // alpha = dPhi/dA, beta = dPhi/dA-dot for this channel
    R al[NLM], be[NLM];
    R An2[5], Ad2[5];
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
        const R pl = row[BS_P + NR + (l - 1) * NA + n];
        const R alv = row[BS_AV + NR + (l - 1) * NA + n];
#pragma unroll
        for (int lm = lo; lm < hi; ++lm) {
            const R A_ = row[BS_A + n * NLM + lm], Ad_ = row[BS_AD + n * NLM + lm];
            al[lm] = R(2) * pl * A_ - R(2) * alv * Ad_;
            be[lm] = R(-2) * alv * A_;
            if (l == 2) { An2[lm - 3] = A_; Ad2[lm - 3] = Ad_; }
        }
    }
    {
        const R p4 = row[BS_P + NR + LM * NA + n], a4 = row[BS_AV + NR + LM * NA + n];
        R G4[5], Hv[5], T[6], Td[6], Sx[6];
        nepm::fourbody(An2, G4);
        nepm::fourbody_T(An2, T);
        nepm::fourbody_T(Ad2, Td);
        nepm::sym_anticomm(T, Td, Sx);
        nepm::fourbody_map(Sx, Hv);
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            al[3 + t] += p4 * G4[t] - a4 * Hv[t];
            be[3 + t] -= a4 * G4[t];
        }
    }
    for (int s = 0; s < na; ++s) {
        const int ent = b.nbr[(size_t)s * b.ntot + col];
        if (MS && species_at<R>(spos[ent >> 5]) != tj_sel) continue;
        const PairGeom<R> g = pair_geom<R>(ent, pi, spos, s_off);
        R ddx, ddy, ddz;
        pair_dir<R>(g, se, eix, eiy, eiz, G, ddx, ddy, ddz);
        const R ud = g.ux * ddx + g.uy * ddy + g.uz * ddz;
        R Y[NLM], Dd[NLM];
        nepm::harmonics(g.ux, g.uy, g.uz, Y);
        nepm::harmonics_dir(g.ux, g.uy, g.uz, ddx, ddy, ddz, Dd);
        R S1 = R(0), S3 = R(0), SD = R(0), SL = R(0);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
            S1 += al[lm] * Y[lm];
            S3 += be[lm] * Y[lm];
            SD += be[lm] * Dd[lm];
            SL += R(l) * be[lm] * Y[lm];
        }
        const R S2 = g.inv_r * (SD - ud * SL);
        R T[KA], dT[KA], fc, dfc, dxdr;
        nepm::cheb<KA, true>(g.r, P.inv_rcA, T, dT, fc, dfc, dxdr);
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            const R fk = R(0.5) * (T[kk] + R(1)) * fc;
            const R dfk = R(0.5) * dT[kk] * dxdr * fc + R(0.5) * (T[kk] + R(1)) * dfc;
            gA[kk] += fk * (S1 + S2) + dfk * ud * S3;
        }
    }
}

// The persistent batched kernel.
template <typename R, int MODE, int BT, bool MS = false>
__global__ void __launch_bounds__(BT) k_batch(const Model<R> P, const Batch b)
{
    using P4 = typename V4<R>::T;
    using A_ = Acc<R>;
    __shared__ P4 spos[BMAXA];
    __shared__ typename A_::T sF[3][BMAXA];
    __shared__ R se[3][BMAXA];
    __shared__ P4 s_off[27];
    __shared__ double sh[BT / 32];
    __shared__ R sG[9];
    __shared__ int s_cfg;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int t = atomicAdd(b.queue, 1);
            s_cfg = t < b.S ? b.order[t] : -1;
        }
        __syncthreads();
        const int cfg = s_cfg;
        if (cfg < 0) break;
        const long long a0 = b.off[cfg];
        const int N = (int)(b.off[cfg + 1] - a0);
        const double L[3] = {b.box[3 * cfg], b.box[3 * cfg + 1], b.box[3 * cfg + 2]};
        for (int i = threadIdx.x; i < N; i += BT) {
            P4 q;
            double p[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double v = b.x[(size_t)d * b.ntot + a0 + i];
                if (!isfinite(v)) v = 0.0;
                p[d] = v - L[d] * floor(v / L[d]);
            }
            q.x = (R)p[0]; q.y = (R)p[1]; q.z = (R)p[2]; q.w = R(0);
            if (MS) {
                int t = b.types[a0 + i];
                if (t < 0 || t >= b.T) {
                    atomicOr(b.status, ST_BADTYPE);
                    t = 0;
                }
                q.w = (R)t;
            }
            spos[i] = q;
            sF[0][i] = 0; sF[1][i] = 0; sF[2][i] = 0;
        }
        if (threadIdx.x < 27) {
            const int c = threadIdx.x;
            P4 o;
            o.x = (R)((c / 9 - 1) * L[0]);
            o.y = (R)(((c / 3) % 3 - 1) * L[1]);
            o.z = (R)((c % 3 - 1) * L[2]);
            o.w = R(0);
            s_off[c] = o;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += BT) batch_neighbors<R>(P, b, a0, N, i, spos, L);
        if (MODE == MODE_LISTS) continue;   // lists only (population evaluation)
        double eps = 0.0;
        if (threadIdx.x < 9) sG[threadIdx.x] = R(0);
        if (MODE != MODE_BACKWARD) {
            double esum = 0.0;
            double w[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) w[t] = 0.0;
            bool bad = false;
            for (int i = threadIdx.x; i < N; i += BT)
                esum += batch_atom_forward<R, MS>(P, b, a0, i, spos, s_off, sF, bad, w);
            if (bad) atomicOr(b.status, ST_NONFINITE);
            const double E = block_sum<BT>(esum, sh);   // also orders the force scatter
            if (threadIdx.x == 0) b.E[cfg] = E;
            double Wc[9];
#pragma unroll 1
            for (int t = 0; t < 9; ++t) Wc[t] = block_sum<BT>(w[t], sh);
            if (b.W && threadIdx.x == 0)
                for (int t = 0; t < 9; ++t) b.W[(size_t)cfg * 9 + t] = Wc[t];
            double lv = 0.0;
            if (MODE == MODE_LOSS && b.Wt && b.hv[cfg]) {
                // six components xx yy zz yz zx xy of (W - W_target) / N
                const int ia[6] = {0, 4, 8, 5, 6, 1};
                const double inv = 1.0 / ((double)N * N);
                for (int c = 0; c < 6; ++c) {
                    const double dw = Wc[ia[c]] - b.Wt[(size_t)cfg * 6 + c];
                    lv += b.wv * dw * dw * inv / (6.0 * b.nv);
                    if (threadIdx.x == 0) sG[ia[c]] = (R)(b.wv * 2.0 * dw * inv / (6.0 * b.nv));
                }
            }
            double f2 = 0.0;
            for (int i = threadIdx.x; i < N; i += BT) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const size_t o = (size_t)d * b.ntot + a0 + i;
                    const double f = A_::value(sF[d][i]);
                    b.F[o] = f;
                    if (MODE == MODE_LOSS) {
                        const double r = f - b.Ft[o];
                        f2 += r * r;
                        se[d][i] = (R)(b.wf * 2.0 * r / (3.0 * (double)b.ntot));
                    }
                }
            }
            if (MODE == MODE_LOSS) {
                const double F2 = block_sum<BT>(f2, sh);
                const double dE = (E - b.Et[cfg]) / N;
                eps = b.we * 2.0 * dE / ((double)N * b.S);
                if (threadIdx.x == 0) {
                    b.lpart[(size_t)cfg * 3] = b.we * dE * dE / b.S;
                    b.lpart[(size_t)cfg * 3 + 1] = b.wf * F2 / (3.0 * (double)b.ntot);
                    b.lpart[(size_t)cfg * 3 + 2] = lv;
                }
            }
        } else {
            for (int i = threadIdx.x; i < N; i += BT)
#pragma unroll
                for (int d = 0; d < 3; ++d) se[d][i] = (R)b.dLdF[(size_t)d * b.ntot + a0 + i];
            eps = b.dLdE[cfg];
            if (b.dLdW && threadIdx.x < 9) sG[threadIdx.x] = (R)b.dLdW[(size_t)cfg * 9 + threadIdx.x];
        }
        __syncthreads();
        if (MODE != MODE_FORWARD) {
            double* gp = b.gpart + (size_t)cfg * b.np;
            for (int i = threadIdx.x; i < N; i += BT)
                batch_atom_tangent<R, MS>(P, b, a0, i, eps, spos, s_off, se, sG);
            __syncthreads();
            // network weights: G_W = sum_i u (x) q - v (x) q-dot; b0, w1, b1
            const R* scr = (const R*)b.scr;
            for (int e = threadIdx.x; e < H * D + 2 * H + 1; e += BT) {
                double acc = 0.0;
                // sums over the atoms: R partials over GSUM_BLK atoms, FP64
                // across the partials (few FP64 instructions; the per-atom
                // products are R anyway)
                if (e < H * D) {
                    const int mu = e / D, nu = e % D;
                    for (int i0 = 0; i0 < N; i0 += GSUM_BLK) {
                        const int i1 = i0 + GSUM_BLK < N ? i0 + GSUM_BLK : N;
                        R part = R(0);
                        for (int i = i0; i < i1; ++i) {
                            const R* row = scr + (size_t)(a0 + i) * BSTRIDE;
                            part += row[BS_U + mu] * row[BS_Q + nu];
                            part -= row[BS_V + mu] * row[BS_QD + nu];
                        }
                        acc += (double)part;
                    }
                    // W = w0 * s: chain to w0 through the scaler folded into P.w0
                    acc *= (double)P.sc[nu];
                } else if (e < OFF_W1) {
                    for (int i0 = 0; i0 < N; i0 += GSUM_BLK) {
                        const int i1 = i0 + GSUM_BLK < N ? i0 + GSUM_BLK : N;
                        R part = R(0);
                        for (int i = i0; i < i1; ++i)
                            part += scr[(size_t)(a0 + i) * BSTRIDE + BS_U + (e - OFF_B0)];
                        acc -= (double)part;
                    }
                } else if (e < OFF_B1) {
                    for (int i0 = 0; i0 < N; i0 += GSUM_BLK) {
                        const int i1 = i0 + GSUM_BLK < N ? i0 + GSUM_BLK : N;
                        R part = R(0);
                        for (int i = i0; i < i1; ++i)
                            part += scr[(size_t)(a0 + i) * BSTRIDE + BS_GW1 + (e - OFF_W1)];
                        acc += (double)part;
                    }
                } else {
                    acc = -eps * N;
                }
                gp[e] = acc;
            }
            // radial basis coefficients (several species: one pass per
            // block (centre species, neighbour species))
            const int TT = MS ? b.T : 1;
            const int off_ca = OFF_CR + TT * TT * NR * KR;
#pragma unroll 1
            for (int blk = 0; blk < TT * TT; ++blk) {
                R gR[NR * KR];
#pragma unroll
                for (int t = 0; t < NR * KR; ++t) gR[t] = R(0);
                for (int i = threadIdx.x; i < N; i += BT)
                    batch_atom_grad_cR<R, MS>(P, b, a0, i, spos, s_off, se, sG, gR, blk / TT,
                                              blk % TT);
#pragma unroll 1
                for (int t = 0; t < NR * KR; ++t) {
                    const double v = block_sum<BT>((double)gR[t], sh);
                    if (threadIdx.x == 0) gp[OFF_CR + blk * NR * KR + t] = v;
                }
            }
            // angular basis coefficients, one channel (and block) at a time
#pragma unroll 1
            for (int blk = 0; blk < TT * TT; ++blk) {
#pragma unroll 1
                for (int n = 0; n < NA; ++n) {
                    R gA[KA];
#pragma unroll
                    for (int t = 0; t < KA; ++t) gA[t] = R(0);
                    for (int i = threadIdx.x; i < N; i += BT)
                        batch_atom_grad_cA<R, MS>(P, b, a0, i, n, spos, s_off, se, sG, gA,
                                                  blk / TT, blk % TT);
#pragma unroll 1
                    for (int t = 0; t < KA; ++t) {
                        const double v = block_sum<BT>((double)gA[t], sh);
                        if (threadIdx.x == 0) gp[off_ca + blk * NA * KA + n * KA + t] = v;
                    }
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Population evaluation (SNES, Sec. III.A): the NEP loss of n_pop parameter
// vectors over the whole batch in one launch.
// ----------------------------------------------------------------------------

// Model k of the population from theta_k (host layout) and the base model
// (hyperparameters, scaler, ZBL): w0 scaled by s_nu, h = c/2, C = sum_k c/2.
// Several species (T > 1): the network into the model and every pair block
// into tables[k][T * T][CSTR] (the model's own coefficient fields unused).
template <typename R>
__global__ void k_build_models(const Model<R> base, const double* __restrict__ scaler,
                               const double* __restrict__ thetas, Model<R>* __restrict__ out,
                               int np, int T, R* __restrict__ tables)
{
    const int k = blockIdx.x;
    const double* th = thetas + (size_t)k * np;
    Model<R>& m = out[k];
    if (T > 1) {
        const double* cR = th + OFF_CR;
        const double* cA = cR + (size_t)T * T * NR * KR;
        R* tab = tables + (size_t)k * T * T * CSTR;
        for (int e = threadIdx.x; e < T * T * CSTR; e += blockDim.x) {
            const int pr = e / CSTR, o = e % CSTR;
            double v = 0.0;
            if (o < NR * KR) {
                v = 0.5 * cR[(size_t)pr * NR * KR + o];
            } else if (o < NR * KR + NR) {
                const int n = o - NR * KR;
                for (int kk = 0; kk < KR; ++kk) v += 0.5 * cR[(size_t)pr * NR * KR + n * KR + kk];
            } else if (o >= C_ANG && o < C_ANG + NA * KA) {
                v = 0.5 * cA[(size_t)pr * NA * KA + (o - C_ANG)];
            } else if (o >= C_ANG + NA * KA && o < C_ANG + NA * KA + NA) {
                const int n = o - C_ANG - NA * KA;
                for (int kk = 0; kk < KA; ++kk) v += 0.5 * cA[(size_t)pr * NA * KA + n * KA + kk];
            }
            tab[e] = (R)v;
        }
    }
    // everything that is not a parameter comes from the base model
    const unsigned* src = reinterpret_cast<const unsigned*>(&base);
    unsigned* dst = reinterpret_cast<unsigned*>(&m);
    for (int t = threadIdx.x; t < (int)(sizeof(Model<R>) / 4); t += blockDim.x) dst[t] = src[t];
    __syncthreads();
    for (int e = threadIdx.x; e < H * D; e += blockDim.x) m.w0[e] = (R)(th[e] * scaler[e % D]);
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
        m.b0[e] = (R)th[OFF_B0 + e];
        m.w1[e] = (R)th[OFF_W1 + e];
    }
    if (threadIdx.x == 0) m.b1 = (R)th[OFF_B1];
    if (T > 1) return;
    for (int e = threadIdx.x; e < NR * KR; e += blockDim.x) m.hR[e] = (R)(0.5 * th[OFF_CR + e]);
    for (int e = threadIdx.x; e < NA * KA; e += blockDim.x) m.hA[e] = (R)(0.5 * th[OFF_CA + e]);
    if (threadIdx.x < NR) {
        double c = 0.0;
        for (int kk = 0; kk < KR; ++kk) c += 0.5 * th[OFF_CR + threadIdx.x * KR + kk];
        m.CR[threadIdx.x] = (R)c;
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + NA) {
        const int n = threadIdx.x - 32;
        double c = 0.0;
        for (int kk = 0; kk < KA; ++kk) c += 0.5 * th[OFF_CA + n * KA + kk];
        m.CA[n] = (R)c;
    }
}

// Work item t = (configuration order[t / n_pop], individual t % n_pop): the
// individual's model is copied to shared memory, the configuration's forward
// pass uses the lists built by the MODE_LISTS launch, and the item writes
// pout[(k * S + cfg) * 3] = (dE / N, sum |dF|^2, sum over the six virial
// components of (dW / N)^2 or 0 without a virial target).
template <typename R, int BT, bool MS = false>
__global__ void __launch_bounds__(BT) k_batch_pop(const Model<R>* __restrict__ models, int n_pop,
                                                  const Batch b, double* __restrict__ pout,
                                                  const R* __restrict__ tables)
{
    using P4 = typename V4<R>::T;
    using A_ = Acc<R>;
    __shared__ Model<R> sP;
    __shared__ P4 spos[BMAXA];
    __shared__ typename A_::T sF[3][BMAXA];
    __shared__ P4 s_off[27];
    __shared__ double sh[BT / 32];
    __shared__ int s_item;
    const long long n_items = (long long)n_pop * b.S;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(b.queue, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= n_items) break;
        const int cfg = b.order[item / n_pop];
        const int k = (int)(item % n_pop);
        {
            const unsigned* src = reinterpret_cast<const unsigned*>(models + k);
            unsigned* dst = reinterpret_cast<unsigned*>(&sP);
            for (int t = threadIdx.x; t < (int)(sizeof(Model<R>) / 4); t += BT) dst[t] = src[t];
        }
        const long long a0 = b.off[cfg];
        const int N = (int)(b.off[cfg + 1] - a0);
        const double L[3] = {b.box[3 * cfg], b.box[3 * cfg + 1], b.box[3 * cfg + 2]};
        for (int i = threadIdx.x; i < N; i += BT) {
            P4 q;
            double p[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double v = b.x[(size_t)d * b.ntot + a0 + i];
                if (!isfinite(v)) v = 0.0;
                p[d] = v - L[d] * floor(v / L[d]);
            }
            q.x = (R)p[0]; q.y = (R)p[1]; q.z = (R)p[2]; q.w = R(0);
            if (MS) {
                int t = b.types[a0 + i];
                if (t < 0 || t >= b.T) {
                    atomicOr(b.status, ST_BADTYPE);
                    t = 0;
                }
                q.w = (R)t;
            }
            spos[i] = q;
            sF[0][i] = 0; sF[1][i] = 0; sF[2][i] = 0;
        }
        if (threadIdx.x < 27) {
            const int c = threadIdx.x;
            P4 o;
            o.x = (R)((c / 9 - 1) * L[0]);
            o.y = (R)(((c / 3) % 3 - 1) * L[1]);
            o.z = (R)((c % 3 - 1) * L[2]);
            o.w = R(0);
            s_off[c] = o;
        }
        __syncthreads();
        double esum = 0.0;
        double w[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) w[t] = 0.0;
        bool bad = false;
        // the individual's pair table (several species)
        Batch bk = b;
        if (MS) bk.coef = tables + (size_t)k * b.T * b.T * CSTR;
        for (int i = threadIdx.x; i < N; i += BT)
            esum += batch_atom_forward<R, MS>(sP, bk, a0, i, spos, s_off, sF, bad, w);
        if (bad) atomicOr(b.status, ST_NONFINITE);
        const double E = block_sum<BT>(esum, sh);   // also orders the force scatter
        double f2 = 0.0;
        for (int i = threadIdx.x; i < N; i += BT) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const size_t o = (size_t)d * b.ntot + a0 + i;
                const double r = A_::value(sF[d][i]) - b.Ft[o];
                f2 += r * r;
            }
        }
        const double F2 = block_sum<BT>(f2, sh);
        double v2 = 0.0;
        if (b.Wt && b.hv[cfg]) {
            const int ia[6] = {0, 4, 8, 5, 6, 1};
            double Wc[9];
#pragma unroll 1
            for (int t = 0; t < 9; ++t) Wc[t] = block_sum<BT>(w[t], sh);
            for (int c = 0; c < 6; ++c) {
                const double dw = (Wc[ia[c]] - b.Wt[(size_t)cfg * 6 + c]) / N;
                v2 += dw * dw;
            }
        }
        if (threadIdx.x == 0) {
            double* o = pout + ((size_t)k * b.S + cfg) * 3;
            o[0] = (E - b.Et[cfg]) / N;
            o[1] = F2;
            o[2] = v2;
        }
    }
}

// losses[k * 6 + (0..5)] = total, L1, L2, RMSE_E, RMSE_F, RMSE_V of
// individual k (one CTA per individual, fixed summation order).
template <int BT>
__global__ void __launch_bounds__(BT) k_pop_loss(const double* __restrict__ pout,
                                                 const double* __restrict__ thetas, int S,
                                                 long long ntot, double nv, double we, double wf,
                                                 double wv, double l1, double l2,
                                                 double* __restrict__ losses, int np)
{
    __shared__ double sh[BT / 32];
    const int k = blockIdx.x;
    double e2 = 0.0, f2 = 0.0, v2 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int c = threadIdx.x; c < S; c += BT) {
        const double* o = pout + ((size_t)k * S + c) * 3;
        e2 += o[0] * o[0];
        f2 += o[1];
        v2 += o[2];
    }
    for (int p = threadIdx.x; p < np; p += BT) {
        const double t = thetas[(size_t)k * np + p];
        a1 += fabs(t);
        a2 += t * t;
    }
    e2 = block_sum<BT>(e2, sh);
    f2 = block_sum<BT>(f2, sh);
    v2 = block_sum<BT>(v2, sh);
    a1 = block_sum<BT>(a1, sh);
    a2 = block_sum<BT>(a2, sh);
    if (threadIdx.x == 0) {
        const double re = sqrt(e2 / S), rf = sqrt(f2 / (3.0 * (double)ntot));
        const double rv = nv > 0 ? sqrt(v2 / (6.0 * nv)) : 0.0;
        const double r1 = l1 * a1 / np, r2 = l2 * sqrt(a2 / np);
        double* o = losses + (size_t)k * 6;
        o[0] = we * re + wf * rf + wv * rv + r1 + r2;
        o[1] = r1;
        o[2] = r2;
        o[3] = re;
        o[4] = rf;
        o[5] = rv;
    }
}

// SNES candidates theta_k = mu + sigma * s_k.
static __global__ void k_snes_sample(const double* __restrict__ mu, const double* __restrict__ sigma,
                                     const double* __restrict__ samples, int n_pop, int np,
                                     double* __restrict__ thetas)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_pop * np) return;
    const int p = (int)(t % np);
    thetas[t] = mu[p] + sigma[p] * samples[t];
}

// SNES utilities by rank (best first, ties by index):
// u_r = max(0, ln(n/2 + 1) - ln r) / sum_j max(0, ln(n/2 + 1) - ln j) - 1/n.
static __global__ void k_snes_utilities(const double* __restrict__ losses, int n_pop,
                                        double* __restrict__ util)
{
    const int k = threadIdx.x;
    double norm = 0.0;
    for (int r = 1; r <= n_pop; ++r) norm += fmax(0.0, log(n_pop / 2.0 + 1.0) - log((double)r));
    if (k >= n_pop) return;
    const double lk = losses[(size_t)k * 6];
    int rank = 0;
    for (int j = 0; j < n_pop; ++j) {
        const double lj = losses[(size_t)j * 6];
        rank += (lj < lk || (lj == lk && j < k)) ? 1 : 0;
    }
    util[k] = fmax(0.0, log(n_pop / 2.0 + 1.0) - log((double)(rank + 1))) / norm - 1.0 / n_pop;
}

// mu += eta_mu sigma sum_k u_k s_k ;  sigma *= exp(eta_sigma / 2 sum_k u_k (s_k^2 - 1)).
static __global__ void k_snes_update(double* __restrict__ mu, double* __restrict__ sigma,
                                     const double* __restrict__ samples,
                                     const double* __restrict__ util, int n_pop, int np,
                                     double eta_mu, double eta_sigma)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double gm = 0.0, gs = 0.0;
    for (int k = 0; k < n_pop; ++k) {
        const double sk = samples[(size_t)k * np + p];
        gm += util[k] * sk;
        gs += util[k] * (sk * sk - 1.0);
    }
    const double sg = sigma[p];
    mu[p] += eta_mu * sg * gm;
    sigma[p] = sg * exp(0.5 * eta_sigma * gs);
}

// grad[p] = sum over configurations of gpart[c][p], in configuration order.
static __global__ void k_batch_grad_reduce(const double* __restrict__ gpart, int S, int np,
                                    double* __restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int c = 0; c < S; ++c) s += gpart[(size_t)c * np + p];
    grad[p] = s;
}

}  // namespace nepk
