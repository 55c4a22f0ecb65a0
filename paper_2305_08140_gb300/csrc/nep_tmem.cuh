// nep_tmem.cuh -- the angular kernel of the FP32 one-species path with the
// per-atom angular state in Tensor Memory.
//
// The angular pair-force pass needs the atom's adjoint dU/dA_nlm (5 x 24
// values) for every pair; held in registers it limits the kernel to two
// blocks per SM.  Here each block allocates 128 columns of Tensor Memory
// (lane = thread, column n * 24 + lm), the descriptor sums A are written there
// after the descriptor pass, turned into the adjoint in place after the
// network, and read back per radial channel (three 8-column loads, double
// buffered; a pair's first channel is loaded at the end of the previous pair)
// inside the pair loop.  The arithmetic is that of k_nep_ang (nep_device.cuh)
// except that the block's ZBL virial is summed in 2^-32 eV fixed point (order
// independent) instead of FP64 per thread; otherwise only where the 120
// values live differs.
//
// tcgen05.ld/st/alloc are warp-collective (.sync.aligned): every one of them
// is executed by all 32 lanes of a warp together -- the pair loop runs to the
// warp's largest pair count, with the work of a lane's missing pairs masked.
#pragma once

#include "nep_device.cuh"

namespace nepk {

constexpr uint32_t TM_COLS = 128;   // Tensor Memory columns per block (power of two)

__device__ __forceinline__ void tm_st8(uint32_t a, const float* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(a), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                    "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                    "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tm_ld8(uint32_t a, float* v)
{
    uint32_t w0, w1, w2, w3, w4, w5, w6, w7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3), "=r"(w4), "=r"(w5), "=r"(w6), "=r"(w7)
                 : "r"(a)
                 : "memory");
    v[0] = __uint_as_float(w0); v[1] = __uint_as_float(w1);
    v[2] = __uint_as_float(w2); v[3] = __uint_as_float(w3);
    v[4] = __uint_as_float(w4); v[5] = __uint_as_float(w5);
    v[6] = __uint_as_float(w6); v[7] = __uint_as_float(w7);
}

__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// wait::ld that also names the 24 registers it makes valid, so that no use of
// them can be scheduled before it
__device__ __forceinline__ void tm_wait_ld24(float* v)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                   "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]),
                   "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]), "+f"(v[16]),
                   "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]),
                   "+f"(v[22]), "+f"(v[23])
                 :
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// the 24 values of radial channel n of this thread's lane
__device__ __forceinline__ void tm_ld24(uint32_t tb, int n, float* v)
{
    tm_ld8(tb + (uint32_t)(n * NLM), v);
    tm_ld8(tb + (uint32_t)(n * NLM + 8), v + 8);
    tm_ld8(tb + (uint32_t)(n * NLM + 16), v + 16);
}
__device__ __forceinline__ void tm_st24(uint32_t tb, int n, const float* v)
{
    tm_st8(tb + (uint32_t)(n * NLM), v);
    tm_st8(tb + (uint32_t)(n * NLM + 8), v + 8);
    tm_st8(tb + (uint32_t)(n * NLM + 16), v + 16);
}

// force_pair_ang with the adjoint in Tensor Memory (warp-collective).  buf[0]
// holds radial channel 0, loaded before the call and not yet waited for;
// with `prefetch` (warp-uniform) channel 0 is loaded again into buf[0] for
// the next pair as soon as this pair's contraction is done.
__device__ __forceinline__ void force_pair_ang_tm(const Model<float>& P, float r, float inv_r,
                                                  float ux, float uy, float uz, uint32_t tb,
                                                  float (&buf)[2][NLM], bool prefetch,
                                                  float& fx, float& fy, float& fz)
{
    float T[KA], dT[KA], fc, dfc, dxdr;
    nepm::cheb<KA, true>(r, P.inv_rcA, T, dT, fc, dfc, dxdr);
    float gn[NA], dgn[NA];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float a = P.CA[n], b = 0.f;
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            a += P.hA[n * KA + kk] * T[kk];
            b += P.hA[n * KA + kk] * dT[kk];
        }
        gn[n] = fc * a;
        dgn[n] = dfc * a + fc * dxdr * b;
    }
    float G[NLM], Dd[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) { G[lm] = 0.f; Dd[lm] = 0.f; }
    // channel n + 1 is loaded while channel n is used
    tm_wait_ld24(buf[0]);
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        if (n + 1 < NA) tm_ld24(tb, n + 1, buf[(n + 1) & 1]);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            G[lm] += buf[n & 1][lm] * gn[n];
            Dd[lm] += buf[n & 1][lm] * dgn[n];
        }
        if (n + 1 < NA) tm_wait_ld24(buf[(n + 1) & 1]);
    }
    if (prefetch) tm_ld24(tb, 0, buf[0]);   // the next pair's channel 0
    float Y[NLM];
    nepm::harmonics(ux, uy, uz, Y);
    float sang = 0.f;
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
        sang += (Dd[lm] - float(l) * inv_r * G[lm]) * Y[lm];
    }
    float vx, vy, vz;
    nepm::harmonics_grad_dot(ux, uy, uz, G, vx, vy, vz);
    fx = sang * ux + vx * inv_r;
    fy = sang * uy + vy * inv_r;
    fz = sang * uz + vz * inv_r;
}

// k_nep_ang (one species, FP32) with the angular state in Tensor Memory; same
// arguments and outputs.  At most TM_COLS x 3 columns are held per SM, so the
// allocation never waits.  It handles the evaluations whose largest angular
// neighbour count (*ang_max, from the neighbour kernel) is at most ang_lim and
// returns at once otherwise (before allocating), k_nep_ang taking those.
__global__ void __launch_bounds__(TILE, 3)
    k_nep_ang_tm(const Model<float> P, const Grid g, const float4* __restrict__ pos4,
                 const int* __restrict__ nbr, const int2* __restrict__ cnt,
                 const int* __restrict__ perm, const double* __restrict__ x64,
                 const float* __restrict__ qr, float4* __restrict__ br,
                 long long* __restrict__ facc, double* __restrict__ partials,
                 double* __restrict__ site_energy, int* __restrict__ status, int stage_slots,
                 const int* __restrict__ ang_max, int ang_lim)
{
    if (*ang_max > ang_lim) return;   // whole grid: k_nep_ang runs instead
    using A_ = Acc<float>;
    __shared__ float4 s_off[27];
    __shared__ int s_max;
    __shared__ uint32_t s_tmem;
    __shared__ long long s_wz[9];   // ZBL virial of the block, fixed point (2^-32 eV)
    __shared__ __align__(16) float s_w[H * WROW];
    __shared__ double s_red[TILE / 32][NPART];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int* s_ent = reinterpret_cast<int*>(s_dyn);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) s_max = 0;
    if (threadIdx.x < 9) s_wz[threadIdx.x] = 0;
    fill_network_rows<float>(s_w, P);
    tm_fence_before();
    fill_stencil<float>(s_off, g);   // ends with __syncthreads
    tm_fence_after();
    const uint32_t tb = s_tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
    const int k = blockIdx.x * TILE + threadIdx.x;
    const bool valid = k < g.n;
    const size_t ld = (size_t)g.ld;
    const int na = valid ? cnt[k].x : 0;
    atomicMax(&s_max, na);
    __syncthreads();
    const bool staged = s_max <= stage_slots;
    if (staged)
        for (int s = 0; s < na; ++s) s_ent[s * TILE + threadIdx.x] = nbr[(size_t)s * ld + k];
    auto entry = [&](int s) -> int {
        return staged ? s_ent[s * TILE + threadIdx.x] : nbr[(size_t)s * ld + k];
    };
    const float4 pi = valid ? pos4[k] : make_float4(0.f, 0.f, 0.f, 0.f);

    // descriptor pass: A_nlm = sum_j g_n(r_ij) Y_lm(u_ij) in registers
    float A[NA][NLM];
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) A[n][lm] = 0.f;
    {
        int ent_n = na > 0 ? entry(0) : 0;
        float4 pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
        for (int s = 0; s < na; ++s) {
            const int ent = ent_n;
            const float4 pj = pj_n;
            if (s + 1 < na) {
                ent_n = entry(s + 1);
                pj_n = pos4[ent_n >> 5];
            }
            const float4 off = s_off[ent & 31];
            const float dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= P.rcA2) continue;   // beyond r_c^A (lists built with a skin)
            const float inv_r = nepm::nep_rsqrt(r2);
            const float r = r2 * inv_r;
            float Tk[KA], dT[KA], fc, dfc, dxdr;
            nepm::cheb<KA, false>(r, P.inv_rcA, Tk, dT, fc, dfc, dxdr);
            float gn[NA];
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                float acc = P.CA[n];
#pragma unroll
                for (int kk = 0; kk < KA; ++kk) acc += P.hA[n * KA + kk] * Tk[kk];
                gn[n] = fc * acc;
            }
            const float ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
            float Y[NLM];
            nepm::harmonics_l12(ux, uy, uz, Y);
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int lm = 0; lm < 8; ++lm) A[n][lm] += gn[n] * Y[lm];
            nepm::harmonics_l34(ux, uy, uz, Y);
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int lm = 8; lm < NLM; ++lm) A[n][lm] += gn[n] * Y[lm];
        }
    }

    // descriptor vector; A goes to Tensor Memory
    float q[D];
#pragma unroll
    for (int n = 0; n < NR; ++n) q[n] = valid ? qr[(size_t)n * ld + k] : 0.f;
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            float v = 0.f;
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) v += A[n][lm] * A[n][lm];
            q[NR + (l - 1) * NA + n] = v;
        }
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) q[NR + LM * NA + n] = nepm::fourbody(&A[n][3], (float*)nullptr);
#pragma unroll
    for (int n = 0; n < NA; ++n) tm_st24(tb, n, A[n]);
    tm_wait_st();

    // network forward and backward (rolled over the hidden neurons, as
    // network_adjoint_core_rolled)
    float a[D];
#pragma unroll
    for (int nu = 0; nu < D; ++nu) a[nu] = 0.f;
    float U = -P.b1;
#pragma unroll 1
    for (int mu = 0; mu < H; ++mu) {
        float w[WROW];
        load_row<float>(s_w + mu * WROW, w);
        float h = -w[D];
#pragma unroll
        for (int nu = 0; nu < D; ++nu) h += w[nu] * q[nu];
        const float t = tanhf(h);
        U += w[D + 1] * t;
        const float gm = w[D + 1] * (1.f - t * t);
#pragma unroll
        for (int nu = 0; nu < D; ++nu) a[nu] += gm * w[nu];
    }
    // adjoint dU/dA_nlm in Tensor Memory, channel by channel (4-body term
    // folded into l = 2)
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float v[NLM];
        tm_ld24(tb, n, v);
        tm_wait_ld24(v);
        float dq4[5];
        nepm::fourbody(&v[3], dq4);
        const float a4 = a[NR + LM * NA + n];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
            v[lm] *= 2.f * a[NR + (l - 1) * NA + n];
            if (l == 2) v[lm] += a4 * dq4[lm - 3];
        }
        tm_st24(tb, n, v);
    }
    tm_wait_st();
    // the record the radial-force kernel gathers per neighbour:
    // (x, y, z, b_8), (b_0 + B0, b_1, b_2, b_3), (b_4..b_7)
    if (valid) {
        float bR[KR], B0 = 0.f;
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) bR[kk] = 0.f;
#pragma unroll
        for (int nu = 0; nu < NR; ++nu) {
            B0 += a[nu] * P.CR[nu];
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) bR[kk] += a[nu] * P.hR[nu * KR + kk];
        }
        br[3 * (size_t)k] = make_float4(pi.x, pi.y, pi.z, bR[8]);
        br[3 * (size_t)k + 1] = make_float4(bR[0] + B0, bR[1], bR[2], bR[3]);
        br[3 * (size_t)k + 2] = make_float4(bR[4], bR[5], bR[6], bR[7]);
    }

    // pair-force pass: every lane runs to the warp's largest pair count
    long long fi[3] = {0, 0, 0};
    float wv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wv[t] = 0.f;
    double ez = 0.0;
    bool bad = !isfinite(U);
    const int i_caller = valid ? perm[k] : 0;
    const int nmax = __reduce_max_sync(0xffffffffu, na);
    int ent_n = na > 0 ? entry(0) : 0;
    float4 pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
    float buf[2][NLM];   // adjoint of two radial channels (see force_pair_ang_tm)
    if (nmax > 0) tm_ld24(tb, 0, buf[0]);
    for (int s = 0; s < nmax; ++s) {
        const bool act = s < na;
        const int ent = ent_n;
        const float4 pj = pj_n;
        if (s + 1 < na) {
            ent_n = entry(s + 1);
            pj_n = pos4[ent_n >> 5];
        }
        const int m = ent >> 5;
        const float4 off = s_off[ent & 31];
        float dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
        if (!act) { dx = 1.f; dy = 0.f; dz = 0.f; }   // placeholder pair, result unused
        const float r2 = dx * dx + dy * dy + dz * dz;
        const bool in = act && r2 < P.rcA2;
        const float inv_r = nepm::nep_rsqrt(r2);
        const float r = r2 * inv_r;
        float fx, fy, fz;
        force_pair_ang_tm(P, r, inv_r, dx * inv_r, dy * inv_r, dz * inv_r, tb, buf, s + 1 < nmax,
                          fx, fy, fz);
        if (in) {
            bad |= !isfinite(fx + fy + fz);
            long long cx = A_::conv(fx), cy = A_::conv(fy), cz = A_::conv(fz);
            if (r < P.zbl_r2) {
                const int j_caller = perm[m];
                double d64[3];
                for (int c = 0; c < 3; ++c) {
                    double t = x64[c * g.n + j_caller] - x64[c * g.n + i_caller];
                    if (!g.tric && g.pbc[c]) t -= g.L[c] * rint(t * g.invL[c]);
                    d64[c] = t;
                }
                if (g.tric) min_image_tric(g, d64);
                const double r64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
                if (r64 < P.zbl_rr2) {
                    double Uz, dUz;
                    zbl_pair(r64, P.zbl_k, P.zbl_inv_a, P.zbl_r1, P.zbl_rr2, Uz, dUz);
                    ez += 0.5 * Uz;
                    const double c = 0.5 * dUz / r64;
                    const double f3[3] = {c * d64[0], c * d64[1], c * d64[2]};
                    cx += A_::convd(f3[0]);
                    cy += A_::convd(f3[1]);
                    cz += A_::convd(f3[2]);
                    bad |= !isfinite(c);
                    for (int a1 = 0; a1 < 3; ++a1)
                        for (int b1 = 0; b1 < 3; ++b1)
                            atomicAdd(reinterpret_cast<unsigned long long*>(&s_wz[3 * a1 + b1]),
                                      static_cast<unsigned long long>(
                                          A_::convd(-f3[a1] * d64[b1])));
                }
            }
            fi[0] += cx; fi[1] += cy; fi[2] += cz;
            A_::add(&facc[m], -cx);
            A_::add(&facc[ld + m], -cy);
            A_::add(&facc[2 * ld + m], -cz);
            wv[0] -= fx * dx; wv[1] -= fx * dy; wv[2] -= fx * dz;
            wv[3] -= fy * dx; wv[4] -= fy * dy; wv[5] -= fy * dz;
            wv[6] -= fz * dx; wv[7] -= fz * dy; wv[8] -= fz * dz;
        }
    }
    double e_site = 0.0;
    if (valid) {
        A_::add(&facc[k], fi[0]);
        A_::add(&facc[ld + k], fi[1]);
        A_::add(&facc[2 * ld + k], fi[2]);
        e_site = (double)U + ez;
        if (site_energy) site_energy[i_caller] = e_site;
        if (bad) atomicOr(status, ST_NONFINITE);
    }

    // block partials (fixed order): energy and NEP virial by shuffles, the
    // ZBL virial from its fixed-point block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_site += __shfl_xor_sync(0xffffffffu, e_site, o);
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wv[t] += __shfl_xor_sync(0xffffffffu, wv[t], o);
    if ((threadIdx.x & 31) == 0) {
        s_red[warp][0] = e_site;
#pragma unroll
        for (int t = 0; t < 9; ++t) s_red[warp][1 + t] = (double)wv[t];
    }
    tm_fence_before();
    __syncthreads();
    if (threadIdx.x < NPART) {
        double sum = 0.0;
#pragma unroll
        for (int wi = 0; wi < TILE / 32; ++wi) sum += s_red[wi][threadIdx.x];
        if (threadIdx.x > 0) sum += A_::value(s_wz[threadIdx.x - 1]);
        partials[(size_t)blockIdx.x * NPART + threadIdx.x] = sum;
    }
    if (warp == 0) {
        tm_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(s_tmem), "r"(TM_COLS) : "memory");
    }
}

}  // namespace nepk
