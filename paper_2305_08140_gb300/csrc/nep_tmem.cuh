// nep_tmem.cuh -- the angular kernel of the FP32 one-species path with the
// per-atom angular state in Tensor Memory.
//
// The angular pair-force pass needs the atom's adjoint dU/dA_nlm (5 x 24
// values) for every pair; held in registers it limits the kernel to two
// blocks per SM.  Here each block allocates 128 columns of Tensor Memory
// (lane = thread, column n * 24 + lm).  The descriptor sums A are formed in
// one pass over the atom's angular pairs: radial channels 0-2 in registers (72
// sums, stored to Tensor Memory at the end), channels 3-4 accumulated in their
// Tensor-Memory columns (read, updated and written back per pair); the
// network turns them into the adjoint in place; the
// pair loop streams the adjoint back in 8-column groups (one group in flight
// while the previous one is used).  At <= 128 registers per thread four
// blocks fit per SM (16 warps), which is also the most the 512 columns of
// Tensor Memory hold: the launch pads its dynamic shared memory so that no
// fifth block can be resident.  The arithmetic is that of k_nep_ang
// (nep_device.cuh) except that the angular force of a pair is contracted
// channel by channel.  It carries no ZBL and no close-pair branch: an
// evaluation with a pair inside the outer ZBL radius (a status bit of the
// radial-descriptor pass) goes to k_nep_ang, as do dense clumps.
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
__device__ __forceinline__ void tm_wait_ld8(float* v)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                   "+f"(v[6]), "+f"(v[7])
                 :
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Packed FP32 pairs (sm_100 and later: one FFMA2 instruction does two
// correctly rounded FMAs, so the issue-bound loops below take half the
// instructions for the same arithmetic).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

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

// force_pair_ang with the adjoint in Tensor Memory (warp-collective).  The
// adjoint is read in 15 groups of 8 columns, group-major: harmonic group GR
// (lm 8 GR .. 8 GR + 7, see nepm::harmonics_group) of channels n = 0..4 in
// turn (columns n * 24 + 8 GR), linear index c = 5 GR + n; buf[0] holds
// c = 0 on entry, loaded and not yet waited for; c + 1 (into buf[(c+1) & 1])
// is loaded while c is used.  Only the current group's harmonics Y_lm and
// the channel sums G_lm = sum_n a_nlm g_n, H_lm = sum_n a_nlm g_n' are live:
// the tangential part sum_lm G_lm grad Y_lm and the radial part
//   S = sum_lm Y_lm (H_lm - (l / r) G_lm)
// are added group by group (the same sum as sum_n [g_n' sum_lm a_nlm Y_lm -
// (g_n / r) sum_lm l a_nlm Y_lm], in fewer operations).  With `prefetch`
// (warp-uniform) c = 0 is loaded again into buf[0] for the next pair once the
// last group (c = 14, also in buf[0]) has been used.
template <bool MS = false>
__device__ __forceinline__ void force_pair_ang_tm(const Model<float>& P, float r, float inv_r,
                                                  float ux, float uy, float uz, uint32_t tb,
                                                  float (&buf)[2][8], bool prefetch,
                                                  float& fx, float& fy, float& fz,
                                                  const float* cs = nullptr)
{
    // MS: cs = the pair's angular coefficients (h [0, 45), C [45, 50))
    float gn[NA], dgn[NA];
    {
        float T[KA], dT[KA], fc, dfc, dxdr;
        nepm::cheb<KA, true>(r, P.inv_rcA, T, dT, fc, dfc, dxdr);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            // (sum_k h_nk T_k + C_n, sum_k h_nk T'_k) as one packed pair
            float2 ab = f2(MS ? cs[NA * KA + n] : P.CA[n], 0.f);
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) {
                const float h = MS ? cs[n * KA + kk] : P.hA[n * KA + kk];
                ab = fma2(f2(h, h), f2(T[kk], dT[kk]), ab);
            }
            gn[n] = fc * ab.x;
            dgn[n] = dfc * ab.x + fc * dxdr * ab.y;
        }
    }
    // -l / r for l = 1..4
    const float m1 = -inv_r, m2 = -2.f * inv_r, m3 = -3.f * inv_r, m4 = -4.f * inv_r;
    float sang = 0.f;
    float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
    for (int GR = 0; GR < 3; ++GR) {
        // copies of u that the compiler cannot see through (an empty volatile
        // asm, ordered after the previous group's Tensor-Memory waits): the
        // group's polynomials are formed here, not hoisted and kept live
        float gx = ux, gy = uy, gz = uz;
        asm volatile("" : "+f"(gx), "+f"(gy), "+f"(gz));
        float Y[8];
        if (GR == 0) nepm::harmonics_group<0>(gx, gy, gz, Y);
        if (GR == 1) nepm::harmonics_group<1>(gx, gy, gz, Y);
        if (GR == 2) nepm::harmonics_group<2>(gx, gy, gz, Y);
        float2 G2[4], H2[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) { G2[p] = f2(0.f, 0.f); H2[p] = f2(0.f, 0.f); }
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            const int c = GR * NA + n;
            tm_wait_ld8(buf[c & 1]);
            if (c + 1 < 3 * NA) {
                const int n1 = (c + 1) % NA, g1 = (c + 1) / NA;
                tm_ld8(tb + (uint32_t)(n1 * NLM + 8 * g1), buf[(c + 1) & 1]);
            }
            const float* v = buf[c & 1];
            const float2 gg = f2(gn[n], gn[n]), hh = f2(dgn[n], dgn[n]);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float2 v2 = f2(v[2 * p], v[2 * p + 1]);
                G2[p] = fma2(v2, gg, G2[p]);
                H2[p] = fma2(v2, hh, H2[p]);
            }
        }
        // radial part of the group; the degree l of each lm (group 0: l = 1
        // for lm < 3, else 2; group 1: l = 3 for lm < 15, else 4; group 2: 4)
        const float2 L[4] = {GR == 0 ? f2(m1, m1) : (GR == 1 ? f2(m3, m3) : f2(m4, m4)),
                             GR == 0 ? f2(m1, m2) : (GR == 1 ? f2(m3, m3) : f2(m4, m4)),
                             GR == 0 ? f2(m2, m2) : (GR == 1 ? f2(m3, m3) : f2(m4, m4)),
                             GR == 0 ? f2(m2, m2) : (GR == 1 ? f2(m3, m4) : f2(m4, m4))};
        float2 s2 = mul2(f2(Y[0], Y[1]), fma2(L[0], G2[0], H2[0]));
#pragma unroll
        for (int p = 1; p < 4; ++p) s2 = fma2(f2(Y[2 * p], Y[2 * p + 1]), fma2(L[p], G2[p], H2[p]), s2);
        sang += s2.x + s2.y;
        const float G[8] = {G2[0].x, G2[0].y, G2[1].x, G2[1].y, G2[2].x, G2[2].y, G2[3].x, G2[3].y};
        if (GR == 0) nepm::harmonics_grad_dot_group<0>(gx, gy, gz, G, vx, vy, vz);
        if (GR == 1) nepm::harmonics_grad_dot_group<1>(gx, gy, gz, G, vx, vy, vz);
        if (GR == 2) nepm::harmonics_grad_dot_group<2>(gx, gy, gz, G, vx, vy, vz);
    }
    // the next pair's c = 0: buf[0] held the last group (3 NA is odd), now used
    if (prefetch) tm_ld8(tb, buf[0]);
    fx = sang * ux + vx * inv_r;
    fy = sang * uy + vy * inv_r;
    fz = sang * uz + vz * inv_r;
}

// A_nlm += g v for the 8 columns at a (this lane's Tensor-Memory row): loaded,
// updated and stored back (warp-collective; the store is not waited for).
__device__ __forceinline__ void tm_rmw8(uint32_t a, float g, const float* Y)
{
    float v[8];
    tm_ld8(a, v);
    tm_wait_ld8(v);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float2 t = fma2(f2(g, g), f2(Y[2 * p], Y[2 * p + 1]), f2(v[2 * p], v[2 * p + 1]));
        v[2 * p] = t.x;
        v[2 * p + 1] = t.y;
    }
    tm_st8(a, v);
}

// The descriptor sums A_nlm = sum_j g_n(r_ij) Y_lm(u_ij) over the atom's
// CLOSE variant: pairs whose FP32 r^2 is below the squared outer ZBL radius,
// widened by 10^-5 so that every pair whose FP32 distance r^2 rsqrt(r^2) can
// fall below that radius (rsqrtf: 2 ulp) is among them; they take the FP64
// displacement (close_pair_fp64 refines below the radius itself: pairs in
// the margin, at the ZBL switch's zero, are refined as well).
__device__ __forceinline__ bool close_deferred(const Model<float>& P, float r2)
{
    return r2 < P.zbl_r2 * P.zbl_r2 * 1.00001f;
}

// angular pairs in one pass: radial channels 0-2 in registers (72 sums),
// channels 3-4 in their Tensor-Memory columns, read, updated and written back
// per pair and harmonic group (lm 0-7, 8-15, 16-23).  The Tensor-Memory
// accesses are warp-collective, so the loop runs to the warp's largest pair
// count (nmax), a lane's missing pairs adding zero.  Then each channel's part
// of the descriptor (q_nl = sum_m A_nlm^2, q_n^4b) to shared memory
// (s_q[nu - NR][TILE], this thread's column) and channels 0-2 to Tensor
// Memory (stores not waited for).  CLOSE: pairs inside the outer ZBL radius
// (close_deferred) take their displacement from the FP64 positions (as
// close_pair_fp64; g, x64, perm and this atom's slot k serve it); they are
// left out of the pass (cmask: their slots) and added after it, one per lane
// and iteration, so that the FP64 work runs once per deferred pair of the
// busiest lane instead of in every slot in which some lane has one.
template <bool CLOSE, bool MS, typename Entry>
__device__ __forceinline__ void ang_desc_sums(const Model<float>& P, const float4* __restrict__ pos4,
                                              const StencilSplit<float>& s_off, int na, int nmax,
                                              const float4 pi, Entry entry, uint32_t tb,
                                              float* s_q, const Grid& g,
                                              const double* __restrict__ x64,
                                              const int* __restrict__ perm, int k,
                                              const float* s_coef, int ti, int T)
{
    // MS: the pair's angular coefficients from the table in shared memory
    constexpr int NN = 3;   // channels in registers
    float2 A[NN][NLM / 2];   // A_nlm in packed pairs (lm, lm + 1)
#pragma unroll
    for (int n = 0; n < NN; ++n)
#pragma unroll
        for (int p = 0; p < NLM / 2; ++p) A[n][p] = f2(0.f, 0.f);
    {
        float z[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) z[t] = 0.f;
#pragma unroll
        for (int c = NN * NLM; c < NA * NLM; c += 8) tm_st8(tb + (uint32_t)c, z);
    }
    // one pair (act = false: a placeholder that adds zero); collective over
    // the warp (the channel 3-4 columns)
    auto add_pair = [&](float dx, float dy, float dz, float r2, bool act, float tj) {
        if (!act) { dx = 1.f; dy = 0.f; dz = 0.f; r2 = 1.f; }
        // beyond r_c^A (lists built with a skin) or a placeholder: g_n = 0
        const bool in = act && r2 < P.rcA2;
        const float inv_r = nepm::nep_rsqrt(r2);
        const float r = r2 * inv_r;
        float Tk[KA], dT[KA], fc, dfc, dxdr;
        nepm::cheb<KA, false>(r, P.inv_rcA, Tk, dT, fc, dfc, dxdr);
        const float fcm = in ? fc : 0.f;
        const float* cs = MS ? s_coef + ((size_t)ti * T + (int)tj) * CSTR + C_ANG : nullptr;
        float gn[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            float acc = MS ? cs[NA * KA + n] : P.CA[n];
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) acc += (MS ? cs[n * KA + kk] : P.hA[n * KA + kk]) * Tk[kk];
            gn[n] = fcm * acc;
        }
        const float ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
        // the previous pair's stores to the channel 3-4 columns are complete
        // before they are read again
        tm_wait_st();
#pragma unroll
        for (int GR = 0; GR < 3; ++GR) {
            float gx = ux, gy = uy, gz = uz;
            asm volatile("" : "+f"(gx), "+f"(gy), "+f"(gz));
            float Y[8];
            if (GR == 0) nepm::harmonics_group<0>(gx, gy, gz, Y);
            if (GR == 1) nepm::harmonics_group<1>(gx, gy, gz, Y);
            if (GR == 2) nepm::harmonics_group<2>(gx, gy, gz, Y);
#pragma unroll
            for (int n = 0; n < NN; ++n)
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    A[n][4 * GR + p] = fma2(f2(gn[n], gn[n]), f2(Y[2 * p], Y[2 * p + 1]),
                                            A[n][4 * GR + p]);
#pragma unroll
            for (int n = NN; n < NA; ++n) tm_rmw8(tb + (uint32_t)(n * NLM + 8 * GR), gn[n], Y);
        }
    };
    unsigned long long cmask = 0;   // CLOSE: deferred slots (< 64: at most TILE_ANG_LIM pairs)
    int ent_n = na > 0 ? entry(0) : 0;
    float4 pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
    for (int s = 0; s < nmax; ++s) {
        const bool act = s < na;
        const int ent = ent_n;
        const float4 pj = pj_n;
        if (s + 1 < na) {
            ent_n = entry(s + 1);
            pj_n = pos4[ent_n >> 5];
        }
        const int code = ent & 31;
        const float dx = pj.x - pi.x + s_off.x[code], dy = pj.y - pi.y + s_off.y[code],
                    dz = pj.z - pi.z + s_off.z[code];
        const float r2 = dx * dx + dy * dy + dz * dz;
        const bool defer = CLOSE && act && close_deferred(P, r2);
        if (defer) cmask |= 1ull << s;
        add_pair(dx, dy, dz, r2, act && !defer, pj.w);
    }
    if constexpr (CLOSE) {
        // the deferred pairs with their FP64 displacements
        const int cm = __reduce_max_sync(0xffffffffu, __popcll(cmask));
        const int kc = perm[k < g.n ? k : 0];
        for (int j = 0; j < cm; ++j) {
            const bool act = cmask != 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, tj = 0.f;
            if (act) {
                const int ent = entry(__ffsll((long long)cmask) - 1);
                cmask &= cmask - 1;
                double d[3];
                disp64(g, x64, kc, perm[ent >> 5], d);
                dx = (float)d[0];
                dy = (float)d[1];
                dz = (float)d[2];
                r2 = dx * dx + dy * dy + dz * dz;
                if constexpr (MS) tj = pos4[ent >> 5].w;
            }
            add_pair(dx, dy, dz, r2, act, tj);
        }
    }
    // channels 3-4: the final sums back from Tensor Memory
    tm_wait_st();
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float An[NLM];
        if (n < NN) {
#pragma unroll
            for (int p = 0; p < NLM / 2; ++p) { An[2 * p] = A[n][p].x; An[2 * p + 1] = A[n][p].y; }
        } else {
            tm_ld24(tb, n, An);
            tm_wait_ld24(An);
        }
#pragma unroll
        for (int l = 1; l <= LM; ++l) {
            float v = 0.f;
#pragma unroll
            for (int lm = l * l - 1; lm < (l + 1) * (l + 1) - 1; ++lm) v += An[lm] * An[lm];
            s_q[((l - 1) * NA + n) * TILE + threadIdx.x] = v;
        }
        s_q[(LM * NA + n) * TILE + threadIdx.x] = nepm::fourbody(&An[3], (float*)nullptr);
        if (n < NN) tm_st24(tb, n, An);
    }
}

// k_nep_ang (FP32) with the angular state in Tensor Memory; same arguments and
// outputs.  MS (several species): the pair coefficients come from the table
// coef ([T * T][CSTR], copied to shared memory), the record of atom k is one
// radial adjoint per neighbour species t (br[(k T + t) * 3], as k_nep_ang
// writes it), the ZBL parameters are the pair's.  At most TM_BLOCKS_PER_SM blocks may be resident
// (TM_BLOCKS_PER_SM x TM_COLS = 512 columns, so the allocation never waits):
// the launch checks the occupancy and pads the dynamic shared memory to
// enforce it.  It takes the tiles whose flag in tflag (from the
// radial-descriptor pass) is 0 (CLOSE = false) or exactly TILE_CLOSE (CLOSE =
// true: pairs inside the outer ZBL radius, whose displacements come from the
// FP64 positions and whose ZBL term is added in FP64, as in k_nep_ang);
// k_nep_ang takes the dense tiles.  One tile per block with a grid of all
// tiles, or a loop over the tiles with a shorter grid; a block without a tile
// of its own returns before allocating.
constexpr int TM_BLOCKS_PER_SM = 4;
// dynamic shared memory: [0, TM_SQ_OFF) staged angular entries (at most
// STAGE_MAX_SLOTS per atom), then the angular descriptor [D - NR][TILE]; with
// CLOSE also the ZBL virial of every atom [9][TILE] (double)
constexpr int TM_STAGE_SLOTS = 32;
constexpr size_t TM_SQ_OFF = sizeof(int) * TM_STAGE_SLOTS * TILE;
constexpr size_t TM_DYN_MIN = TM_SQ_OFF + sizeof(float) * (D - NR) * TILE;
constexpr size_t TM_WZ_OFF = (TM_DYN_MIN + 15) / 16 * 16;
constexpr size_t TM_DYN_MIN_CLOSE = TM_WZ_OFF + sizeof(double) * 9 * TILE;
// MS: the pair coefficient table after the regions above (at most NT_MAX^2 pairs)
constexpr size_t TM_COEF_BYTES = sizeof(float) * NT_MAX * NT_MAX * CSTR;
template <bool CLOSE, bool MS>
__host__ __device__ constexpr size_t tm_coef_off()
{
    return CLOSE ? TM_DYN_MIN_CLOSE : (TM_DYN_MIN + 15) / 16 * 16;
}
template <bool CLOSE, bool MS>
__host__ __device__ constexpr size_t tm_dyn_min()
{
    return tm_coef_off<CLOSE, MS>() + (MS ? TM_COEF_BYTES : 0);
}
template <bool CLOSE, bool MS>
__global__ void __launch_bounds__(TILE, TM_BLOCKS_PER_SM)
    k_nep_ang_tm(const Model<float> P, const Grid g, const float4* __restrict__ pos4,
                 const int* __restrict__ nbr, const int2* __restrict__ cnt,
                 const int* __restrict__ perm, const double* __restrict__ x64,
                 const float* __restrict__ qr, float4* __restrict__ br,
                 long long* __restrict__ facc, double* __restrict__ partials,
                 double* __restrict__ site_energy, int* __restrict__ status, int stage_slots,
                 const int* __restrict__ tflag, const float* __restrict__ coef)
{
    const int want = CLOSE ? TILE_CLOSE : 0;
    const int ntiles = (g.n + TILE - 1) / TILE;
    // CLOSE: the listed tiles (see tile_mark); otherwise every tile
    const int nlist = CLOSE ? tflag[ntiles] : ntiles;
    if (blockIdx.x >= nlist) return;   // no tile for this block
    if (!CLOSE && gridDim.x >= ntiles && tflag[blockIdx.x] != want) return;   // before allocating
    using A_ = Acc<float>;
    __shared__ StencilSplit<float> s_off;
    __shared__ int s_max;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(16) float s_w[H * WROW];
    __shared__ double s_red[TILE / 32][NPART];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int* s_ent = reinterpret_cast<int*>(s_dyn);
    double* s_wz = reinterpret_cast<double*>(s_dyn + TM_WZ_OFF);   // CLOSE only
    float* s_coef = reinterpret_cast<float*>(s_dyn + tm_coef_off<CLOSE, MS>());   // MS only
    const int T = MS ? P.ntypes : 1;
    if constexpr (MS) {
        for (int t = threadIdx.x; t < T * T * CSTR; t += TILE) s_coef[t] = coef[t];
    }
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fill_network_rows<float>(s_w, P);
    tm_fence_before();
    fill_stencil_split<float>(s_off, g);   // ends with __syncthreads
    tm_fence_after();
    const uint32_t tb = s_tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
    const size_t ld = (size_t)g.ld;
    // (without CLOSE the grid covers the tiles: one iteration)
    const int it_end = CLOSE ? nlist : (int)blockIdx.x + 1;
    for (int it = blockIdx.x; it < it_end; it += CLOSE ? gridDim.x : 1) {
    const int tile = CLOSE ? tflag[ntiles + 1 + it] : it;
    if (tflag[tile] != want) continue;   // the whole block
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();   // also: the previous tile's shared data is no longer read
    const int k = tile * TILE + threadIdx.x;
    const bool valid = k < g.n;
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
    const int ti = MS ? (int)pi.w : 0;

    // descriptor vector: angular part in one pass over the pairs (the sums A
    // to Tensor Memory, q via shared memory), radial part from the neighbour
    // kernel
    float* s_q = reinterpret_cast<float*>(s_dyn + TM_SQ_OFF);
    const int nmax = __reduce_max_sync(0xffffffffu, na);
    ang_desc_sums<CLOSE, MS>(P, pos4, s_off, na, nmax, pi, entry, tb, s_q, g, x64, perm, k,
                             s_coef, ti, T);
    float q[D];
#pragma unroll
    for (int n = 0; n < NR; ++n) q[n] = valid ? qr[(size_t)n * ld + k] : 0.f;
#pragma unroll
    for (int nu = NR; nu < D; ++nu) q[nu] = s_q[(nu - NR) * TILE + threadIdx.x];
    tm_wait_st();

    // network forward and backward (rolled over the hidden neurons, as
    // network_adjoint_core_rolled)
    // (packed pairs of descriptor components: the pre-activation is the sum of
    // an even and an odd partial sum)
    float2 a2[D / 2];
#pragma unroll
    for (int p = 0; p < D / 2; ++p) a2[p] = f2(0.f, 0.f);
    float U = -P.b1;
#pragma unroll 1
    for (int mu = 0; mu < H; ++mu) {
        float w[WROW];
        load_row<float>(s_w + mu * WROW, w);
        float2 h2 = f2(-w[D], 0.f);
#pragma unroll
        for (int p = 0; p < D / 2; ++p) h2 = fma2(f2(w[2 * p], w[2 * p + 1]), f2(q[2 * p], q[2 * p + 1]), h2);
        const float h = h2.x + h2.y;
        const float t = tanhf(h);
        U += w[D + 1] * t;
        const float gm = w[D + 1] * (1.f - t * t);
#pragma unroll
        for (int p = 0; p < D / 2; ++p) a2[p] = fma2(f2(gm, gm), f2(w[2 * p], w[2 * p + 1]), a2[p]);
    }
    float a[D];
#pragma unroll
    for (int p = 0; p < D / 2; ++p) { a[2 * p] = a2[p].x; a[2 * p + 1] = a2[p].y; }
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
    // the record the radial-force kernel gathers per neighbour (rec_store); MS:
    // per neighbour species t, (b_0..b_3), (b_4..b_7), (b_8, B0, 0, 0)
    if (valid) {
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float* c = MS ? s_coef + ((size_t)ti * T + t) * CSTR + C_RAD : nullptr;
            float bR[KR], B0 = 0.f;
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) bR[kk] = 0.f;
#pragma unroll
            for (int nu = 0; nu < NR; ++nu) {
                B0 += a[nu] * (MS ? c[NR * KR + nu] : P.CR[nu]);
#pragma unroll
                for (int kk = 0; kk < KR; ++kk)
                    bR[kk] += a[nu] * (MS ? c[nu * KR + kk] : P.hR[nu * KR + kk]);
            }
            if constexpr (MS) {
                const size_t slot = (size_t)k * T + t;
                br[3 * slot] = make_float4(bR[0], bR[1], bR[2], bR[3]);
                br[3 * slot + 1] = make_float4(bR[4], bR[5], bR[6], bR[7]);
                br[3 * slot + 2] = make_float4(bR[8], B0, 0.f, 0.f);
            } else {
                rec_store(br, (size_t)k, make_float4(pi.x, pi.y, pi.z, bR[8]),
                          make_float4(bR[0] + B0, bR[1], bR[2], bR[3]),
                          make_float4(bR[4], bR[5], bR[6], bR[7]));
            }
        }
    }

    // pair-force pass: every lane runs to the warp's largest pair count
    long long fi[3] = {0, 0, 0};
    float wv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wv[t] = 0.f;
    double ez = 0.0;   // CLOSE: half the ZBL energy of the atom's pairs
    bool zhad = false;              // CLOSE: a ZBL term was added
    bool bad = !isfinite(U);
    const int i_caller = valid ? perm[k] : 0;
    float buf[2][8];   // two 8-column groups of the adjoint (see force_pair_ang_tm)
    // one pair (act = false: a placeholder, result unused); collective over
    // the warp (the adjoint columns); more: prefetch for a next pair
    auto force_pair = [&](float dx, float dy, float dz, float r2, bool act, int m, float tj,
                          bool more) -> bool {
        if (!act) { dx = 1.f; dy = 0.f; dz = 0.f; r2 = 1.f; }
        const bool in = act && r2 < P.rcA2;
        const float inv_r = nepm::nep_rsqrt(r2);
        const float r = r2 * inv_r;
        float fx, fy, fz;
        force_pair_ang_tm<MS>(P, r, inv_r, dx * inv_r, dy * inv_r, dz * inv_r, tb, buf, more,
                              fx, fy, fz,
                              MS ? s_coef + ((size_t)ti * T + (int)tj) * CSTR + C_ANG : nullptr);
        if (in) {
            bad |= !isfinite(fx + fy + fz);
            const long long cx = A_::conv(fx), cy = A_::conv(fy), cz = A_::conv(fz);
            fi[0] += cx; fi[1] += cy; fi[2] += cz;
            A_::add(&facc[m], -cx);
            A_::add(&facc[ld + m], -cy);
            A_::add(&facc[2 * ld + m], -cz);
            wv[0] -= fx * dx; wv[1] -= fx * dy; wv[2] -= fx * dz;
            wv[3] -= fy * dx; wv[4] -= fy * dy; wv[5] -= fy * dz;
            wv[6] -= fz * dx; wv[7] -= fz * dy; wv[8] -= fz * dz;
        }
        return in && r < P.zbl_r2;
    };
    // CLOSE: the pairs deferred as in ang_desc_sums (slots < 64)
    unsigned long long cmask = 0;
    int ent_n = na > 0 ? entry(0) : 0;
    float4 pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
    if (nmax > 0) tm_ld8(tb, buf[0]);
    for (int s = 0; s < nmax; ++s) {
        const bool act = s < na;
        const int ent = ent_n;
        const float4 pj = pj_n;
        if (s + 1 < na) {
            ent_n = entry(s + 1);
            pj_n = pos4[ent_n >> 5];
        }
        const int code = ent & 31;
        const float dx = pj.x - pi.x + s_off.x[code], dy = pj.y - pi.y + s_off.y[code],
                    dz = pj.z - pi.z + s_off.z[code];
        const float r2 = dx * dx + dy * dy + dz * dz;
        const bool defer = CLOSE && act && close_deferred(P, r2);
        if (defer) cmask |= 1ull << s;
        force_pair(dx, dy, dz, r2, act && !defer, ent >> 5, pj.w, s + 1 < nmax);
    }
    if constexpr (CLOSE) {
        // the deferred pairs: the FP64 displacement, formed once for the NEP
        // terms (rounded, as close_pair_fp64) and the ZBL term (Eq. 2-4,
        // FP64), in slot order; each term converted and added on its own, as
        // in k_nep_ang; the FP64 virial of the atom to shared memory
        double wz[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) wz[t] = 0.0;
        const int cm = __reduce_max_sync(0xffffffffu, __popcll(cmask));
        if (cm > 0) tm_ld8(tb, buf[0]);
        for (int j = 0; j < cm; ++j) {
            const bool act = cmask != 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, tj = 0.f;
            double d64[3] = {0.0, 0.0, 0.0};
            int m = 0;
            if (act) {
                m = entry(__ffsll((long long)cmask) - 1) >> 5;
                cmask &= cmask - 1;
                disp64(g, x64, i_caller, perm[m], d64);
                dx = (float)d64[0];
                dy = (float)d64[1];
                dz = (float)d64[2];
                r2 = dx * dx + dy * dy + dz * dz;
                if constexpr (MS) tj = pos4[m].w;
            }
            if (force_pair(dx, dy, dz, r2, act, m, tj, j + 1 < cm)) {
                const double r64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
                if (r64 < P.zbl_rr2) {
                    double Uz, dUz;
                    const int pz = MS ? ti * T + (int)tj : 0;
                    zbl_pair(r64, MS ? P.zbl_kp[pz] : P.zbl_k, MS ? P.zbl_inv_ap[pz] : P.zbl_inv_a,
                             P.zbl_r1, P.zbl_rr2, Uz, dUz);
                    ez += 0.5 * Uz;
                    const double c = 0.5 * dUz / r64;
                    const double f3[3] = {c * d64[0], c * d64[1], c * d64[2]};
                    const long long zx = A_::convd(f3[0]), zy = A_::convd(f3[1]),
                                    zz = A_::convd(f3[2]);
                    fi[0] += zx; fi[1] += zy; fi[2] += zz;
                    A_::add(&facc[m], -zx);
                    A_::add(&facc[ld + m], -zy);
                    A_::add(&facc[2 * ld + m], -zz);
                    bad |= !isfinite(c);
                    zhad = true;
#pragma unroll
                    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
                        for (int b3 = 0; b3 < 3; ++b3) wz[3 * a3 + b3] -= f3[a3] * d64[b3];
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) s_wz[t * TILE + threadIdx.x] = wz[t];
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

    // block partials (fixed order): energy and virial by shuffles (the FP64
    // ZBL virial of CLOSE tiles on its own, then added; skipped, as the sums of
    // zeros it would give, by warps without a ZBL term: FP64 adds are slow here)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_site += __shfl_xor_sync(0xffffffffu, e_site, o);
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wv[t] += __shfl_xor_sync(0xffffffffu, wv[t], o);
    double wzs[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wzs[t] = 0.0;
    if (CLOSE && __any_sync(0xffffffffu, zhad)) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            wzs[t] = s_wz[t * TILE + threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wzs[t] += __shfl_xor_sync(0xffffffffu, wzs[t], o);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[warp][0] = e_site;
#pragma unroll
        for (int t = 0; t < 9; ++t) s_red[warp][1 + t] = (double)wv[t] + wzs[t];
    }
    tm_fence_before();
    __syncthreads();
    if (threadIdx.x < NPART) {
        double sum = 0.0;
#pragma unroll
        for (int wi = 0; wi < TILE / 32; ++wi) sum += s_red[wi][threadIdx.x];
        partials[(size_t)tile * NPART + threadIdx.x] = sum;
    }
    }   // tile loop
    if (warp == 0) {
        tm_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(s_tmem), "r"(TM_COLS) : "memory");
    }
}

}  // namespace nepk
