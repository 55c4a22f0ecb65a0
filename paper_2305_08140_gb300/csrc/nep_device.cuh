// nep_device.cuh -- CUDA kernels of one NEP-ZBL force evaluation and of the
// velocity-Verlet step, templated on the arithmetic type R (float: mixed
// precision path; double: plain FP64 path).
//
// Data layout (all in HBM, owned by the context):
//   x, v, F        double SoA [3][n] in the caller's atom order
//   perm[k]        caller index of the k-th atom in cell order
//   pos4[k]        (x, y, z) relative to the origin of the atom's cell, in R,
//                  .w = species; k in cell order (16 B per atom for float)
//   cell_start[c]  first cell-ordered slot of cell c (cells row-major x,y,z)
//   nbr[s * ld + k]  neighbour slot s of atom k: (m << 5) | stencil code, m in
//                  cell order; slots [0, na) hold r < rc_A (also radial),
//                  slots [M - nro, M) hold rc_A <= r < rc_R
//   facc[a * ld + k] force accumulators in cell order: int64 fixed point
//                  (2^-32 eV/A) for float, double for double
//   coef[p * CSTR]  (several species) coefficients of the ordered species
//                  pair p = t_i * T + t_j: radial h (c/2) [0, 45), C [45, 50),
//                  angular h [52, 97), C [97, 102)
//   br[(k * T + t) * 3]  radial adjoint of atom k contracted with the
//                  coefficients of neighbour species t (b_0..b_8, B0, 0, 0);
//                  one species: the record of atom k (see rec_store)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nep_math.cuh"

namespace nepk {

constexpr int NR = 5, NA = 5, KR = 9, KA = 9, LM = 4, NLM = 24, H = 30;
constexpr int D = NR + NA * LM + NA;   // 30
constexpr int TILE = 128;              // atoms per block of the force kernel
constexpr int NPART = 10;              // energy + 9 virial components per tile
constexpr int NT_MAX = 4;              // species
constexpr int CSTR = 104;              // coefficients per ordered species pair
constexpr int C_RAD = 0, C_ANG = 52;   // radial / angular block offsets

// status bits
constexpr int ST_OVERFLOW = 1, ST_NONFINITE = 2, ST_FORCE_RANGE = 4, ST_BADTYPE = 8;

// Per-tile kernel choice (FP32).  The radial-descriptor pass (k_neighbors'
// second pass, or k_radial_q with several species or a Verlet skin; blocks of
// TILE atoms, so block b is tile b) ORs into tflag[tile]: TILE_CLOSE when an
// atom of the tile has a pair closer than the outer ZBL radius, TILE_DENSE
// when one has more than TILE_ANG_LIM angular neighbours.  The Tensor-Memory
// angular kernel without the ZBL and close-pair branches (k_nep_ang_tm<false>)
// takes the tiles with neither bit, its close-pair variant the tiles with
// TILE_CLOSE alone, the register kernel k_nep_ang the dense ones; with one
// species the radial-force instantiation without the close-pair branch takes
// the tiles without TILE_CLOSE, the other the rest.  Each tile is
// done by exactly one kernel of each pair, so its forces and partial sums are
// those of the kernel that would do the whole evaluation.
constexpr int TILE_CLOSE = 1, TILE_DENSE = 2;
constexpr int TILE_ANG_LIM = 48;
// Behind the ntiles flags, tflag[ntiles] counts the flagged tiles and
// tflag[ntiles + 1 + i] lists them (in the order they were first flagged; the
// kernels that take few tiles loop over this list, and every tile's result is
// the same whichever block takes it).
__device__ __forceinline__ void tile_mark(int* __restrict__ tflag, int ntiles, int tile, int bits)
{
    if (atomicOr(&tflag[tile], bits) == 0) tflag[ntiles + 1 + atomicAdd(&tflag[ntiles], 1)] = tile;
}

template <typename R> struct V4 { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

// Model constants passed by value as a kernel argument (constant bank).
template <typename R>
struct Model {
    R w0[H * D];        // w0[mu][nu] * s_nu
    R b0[H], w1[H], b1;
    R hR[NR * KR], CR[NR];   // c/2 and sum_k c/2 (radial)
    R hA[NA * KA], CA[NA];   // angular
    R rcR2, rcA2, inv_rcR, inv_rcA;
    R sc[D];                 // s_nu (for the gradient with respect to w0)
    R zbl_r2;                // outer switch radius (pair test)
    double zbl_k;            // e^2/(4 pi eps0) Zi Zj (eV A)
    double zbl_inv_a;        // 1 / a (Eq. 4)
    double zbl_r1, zbl_rr2;  // switch radii
    int ntypes;              // species
    double zbl_kp[NT_MAX * NT_MAX];      // zbl_k of the ordered pair t_i * T + t_j
    double zbl_inv_ap[NT_MAX * NT_MAX];  // zbl_inv_a of the pair
};

// Cell grid and sizes.
struct Grid {
    int nc[3];
    int pbc[3];
    double lc[3], inv_lc[3];   // cell edge
    double L[3], invL[3];      // box (periodic wrap)
    int n;                     // atoms
    int ld;                    // leading dimension of nbr / facc (atom capacity)
    int M;                     // neighbour slots per atom
    int ntypes;                // species (types must lie in [0, ntypes))
    // triclinic cell: rows of h are the cell vectors, x = s h for fractional s;
    // cells are the parallelepipeds h_a / nc_a (tric = 0: the orthorhombic
    // fields above are used and h, hinv are diagonal)
    int tric;
    double h[9], hinv[9];
    // z sub-slices per cell (1, 2, 4 or 8; 1 for triclinic cells): the atoms of
    // a cell are grouped by slice floor(z_rel zs / lc_z) (clamped), and
    // start[] is indexed by sub-cell c * zs + slice, so that the neighbour
    // search can take the part of a stencil cell within reach in z
    int zs;
};

// Fractional coordinates s = x h^-1 (row vectors).
__device__ __forceinline__ void to_frac(const Grid& g, const double (&x)[3], double (&f)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = x[0] * g.hinv[a] + x[1] * g.hinv[3 + a] + x[2] * g.hinv[6 + a];
}

// Nearest-image displacement (triclinic): d -= sum_a rint(s_a) h_a over periodic a.
__device__ __forceinline__ void min_image_tric(const Grid& g, double (&d)[3])
{
    double f[3];
    to_frac(g, d, f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!g.pbc[a]) continue;
        const double k = rint(f[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) d[b] -= k * g.h[3 * a + b];
    }
}

// Cell of a position (triclinic) and its Cartesian offset from the cell's
// origin: periodic fractional coordinates wrapped into [0, 1), cell indices
// clamped to the grid (open dimensions).
__device__ __forceinline__ void cell_tric(const Grid& g, const double (&x)[3], int (&c)[3],
                                          double (&rel)[3])
{
    double f[3];
    to_frac(g, x, f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (g.pbc[a]) f[a] -= floor(f[a]);
        int k = (int)floor(f[a] * g.nc[a]);
        k = k < 0 ? 0 : (k >= g.nc[a] ? g.nc[a] - 1 : k);
        c[a] = k;
        f[a] -= (double)k / g.nc[a];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) rel[b] = f[0] * g.h[b] + f[1] * g.h[3 + b] + f[2] * g.h[6 + b];
}

// Cartesian offset of the stencil cell (oa, ob, oc) from the home cell
// (triclinic), in double; the same expression wherever it is needed.
__device__ __forceinline__ double stencil_off_tric(const Grid& g, int oa, int ob, int oc, int b)
{
    return (double)oa * g.h[b] / g.nc[0] + (double)ob * g.h[3 + b] / g.nc[1] +
           (double)oc * g.h[6 + b] / g.nc[2];
}

// ----------------------------------------------------------------------------
// Binning: cell of each atom, slot within the cell (atomic), counting sort
// ----------------------------------------------------------------------------

__device__ __forceinline__ int cell_coord(double x, int d, const Grid& g, double& xw)
{
    if (g.pbc[d]) x -= g.L[d] * floor(x * g.invL[d]);
    xw = x;
    int c = (int)floor(x * g.inv_lc[d]);
    c = c < 0 ? 0 : c;
    c = c >= g.nc[d] ? g.nc[d] - 1 : c;
    return c;
}

// Range tests on the bit pattern of a double (integer instructions only: the
// FP64 pipe of this GPU is narrow).  For x >= +0 the IEEE order of doubles is
// the integer order of their bit patterns.
__device__ __forceinline__ bool finite_bits(double x)
{
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
// x in [0, L) for L > 0 (false for -0.0 and NaN)
__device__ __forceinline__ bool in_box_bits(double x, double L)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 && b < __double_as_longlong(L);
}
// x - L floor(x / L), out of line: the caller's rare branch must not be
// turned into predicated FP64 instructions that issue on every thread
static __device__ __noinline__ double wrap_slow(double x, double L, double invL)
{
    return x - L * floor(x * invL);
}

// Cell of each atom and its slot in the cell (atomic count).  With rel
// (orthorhombic or triclinic) the atom's position relative to its cell's
// origin is written too, by caller index, so that k_cell_finalize need not
// recompute it.
template <typename R>
__global__ void k_bin_count(Grid g, const double* __restrict__ x, int* __restrict__ cell_of,
                            int* __restrict__ slot_of, int* __restrict__ count,
                            int* __restrict__ status, const int* __restrict__ gate = nullptr,
                            typename V4<R>::T* __restrict__ rel = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double p[3] = {x[i], x[g.n + i], x[2 * g.n + i]};
    int c[3];
    double r3[3];
    bool bad = false;
    for (int d = 0; d < 3; ++d)
        if (!finite_bits(p[d])) { bad = true; p[d] = 0.0; }
    if (g.tric) {
        cell_tric(g, p, c, r3);
    } else {
        for (int d = 0; d < 3; ++d) {
            double w = p[d];
            if (g.pbc[d] && !in_box_bits(w, g.L[d])) w = wrap_slow(w, g.L[d], g.invL[d]);
            int cd = __double2int_rd(w * g.inv_lc[d]);
            cd = cd < 0 ? 0 : cd;
            cd = cd >= g.nc[d] ? g.nc[d] - 1 : cd;
            c[d] = cd;
            r3[d] = w - cd * g.lc[d];
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    int cell = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
    if (g.zs > 1) {
        int t = __double2int_rd(r3[2] * (g.zs * g.inv_lc[2]));
        t = t < 0 ? 0 : (t >= g.zs ? g.zs - 1 : t);
        cell = cell * g.zs + t;
    }
    cell_of[i] = cell;   // sub-cell
    slot_of[i] = atomicAdd(&count[cell], 1);
    if (rel) {
        typename V4<R>::T q;
        q.x = (R)r3[0]; q.y = (R)r3[1]; q.z = (R)r3[2]; q.w = R(0);
        rel[i] = q;
    }
}

// exclusive scan of count[0..nc) into start[0..nc], 1024 items per block
constexpr int SCAN_T = 256, SCAN_ITEMS = 4, SCAN_B = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total)
{
    // inclusive warp scan
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) sh[w] = s;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int t = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < nw) sh[lane] = t;
    }
    __syncthreads();
    int before = (w > 0 ? sh[w - 1] : 0);
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + s - v;
}

static __global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const int* __restrict__ in, int n,
                                                        int* __restrict__ out,
                                                        int* __restrict__ block_sums,
                            const int* __restrict__ gate = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    __shared__ int sh[32];
    int base = blockIdx.x * SCAN_B + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], sum = 0;
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0;
        sum += v[t];
    }
    int total;
    int ex = block_excl_scan(sum, sh, total);
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        if (base + t < n) out[base + t] = ex;
        ex += v[t];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// one block: exclusive scan of the nb block sums, SCAN_B at a time with a
// running carry; writes out[n] = total
static __global__ void __launch_bounds__(SCAN_T) k_scan_sums(int* __restrict__ sums, int nb,
                                                      int* __restrict__ out, int n,
                            const int* __restrict__ gate = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    __shared__ int sh[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_B) {
        int base = b0 + threadIdx.x * SCAN_ITEMS;
        int v[SCAN_ITEMS], sum = 0;
#pragma unroll
        for (int t = 0; t < SCAN_ITEMS; ++t) {
            v[t] = (base + t < nb) ? sums[base + t] : 0;
            sum += v[t];
        }
        int total;
        int ex = carry + block_excl_scan(sum, sh, total);
#pragma unroll
        for (int t = 0; t < SCAN_ITEMS; ++t) {
            if (base + t < nb) sums[base + t] = ex;
            ex += v[t];
        }
        carry += total;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

static __global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ sums,
                            const int* __restrict__ gate = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / SCAN_B];
}

static __global__ void k_bin_scatter(int n, const int* __restrict__ cell_of,
                              const int* __restrict__ slot_of, const int* __restrict__ start,
                              int* __restrict__ perm,
                            const int* __restrict__ gate = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[cell_of[i]] + slot_of[i]] = i;
}

// One thread per cell: order the cell's atoms by caller index (so everything
// downstream is independent of the atomic slot order) and write their
// cell-relative positions.
template <typename R>
__global__ void k_cell_finalize(Grid g, int ncell, const int* __restrict__ start,
                                int* __restrict__ perm, const double* __restrict__ x,
                                const int32_t* __restrict__ types,
                                typename V4<R>::T* __restrict__ pos4,
                                int* __restrict__ cell_sorted, int* __restrict__ status,
                                const int* __restrict__ gate = nullptr,
                                int* __restrict__ invperm = nullptr,
                                const typename V4<R>::T* __restrict__ relp = nullptr)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int zs = g.zs > 1 ? g.zs : 1;
    int b = start[c * zs], e = start[(c + 1) * zs];
    for (int u = 0; u < zs; ++u) {   // each z slice by caller index
        const int bu = start[c * zs + u], eu = start[c * zs + u + 1];
        for (int s = bu + 1; s < eu; ++s) {
            int v = perm[s], t = s;
            while (t > bu && perm[t - 1] > v) { perm[t] = perm[t - 1]; --t; }
            perm[t] = v;
        }
    }
    int cz = c % g.nc[2], cy = (c / g.nc[2]) % g.nc[1], cx = c / (g.nc[2] * g.nc[1]);
    int cc[3] = {cx, cy, cz};
    bool badtype = false;
    for (int s = b; s < e; ++s) {
        int i = perm[s];
        R rel[3];
        if (relp) {
            // written by k_bin_count from the same position
            const typename V4<R>::T q = relp[i];
            rel[0] = q.x; rel[1] = q.y; rel[2] = q.z;
        } else if (g.tric) {
            double p[3], r3[3];
            int c3[3];
            for (int d = 0; d < 3; ++d) {
                p[d] = x[d * g.n + i];
                if (!isfinite(p[d])) p[d] = 0.0;
            }
            cell_tric(g, p, c3, r3);
            for (int d = 0; d < 3; ++d) rel[d] = (R)r3[d];
        } else {
            for (int d = 0; d < 3; ++d) {
                double p = x[d * g.n + i];
                if (!isfinite(p)) p = 0.0;
                double w;
                cell_coord(p, d, g, w);
                rel[d] = (R)(w - cc[d] * g.lc[d]);
            }
        }
        typename V4<R>::T q;
        q.x = rel[0]; q.y = rel[1]; q.z = rel[2];
        int t = types[i];
        if (t < 0 || t >= g.ntypes) { badtype = true; t = 0; }
        q.w = (R)t;
        pos4[s] = q;
        cell_sorted[s] = c;
        if (invperm) invperm[i] = s;
    }
    if (badtype) atomicOr(status, ST_BADTYPE);
}

// k_cell_finalize with the cell-relative positions from k_bin_count (rel):
// one warp per cell.  A cell of at most 32 atoms is ordered by ranking (each
// lane counts the smaller caller indices of the cell by shuffles) and its
// atoms are then written by all lanes at once; a larger cell is ordered by
// lane 0 (insertion sort) and written in chunks of 32.
template <typename R>
__global__ void __launch_bounds__(256) k_cell_finalize_w(
    Grid g, int ncell, const int* __restrict__ start, int* __restrict__ perm,
    const int32_t* __restrict__ types, typename V4<R>::T* __restrict__ pos4,
    int* __restrict__ cell_sorted, int* __restrict__ status, const int* __restrict__ gate,
    int* __restrict__ invperm, const typename V4<R>::T* __restrict__ rel)
{
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;   // whole warps leave together
    const int zs = g.zs > 1 ? g.zs : 1;
    const int b = start[c * zs], e = start[(c + 1) * zs], cnt = e - b;
    bool badtype = false;
    auto place = [&](int s, int i) {
        const typename V4<R>::T q = rel[i];
        typename V4<R>::T o;
        o.x = q.x; o.y = q.y; o.z = q.z;
        int t = types[i];
        if (t < 0 || t >= g.ntypes) { badtype = true; t = 0; }
        o.w = (R)t;
        pos4[s] = o;
        cell_sorted[s] = c;
        if (invperm) invperm[i] = s;
    };
    if (cnt <= 32) {
        // rank by (z slice, caller index): the slices are already contiguous
        const int v = lane < cnt ? perm[b + lane] : 0x7fffffff;
        int sl = 0;
        for (int u = 1; u < zs; ++u) sl += b + lane >= start[c * zs + u];
        int rank = 0;
        for (int j = 0; j < cnt; ++j) {
            const int vj = __shfl_sync(0xffffffffu, v, j), sj = __shfl_sync(0xffffffffu, sl, j);
            rank += sj < sl || (sj == sl && vj < v);
        }
        if (lane < cnt) {
            perm[b + rank] = v;
            place(b + rank, v);
        }
    } else {
        if (lane == 0)
            for (int u = 0; u < zs; ++u) {   // each z slice by caller index
                const int bu = start[c * zs + u], eu = start[c * zs + u + 1];
                for (int s = bu + 1; s < eu; ++s) {
                    int v = perm[s], t = s;
                    while (t > bu && perm[t - 1] > v) { perm[t] = perm[t - 1]; --t; }
                    perm[t] = v;
                }
            }
        __syncwarp();
        for (int s = b + lane; s < e; s += 32) place(s, perm[s]);
    }
    if (__any_sync(0xffffffffu, badtype) && lane == 0) atomicOr(status, ST_BADTYPE);
}

// ----------------------------------------------------------------------------
// Neighbour lists: 27-cell stencil, minimum image through the stencil offset
// ----------------------------------------------------------------------------

// The 27 stencil offsets (cell-edge multiples) of the neighbour codes, in
// shared memory; filled by the first 27 threads of the block.
template <typename R>
__device__ __forceinline__ typename V4<R>::T stencil_entry(int code, const Grid& g)
{
    int a = code / 9, b = (code / 3) % 3, c = code % 3;
    typename V4<R>::T o;
    if (g.tric) {
        o.x = (R)stencil_off_tric(g, a - 1, b - 1, c - 1, 0);
        o.y = (R)stencil_off_tric(g, a - 1, b - 1, c - 1, 1);
        o.z = (R)stencil_off_tric(g, a - 1, b - 1, c - 1, 2);
    } else {
        o.x = (R)((a - 1) * g.lc[0]);
        o.y = (R)((b - 1) * g.lc[1]);
        o.z = (R)((c - 1) * g.lc[2]);
    }
    o.w = R(0);
    return o;
}
template <typename R>
__device__ __forceinline__ void fill_stencil(typename V4<R>::T* tab, const Grid& g)
{
    if (threadIdx.x < 27) tab[threadIdx.x] = stencil_entry<R>(threadIdx.x, g);
    __syncthreads();
}

// The same offsets split by component (three 27-entry arrays, the same
// values).  A warp's lookups with arbitrary codes then touch 27 distinct
// banks per component (one shared-memory wavefront each), where 16-byte
// entries, one per code, conflict (~6 wavefronts per warp-wide lookup).
template <typename R>
struct StencilSplit {
    R x[27], y[27], z[27];
};
template <typename R>
__device__ __forceinline__ void fill_stencil_split(StencilSplit<R>& t, const Grid& g)
{
    if (threadIdx.x < 27) {
        const typename V4<R>::T o = stencil_entry<R>(threadIdx.x, g);
        t.x[threadIdx.x] = o.x;
        t.y[threadIdx.x] = o.y;
        t.z[threadIdx.x] = o.z;
    }
    __syncthreads();
}

// FP64 displacement x_j - x_i of two atoms given by caller index (minimum
// image along the periodic directions).
__device__ __forceinline__ void disp64(const Grid& g, const double* __restrict__ x64, int i, int j,
                                       double (&d)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double t = x64[(size_t)c * g.n + j] - x64[(size_t)c * g.n + i];
        if (!g.tric && g.pbc[c]) t -= g.L[c] * rint(t * g.invL[c]);
        d[c] = t;
    }
    if (g.tric) min_image_tric(g, d);
}

// Close pairs on the FP32 path.  The displacement formed from cell-relative
// FP32 coordinates carries an absolute error of up to ~2e-6 A (three rounded
// coordinates and two roundings of the sums, each <= half an ulp at < 8 A),
// which is a relative error of ~7e-6 at r = 0.3 A, passed on to every NEP
// pair term of the pair.  Pairs closer than the outer ZBL radius (rare
// outside cascades) therefore take their displacement from the FP64
// positions, rounded once to FP32 (relative error <= 2^-24 per component).
// close2: the squared outer ZBL radius; k, m: cell-ordered slots of i and j.
template <typename R>
__device__ __forceinline__ void close_pair_fp64(R close2, const Grid& g,
                                                const double* __restrict__ x64,
                                                const int* __restrict__ perm, int k, int m, R& dx,
                                                R& dy, R& dz, R& r2)
{
    if constexpr (sizeof(R) == 4) {
        if (r2 < close2) {
            double d[3];
            disp64(g, x64, perm[k], perm[m], d);
            dx = (R)d[0];
            dy = (R)d[1];
            dz = (R)d[2];
            r2 = dx * dx + dy * dy + dz * dz;
        }
    }
}

// Radial basis coefficients for the neighbour kernel that also sums the
// radial descriptor (one species).
template <typename R>
struct RadCoef {
    R inv_rcR;
    R hR[NR * KR], CR[NR];
    R close2;   // squared outer ZBL radius (close pairs, see close_pair_fp64)
};

// WQ: also the radial descriptor q_n of every atom (one species, lists
// rebuilt every step), from the pairs the force kernels will see: after the
// search each thread walks its own freshly written list with the
// displacement in the force kernels' form (pj - pi) + offset, so pairs with
// r >= r_c in that form are left out as they skip them.  The search itself
// only tests and stores (few lanes of a warp hit at any one candidate, so
// descriptor work inside the hit branch would run with most lanes idle).
// TRIC: triclinic cells (stencil offsets are vectors; the orthorhombic
// instantiation keeps per-axis offsets).
// CH: the candidates of a stencil cell are tested in unrolled chunks of CHW
// that only set hit bits (angular, radial); the set bits are stored
// afterwards in candidate order.  The chunk reads up to CHW - 1 positions
// past the range, so pos4 must hold NB_CHUNK - 1 >= CHW - 1 readable entries
// past the last atom; the bits of those are masked off.
// Orthorhombic cells (CH): only the candidates that can be within reach are
// tested.  A stencil column (ox, oy) whose nearest point is farther than the
// list cutoff r_l in x/y is skipped; otherwise its z reach is
// R = sqrt(r_l^2 - dx_min^2 - dy_min^2) (+ a 1e-3 A margin), and of each cell
// of the column only the z slices (see Grid::zs) that overlap
// [z_i - R, z_i + R] are tested.  The lateral bound uses the cell extents in
// periodic directions only (atoms outside an open extent are clamped into
// the edge cells); the z slices clamp the same way, so the windows are exact
// in every case.  Every candidate left out is farther than r_l, so the lists
// hold the same pairs for any zs and CHW (in slice order within a cell).
constexpr int NB_CHUNK = 16;
// MSW > 0 (with WQ, several species): the basis sums per neighbour species,
// MSW >= T slots, and q_n = sum_t [C_n(t_i, t) Sb_t,0 + sum_k h_nk(t_i, t) Sb_t,k]
// with the pair coefficients from coefR ([T * T][CSTR], radial block).
template <typename R, bool WQ, bool TRIC = false, bool CH = false, int CHW = NB_CHUNK, int MSW = 0>
__global__ void __launch_bounds__(128, MSW ? 6 : 8) k_neighbors(Grid g, R rcR2, R rcA2,
                                                   const typename V4<R>::T* __restrict__ pos4,
                                                   const int* __restrict__ cell_sorted,
                                                   const int* __restrict__ start,
                                                   int* __restrict__ nbr, int2* __restrict__ cnt,
                                                   int* __restrict__ status,
                                                   int* __restrict__ maxc,
                                                   unsigned long long* __restrict__ pairs,
                                                   const int* __restrict__ gate,
                                                   const RadCoef<R> rq, R* __restrict__ qr,
                                                   const int* __restrict__ perm,
                                                   const double* __restrict__ x64,
                                                   int* __restrict__ tflag = nullptr,
                                                   const R* __restrict__ coefR = nullptr)
{
    using P4 = typename V4<R>::T;
    if (gate && *gate == 0) return;   // lists still valid (Verlet skin)
    __shared__ P4 s_off[WQ ? 27 : 1];
    if constexpr (WQ) fill_stencil<R>(s_off, g);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    // tot: all hits (overflow test); sa / sro: stored angular / radial-only
    int tot = 0, sa = 0, sro = 0;
    if (k < g.n) {
        const P4 p = pos4[k];
        const int c = cell_sorted[k];
        const int ncx = g.nc[0], ncy = g.nc[1], ncz = g.nc[2];
        const int cz = c % ncz, cy = (c / ncz) % ncy, cx = c / (ncz * ncy);
        // cell edges in R: the offsets ox * lc are exact multiples, the same
        // values the force kernel adds for the stencil codes
        const R lx = (R)g.lc[0], ly = (R)g.lc[1], lz = (R)g.lc[2];
        const int M = g.M;
        int* col = nbr + k;
        const size_t ld = (size_t)g.ld;
        const int zs = TRIC ? 1 : (g.zs > 1 ? g.zs : 1);
        const R zsl = (R)(zs * g.inv_lc[2]);   // slices per A along z
        // reach tests with the list cutoff widened by 1e-3 A (far above the
        // rounding of these FP32 bounds): no candidate within r_l is lost
        const R rl_m = sqrt(rcR2) + R(1e-3), rl_m2 = rl_m * rl_m;
        for (int ox = -1; ox <= 1; ++ox) {
            int X = cx + ox;
            if (g.pbc[0]) { X += X < 0 ? ncx : 0; X -= X >= ncx ? ncx : 0; }
            else if (X < 0 || X >= ncx) continue;
            const R px0 = p.x - R(ox) * lx;
            // nearest x of the column's atoms (periodic: inside [0, lx))
            R dxm = R(0);
            if (!TRIC && CH && g.pbc[0] && ox != 0)
                dxm = ox > 0 ? lx - p.x : p.x;
            dxm = dxm > R(0) ? dxm : R(0);
            for (int oy = -1; oy <= 1; ++oy) {
                int Y = cy + oy;
                if (g.pbc[1]) { Y += Y < 0 ? ncy : 0; Y -= Y >= ncy ? ncy : 0; }
                else if (Y < 0 || Y >= ncy) continue;
                const R py0 = p.y - R(oy) * ly;
                R dym = R(0);
                if (!TRIC && CH && g.pbc[1] && oy != 0)
                    dym = oy > 0 ? ly - p.y : p.y;
                dym = dym > R(0) ? dym : R(0);
                const R reach2 = rl_m2 - dxm * dxm - dym * dym;
                if (!TRIC && CH && reach2 <= R(0)) continue;   // column out of reach
                const R reach = TRIC || !CH ? R(0) : sqrt(reach2);
                const int rowXY = (X * ncy + Y) * ncz;
                for (int oz = -1; oz <= 1; ++oz) {
                    int Z = cz + oz;
                    if (g.pbc[2]) { Z += Z < 0 ? ncz : 0; Z -= Z >= ncz ? ncz : 0; }
                    else if (Z < 0 || Z >= ncz) continue;
                    // offset of this stencil cell: the values the force
                    // kernels add for the code (fill_stencil)
                    R px = px0, py = py0, pz = p.z - R(oz) * lz;
                    if constexpr (TRIC) {
                        px = p.x - (R)stencil_off_tric(g, ox, oy, oz, 0);
                        py = p.y - (R)stencil_off_tric(g, ox, oy, oz, 1);
                        pz = p.z - (R)stencil_off_tric(g, ox, oy, oz, 2);
                    }
                    const int code = (ox + 1) * 9 + (oy + 1) * 3 + (oz + 1);
                    const int c2 = rowXY + Z;
                    if constexpr (CH) {
                        // the cell's z slices within reach of pz (clamped: the
                        // edge slices of a cell hold any atom beyond them)
                        int t0 = 0, t1 = zs - 1;
                        if (!TRIC && zs > 1) {
                            const R zlo = pz - reach, zhi = pz + reach;
                            // nothing within reach (atoms of periodic or
                            // interior cells lie inside [0, lz))
                            const bool inside = g.pbc[2] || (Z > 0 && Z < ncz - 1);
                            if (inside && (zhi < R(0) || zlo >= lz)) continue;
                            t0 = (int)floor(zlo * zsl);
                            t1 = (int)floor(zhi * zsl);
                            t0 = t0 < 0 ? 0 : (t0 >= zs ? zs - 1 : t0);
                            t1 = t1 < 0 ? 0 : (t1 >= zs ? zs - 1 : t1);
                        } else if (!TRIC && g.pbc[2]) {
                            if (pz + reach < R(0) || pz - reach >= lz) continue;
                        }
                        const int e = start[c2 * zs + t1 + 1];
                        for (int m0 = start[c2 * zs + t0]; m0 < e; m0 += CHW) {
                            const P4* q0 = pos4 + m0;
                            unsigned hr = 0u, ha = 0u;   // r < rc_R, r < rc_A
#pragma unroll
                            for (int j = 0; j < CHW; ++j) {
                                const P4 q = q0[j];
                                const R dx = q.x - px, dy = q.y - py, dz = q.z - pz;
                                const R r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 < rcR2) hr |= 1u << j;
                                if (r2 < rcA2) ha |= 1u << j;
                            }
                            // this range's atoms only, never the atom itself
                            const int nv = e - m0;
                            unsigned keep = nv >= CHW ? (CHW == 32 ? 0xffffffffu : (1u << CHW) - 1u)
                                                      : (1u << nv) - 1u;
                            const unsigned self = (unsigned)(k - m0);
                            if (self < (unsigned)CHW) keep &= ~(1u << self);
                            ha &= hr & keep;
                            hr &= keep & ~ha;   // radial only
                            const int na_c = __popc(ha), nr_c = __popc(hr);
                            tot += na_c + nr_c;
                            const int base = (m0 << 5) | code;   // entry of candidate j: base + 32 j
                            if (sa + sro + na_c + nr_c <= M) {
                                // room for all of them: no test per hit
                                int* pa = col + (size_t)sa * ld;
                                while (ha) {
                                    *pa = base + ((__ffs(ha) - 1) << 5);
                                    ha &= ha - 1u;
                                    pa += ld;
                                }
                                int* pr = col + (size_t)(M - 1 - sro) * ld;
                                while (hr) {
                                    *pr = base + ((__ffs(hr) - 1) << 5);
                                    hr &= hr - 1u;
                                    pr -= ld;
                                }
                                sa += na_c;
                                sro += nr_c;
                            } else {
                                while (ha) {
                                    const int j = __ffs(ha) - 1;
                                    ha &= ha - 1u;
                                    if (sa + sro < M) col[(size_t)(sa++) * ld] = base + (j << 5);
                                }
                                while (hr) {
                                    const int j = __ffs(hr) - 1;
                                    hr &= hr - 1u;
                                    if (sa + sro < M) col[(size_t)(M - 1 - sro++) * ld] = base + (j << 5);
                                }
                            }
                        }
                    } else {
                        const int zsn = g.zs > 1 ? g.zs : 1;
                        const int e = start[(c2 + 1) * zsn];
                        for (int m = start[c2 * zsn]; m < e; ++m) {
                            const P4 q = pos4[m];
                            const R dx = q.x - px, dy = q.y - py, dz = q.z - pz;
                            const R r2 = dx * dx + dy * dy + dz * dz;
                            const bool hit = r2 < rcR2 && m != k;
                            const bool ang = r2 < rcA2;
                            const bool room = sa + sro < M;
                            if (hit && room)
                                col[(size_t)(ang ? sa : M - 1 - sro) * ld] = (m << 5) | code;
                            tot += hit;
                            sa += hit && room && ang;
                            sro += hit && room && !ang;
                        }
                    }
                }
            }
        }
        cnt[k] = make_int2(sa, sro);
        if (tot > M) atomicOr(status, ST_OVERFLOW);
        if constexpr (WQ) {
            // Sb_k = sum_j f_c T_k over the stored pairs within r_c in the
            // force kernels' form; q_n = C_n Sb_0 + sum_k h_nk Sb_k.  Entry
            // s + 2 and position s + 1 are in flight during pair s.
            R Sb[KR];
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) Sb[kk] = R(0);
            constexpr int NS = MSW > 0 ? MSW : 1;
            R Sm[NS][KR];   // several species: per neighbour species
#pragma unroll
            for (int t = 0; t < NS; ++t)
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) Sm[t][kk] = R(0);
            bool close = false;
            const int ns = sa + sro;
            auto slot = [&](int t) { return t < sa ? t : M - 1 - (t - sa); };
            int ent_n = ns > 0 ? col[(size_t)slot(0) * ld] : 0;
            int ent_nn = ns > 1 ? col[(size_t)slot(1) * ld] : 0;
            P4 pj_n = ns > 0 ? pos4[ent_n >> 5] : p;
            for (int t = 0; t < ns; ++t) {
                const int ent = ent_n;
                const P4 pj = pj_n;
                ent_n = ent_nn;
                if (t + 1 < ns) pj_n = pos4[ent_n >> 5];
                if (t + 2 < ns) ent_nn = col[(size_t)slot(t + 2) * ld];
                const P4 off = s_off[ent & 31];
                R fx = pj.x - p.x + off.x, fy = pj.y - p.y + off.y, fz = pj.z - p.z + off.z;
                R f2 = fx * fx + fy * fy + fz * fz;
                if (f2 < rcR2) {
                    close |= f2 < rq.close2;
                    close_pair_fp64<R>(rq.close2, g, x64, perm, k, ent >> 5, fx, fy, fz, f2);
                    const R rr = f2 * nepm::nep_rsqrt(f2);
                    R T[KR], dT[KR], fc, dfc, dxdr;
                    nepm::cheb<KR, false>(rr, rq.inv_rcR, T, dT, fc, dfc, dxdr);
                    if constexpr (MSW > 0) {
                        const int tj = (int)pj.w;
#pragma unroll
                        for (int t = 0; t < NS; ++t) {
                            const R wt = tj == t ? fc : R(0);
#pragma unroll
                            for (int kk = 0; kk < KR; ++kk) Sm[t][kk] += wt * T[kk];
                        }
                    } else if constexpr (sizeof(R) == 4) {
                        // packed pairs: one FFMA2 per two basis functions
#pragma unroll
                        for (int kk = 0; kk + 1 < KR; kk += 2) {
                            const float2 t = __ffma2_rn(make_float2(fc, fc),
                                                        make_float2(T[kk], T[kk + 1]),
                                                        make_float2(Sb[kk], Sb[kk + 1]));
                            Sb[kk] = t.x;
                            Sb[kk + 1] = t.y;
                        }
                        Sb[KR - 1] += fc * T[KR - 1];
                    } else {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) Sb[kk] += fc * T[kk];
                    }
                }
            }
            if constexpr (MSW > 0) {
                const int T = g.ntypes, ti = (int)p.w;
                R q[NR];
#pragma unroll
                for (int n = 0; n < NR; ++n) q[n] = R(0);
#pragma unroll
                for (int t = 0; t < NS; ++t) {
                    if (t < T) {
                        const R* c = coefR + ((size_t)ti * T + t) * CSTR + C_RAD;
#pragma unroll
                        for (int n = 0; n < NR; ++n) {
                            R acc = c[NR * KR + n] * Sm[t][0];
#pragma unroll
                            for (int kk = 0; kk < KR; ++kk) acc += c[n * KR + kk] * Sm[t][kk];
                            q[n] += acc;
                        }
                    }
                }
#pragma unroll
                for (int n = 0; n < NR; ++n) qr[(size_t)n * ld + k] = q[n];
            } else {
#pragma unroll
                for (int n = 0; n < NR; ++n) {
                    R acc = rq.CR[n] * Sb[0];
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) acc += rq.hR[n * KR + kk] * Sb[kk];
                    qr[(size_t)n * ld + k] = acc;
                }
            }
            // this tile's kernel choice (blocks of TILE atoms: block = tile)
            const int bits = (close ? TILE_CLOSE : 0) | (sa > TILE_ANG_LIM ? TILE_DENSE : 0);
            if (tflag && bits) tile_mark(tflag, (g.n + TILE - 1) / TILE, blockIdx.x, bits);
        }
    }
    // statistics: block maxima and pair sums
    int na = sa;
    unsigned long long pr = (unsigned long long)tot, pa = (unsigned long long)sa;
    for (int o = 16; o > 0; o >>= 1) {
        tot = max(tot, __shfl_xor_sync(0xffffffffu, tot, o));
        na = max(na, __shfl_xor_sync(0xffffffffu, na, o));
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pa += __shfl_xor_sync(0xffffffffu, pa, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (tot > 0) atomicMax(&maxc[0], tot);
        if (na > 0) atomicMax(&maxc[1], na);
        if (pr) atomicAdd(&pairs[0], pr);
        if (pa) atomicAdd(&pairs[1], pa);
    }
}

// ----------------------------------------------------------------------------
// Verlet skin: lists built with r_c + skin are reused until an atom has moved
// more than skin/2 since the last build (then no pair can have crossed r_c
// unseen).  The rebuild kernels above return at once when *gate == 0.
// ----------------------------------------------------------------------------

// gate |= any atom moved more than skin/2 (minimum image in periodic dims)
static __global__ void k_skin_check(Grid g, const double* __restrict__ x,
                                    const double* __restrict__ xref, double thr2,
                                    int* __restrict__ gate)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool moved = false;
    if (i < g.n) {
        double d2 = 0.0;
        if (g.tric) {
            double d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) d[a] = x[(size_t)a * g.n + i] - xref[(size_t)a * g.n + i];
            min_image_tric(g, d);
            d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double d = x[(size_t)a * g.n + i] - xref[(size_t)a * g.n + i];
                if (g.pbc[a]) d -= g.L[a] * rint(d * g.invL[a]);
                d2 += d * d;
            }
        }
        moved = !(d2 <= thr2);   // NaN also forces a rebuild
    }
    if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) atomicOr(gate, 1);
}

// count[0..n) = 0 and the reference positions <- x, when rebuilding
static __global__ void k_skin_rebuild_prep(int* __restrict__ count, int ncell,
                                           const double* __restrict__ x,
                                           double* __restrict__ xref, int n3,
                                           const int* __restrict__ gate,
                                           unsigned long long* __restrict__ nrebuild)
{
    if (*gate == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) atomicAdd(nrebuild, 1ull);
    if (i <= ncell) count[i] = 0;
    if (i < n3) xref[i] = x[i];
}

// cell-relative positions from the current FP64 positions, cells fixed since
// the last build (minimum image with respect to the cell in periodic dims)
template <typename R>
__global__ void k_refresh_pos4(Grid g, const int* __restrict__ perm,
                               const int* __restrict__ cell_sorted,
                               const double* __restrict__ x,
                               typename V4<R>::T* __restrict__ pos4)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const int i = perm[k];
    const int c = cell_sorted[k];
    const int cc[3] = {c / (g.nc[2] * g.nc[1]), (c / g.nc[2]) % g.nc[1], c % g.nc[2]};
    R rel[3];
    if (g.tric) {
        double d[3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
            d[b] = x[(size_t)b * g.n + i] - ((double)cc[0] * g.h[b] / g.nc[0] +
                                             (double)cc[1] * g.h[3 + b] / g.nc[1] +
                                             (double)cc[2] * g.h[6 + b] / g.nc[2]);
        min_image_tric(g, d);
#pragma unroll
        for (int b = 0; b < 3; ++b) rel[b] = (R)d[b];
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double d = x[(size_t)a * g.n + i] - cc[a] * g.lc[a];
            if (g.pbc[a]) d -= g.L[a] * rint(d * g.invL[a]);
            rel[a] = (R)d;
        }
    }
    typename V4<R>::T q = pos4[k];
    q.x = rel[0]; q.y = rel[1]; q.z = rel[2];
    pos4[k] = q;
}

// ----------------------------------------------------------------------------
// Force accumulation policy
// ----------------------------------------------------------------------------

template <typename R> struct Acc;

// FP32 path: 64-bit fixed point with 2^-32 eV/A resolution; integer sums do
// not depend on the order of the atomics, so the forces are deterministic.
template <> struct Acc<float> {
    using T = long long;
    static constexpr double SCALE = 4294967296.0;
    __device__ static __forceinline__ long long conv(float f)
    {
        return __float2ll_rn(f * 4294967296.0f);
    }
    __device__ static __forceinline__ long long convd(double f)
    {
        return __double2ll_rn(f * 4294967296.0);
    }
    __device__ static __forceinline__ void add(long long* p, long long v)
    {
        atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
    }
    __device__ static __forceinline__ double value(long long v) { return (double)v * (1.0 / 4294967296.0); }
};

template <> struct Acc<double> {
    using T = double;
    __device__ static __forceinline__ double conv(double f) { return f; }
    __device__ static __forceinline__ double convd(double f) { return f; }
    __device__ static __forceinline__ void add(double* p, double v) { atomicAdd(p, v); }
    __device__ static __forceinline__ double value(double v) { return v; }
};

// The FP32 one-species radial record of atom k (position and radial adjoint,
// written by the angular kernels, gathered per neighbour by k_radial_force):
// rec[3k] = (x, y, z, b_8), rec[3k + 1] = (b_0 + B0, b_1, b_2, b_3),
// rec[3k + 2] = (b_4..b_7).
__device__ __forceinline__ void rec_store(float4* __restrict__ rec, size_t k, const float4 r0,
                                          const float4 r1, const float4 r2)
{
    rec[3 * k] = r0;
    rec[3 * k + 1] = r1;
    rec[3 * k + 2] = r2;
}
// ZBL pair term of Eq. 2-4 with the Tersoff switch, in FP64: U and dU/dr.
__device__ __forceinline__ void zbl_pair(double r, double k, double inv_a, double r1, double r2,
                                         double& U, double& dU)
{
    double x = r * inv_a;
    double e1 = 0.32825 * exp(-2.54931 * x);
    double e2 = 0.09219 * exp(-0.29182 * x);
    double e3 = 0.58110 * exp(-0.59231 * x);
    double phi = e1 + e2 + e3;
    double dphi = -(2.54931 * e1 + 0.29182 * e2 + 0.59231 * e3);   // d phi / dx
    double fc = 1.0, dfc = 0.0;
    if (r >= r1) {
        double s, c;
        sincospi((r - r1) / (r2 - r1), &s, &c);
        fc = 0.5 + 0.5 * c;
        dfc = -0.5 * M_PI / (r2 - r1) * s;
    }
    double inv_r = 1.0 / r;
    double v = k * inv_r * phi;
    double dv = -v * inv_r + k * inv_r * dphi * inv_a;
    U = v * fc;
    dU = dv * fc + v * dfc;
}

// ----------------------------------------------------------------------------
// Per-atom building blocks (inlined into the force kernels)
// ----------------------------------------------------------------------------

// Adds one neighbour (displacement d) to the descriptor sums of an atom: the
// radial basis sums Sb_k = sum_j f_c T_k(x_j) (q_n follows per atom from
// radial_q) and, for an angular neighbour, A_nlm = sum_j g_n Y_lm.
template <typename R>
__device__ __forceinline__ void desc_pair(const Model<R>& P, R dx, R dy, R dz, R r, R inv_r,
                                          bool ang, R (&Sb)[KR], R (&A)[NA][NLM])
{
    R T[KR], dT[KR], fc, dfc, dxdr;
    nepm::cheb<KR, false>(r, P.inv_rcR, T, dT, fc, dfc, dxdr);
#pragma unroll
    for (int kk = 0; kk < KR; ++kk) Sb[kk] += fc * T[kk];
    if (ang) {
        nepm::cheb<KA, false>(r, P.inv_rcA, T, dT, fc, dfc, dxdr);
        R Y[NLM];
        nepm::harmonics(dx * inv_r, dy * inv_r, dz * inv_r, Y);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            R acc = P.CA[n];
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) acc += P.hA[n * KA + kk] * T[kk];
            const R gn = fc * acc;
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) A[n][lm] += gn * Y[lm];
        }
    }
}

// q_n = sum_j g_n(r_j) = C_n Sb_0 + sum_k h_nk Sb_k (T_0 = 1).
template <typename R>
__device__ __forceinline__ void radial_q(const Model<R>& P, const R (&Sb)[KR], R (&qR)[NR])
{
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        R acc = P.CR[n] * Sb[0];
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) acc += P.hR[n * KR + kk] * Sb[kk];
        qR[n] = acc;
    }
}

// Network U(q) and its backward.  On return A holds dU/dA_nlm (4-body term
// folded into l = 2) and aR the radial adjoint dU/dq_n.
template <typename R>
__device__ __forceinline__ R network_adjoint_core(const Model<R>& P, const R (&qR)[NR],
                                                  R (&A)[NA][NLM], R (&aR)[NR])
{
    R h[H];
#pragma unroll
    for (int mu = 0; mu < H; ++mu) h[mu] = -P.b0[mu];
#pragma unroll
    for (int nu = 0; nu < NR; ++nu)
#pragma unroll
        for (int mu = 0; mu < H; ++mu) h[mu] += P.w0[mu * D + nu] * qR[nu];
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;   // harmonic range
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            R q = R(0);
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) q += A[n][lm] * A[n][lm];
            const int nu = NR + (l - 1) * NA + n;
#pragma unroll
            for (int mu = 0; mu < H; ++mu) h[mu] += P.w0[mu * D + nu] * q;
        }
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        const R q4 = nepm::fourbody(&A[n][3], (R*)nullptr);
        const int nu = NR + LM * NA + n;
#pragma unroll
        for (int mu = 0; mu < H; ++mu) h[mu] += P.w0[mu * D + nu] * q4;
    }
    R U = -P.b1;
#pragma unroll
    for (int mu = 0; mu < H; ++mu) {
        const R t = tanh(h[mu]);
        U += P.w1[mu] * t;
        h[mu] = P.w1[mu] * (R(1) - t * t);   // dU/dh_mu
    }
#pragma unroll
    for (int nu = 0; nu < NR; ++nu) {
        R a = R(0);
#pragma unroll
        for (int mu = 0; mu < H; ++mu) a += h[mu] * P.w0[mu * D + nu];
        aR[nu] = a;
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        R a4 = R(0), a2 = R(0);
#pragma unroll
        for (int mu = 0; mu < H; ++mu) {
            a4 += h[mu] * P.w0[mu * D + NR + LM * NA + n];
            a2 += h[mu] * P.w0[mu * D + NR + NA + n];
        }
        R dq4[5];
        nepm::fourbody(&A[n][3], dq4);
#pragma unroll
        for (int t = 0; t < 5; ++t) A[n][3 + t] = R(2) * a2 * A[n][3 + t] + a4 * dq4[t];
    }
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        if (l == 2) continue;
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            R a = R(0);
#pragma unroll
            for (int mu = 0; mu < H; ++mu) a += h[mu] * P.w0[mu * D + NR + (l - 1) * NA + n];
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) A[n][lm] *= R(2) * a;
        }
    }
    return U;
}

// Rows of the network for the rolled loop below: row mu holds
// (w0[mu][0..29] s, b0_mu, w1_mu), 32 values, in shared memory.
constexpr int WROW = 32;
static_assert(D + 2 == WROW, "network row layout");

template <typename R>
__device__ __forceinline__ void fill_network_rows(R* sw, const Model<R>& P)
{
    for (int t = threadIdx.x; t < H * WROW; t += blockDim.x) {
        const int mu = t / WROW, c = t % WROW;
        sw[t] = c < D ? P.w0[mu * D + c] : (c == D ? P.b0[mu] : P.w1[mu]);
    }
}

template <typename R>
__device__ __forceinline__ void load_row(const R* __restrict__ src, R (&w)[WROW]);
template <>
__device__ __forceinline__ void load_row<float>(const float* __restrict__ src, float (&w)[WROW])
{
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int c = 0; c < WROW / 4; ++c) {
        const float4 v = s4[c];
        w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
    }
}
template <>
__device__ __forceinline__ void load_row<double>(const double* __restrict__ src, double (&w)[WROW])
{
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int c = 0; c < WROW / 2; ++c) {
        const double2 v = s2[c];
        w[2 * c] = v.x; w[2 * c + 1] = v.y;
    }
}

// network_adjoint_core with the hidden layer as one rolled loop over the
// neurons: for each mu the row is read from shared memory (sw, see
// fill_network_rows), h_mu = sum_nu w_mu,nu q_nu - b0_mu, and its term
// w1_mu (1 - tanh^2) w_mu,nu is added to dU/dq_nu at once, so forward and
// backward share one pass over the weights and the code stays small.  Same
// sums in the same order as network_adjoint_core.
template <typename R>
__device__ __forceinline__ R network_adjoint_core_rolled(const Model<R>& P,
                                                         const R* __restrict__ sw,
                                                         const R (&qR)[NR], R (&A)[NA][NLM],
                                                         R (&aR)[NR])
{
    R q[D];
#pragma unroll
    for (int nu = 0; nu < NR; ++nu) q[nu] = qR[nu];
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            R v = R(0);
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) v += A[n][lm] * A[n][lm];
            q[NR + (l - 1) * NA + n] = v;
        }
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) q[NR + LM * NA + n] = nepm::fourbody(&A[n][3], (R*)nullptr);
    R a[D];
#pragma unroll
    for (int nu = 0; nu < D; ++nu) a[nu] = R(0);
    R U = -P.b1;
#pragma unroll 1
    for (int mu = 0; mu < H; ++mu) {
        R w[WROW];
        load_row<R>(sw + mu * WROW, w);
        R h = -w[D];
#pragma unroll
        for (int nu = 0; nu < D; ++nu) h += w[nu] * q[nu];
        const R t = tanh(h);
        U += w[D + 1] * t;
        const R gm = w[D + 1] * (R(1) - t * t);   // dU/dh_mu
#pragma unroll
        for (int nu = 0; nu < D; ++nu) a[nu] += gm * w[nu];
    }
#pragma unroll
    for (int nu = 0; nu < NR; ++nu) aR[nu] = a[nu];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        const R a4 = a[NR + LM * NA + n], a2 = a[NR + NA + n];
        R dq4[5];
        nepm::fourbody(&A[n][3], dq4);
#pragma unroll
        for (int t = 0; t < 5; ++t) A[n][3 + t] = R(2) * a2 * A[n][3 + t] + a4 * dq4[t];
    }
#pragma unroll
    for (int l = 1; l <= LM; ++l) {
        if (l == 2) continue;
        const int lo = l * l - 1, hi = (l + 1) * (l + 1) - 1;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            const R al = a[NR + (l - 1) * NA + n];
#pragma unroll
            for (int lm = lo; lm < hi; ++lm) A[n][lm] *= R(2) * al;
        }
    }
    return U;
}

// One species: the radial adjoint contracted with the basis coefficients,
// sum_n dU/dq_n g'_n(r) = df_c (B0 + sum_k bR_k T_k) + f_c x' sum_k bR_k T'_k.
template <typename R>
__device__ __forceinline__ R network_adjoint(const Model<R>& P, const R (&qR)[NR],
                                             R (&A)[NA][NLM], R (&bR)[KR], R& B0)
{
    R aR[NR];
    const R U = network_adjoint_core<R>(P, qR, A, aR);
    B0 = R(0);
#pragma unroll
    for (int kk = 0; kk < KR; ++kk) bR[kk] = R(0);
#pragma unroll
    for (int nu = 0; nu < NR; ++nu) {
        B0 += aR[nu] * P.CR[nu];
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) bR[kk] += aR[nu] * P.hR[nu * KR + kk];
    }
    return U;
}

// dU_i/dd_ij for one neighbour from the atom's adjoint (NEP part only).
template <typename R>
__device__ __forceinline__ void force_pair(const Model<R>& P, R r, R inv_r, R ux, R uy, R uz,
                                           bool ang, const R (&Ab)[NA][NLM], const R (&bR)[KR],
                                           R B0, R& fx, R& fy, R& fz)
{
    R T[KR], dT[KR], fc, dfc, dxdr;
    nepm::cheb<KR, true>(r, P.inv_rcR, T, dT, fc, dfc, dxdr);
    R s1 = B0, s2 = R(0);
#pragma unroll
    for (int kk = 0; kk < KR; ++kk) {
        s1 += bR[kk] * T[kk];
        s2 += bR[kk] * dT[kk];
    }
    R fs = dfc * s1 + fc * dxdr * s2;   // coefficient of u
    R vx = R(0), vy = R(0), vz = R(0);  // coefficient of 1/r
    if (ang) {
        nepm::cheb<KA, true>(r, P.inv_rcA, T, dT, fc, dfc, dxdr);
        R gn[NA], dgn[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            R a = P.CA[n], b = R(0);
#pragma unroll
            for (int kk = 0; kk < KA; ++kk) {
                a += P.hA[n * KA + kk] * T[kk];
                b += P.hA[n * KA + kk] * dT[kk];
            }
            gn[n] = fc * a;
            dgn[n] = dfc * a + fc * dxdr * b;
        }
        R Y[NLM], G[NLM];
        nepm::harmonics(ux, uy, uz, Y);
        R sang = R(0);
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
            R gsum = R(0), dsum = R(0);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                gsum += Ab[n][lm] * gn[n];
                dsum += Ab[n][lm] * dgn[n];
            }
            G[lm] = gsum;
            sang += (dsum - R(l) * inv_r * gsum) * Y[lm];
        }
        fs += sang;
        nepm::harmonics_grad_dot(ux, uy, uz, G, vx, vy, vz);
    }
    fx = fs * ux + vx * inv_r;
    fy = fs * uy + vy * inv_r;
    fz = fs * uz + vz * inv_r;
}

// ----------------------------------------------------------------------------
// The force kernel: one thread per atom (cell order), 128 atoms per block.
// Descriptor sums -> network and its backward -> pair forces scattered to
// both atoms of each pair -> per-tile energy and virial.
// ----------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(TILE) k_nep(const Model<R> P, const Grid g,
                                              const typename V4<R>::T* __restrict__ pos4,
                                              const int* __restrict__ nbr,
                                              const int2* __restrict__ cnt,
                                              const int* __restrict__ perm,
                                              const double* __restrict__ x64,
                                              typename Acc<R>::T* __restrict__ facc,
                                              double* __restrict__ partials,
                                              double* __restrict__ site_energy,
                                              int* __restrict__ status, int stage_slots)
{
    using A_ = Acc<R>;
    using P4 = typename V4<R>::T;
    __shared__ P4 s_off[27];
    __shared__ int s_max;
    extern __shared__ int s_ent[];   // [stage_slots][TILE] staged neighbour entries
    if (threadIdx.x == 0) s_max = 0;
    fill_stencil<R>(s_off, g);       // ends with __syncthreads
    const int k = blockIdx.x * TILE + threadIdx.x;
    const int M = g.M;
    const size_t ld = (size_t)g.ld;
    // the block's lists go to shared memory when its longest list fits
    const int2 cnt_k = k < g.n ? cnt[k] : make_int2(0, 0);
    atomicMax(&s_max, cnt_k.x + cnt_k.y);
    __syncthreads();
    const bool staged = s_max <= stage_slots;
    if (staged && k < g.n) {
        for (int s = 0; s < cnt_k.x; ++s) s_ent[s * TILE + threadIdx.x] = nbr[(size_t)s * ld + k];
        for (int u = 0; u < cnt_k.y; ++u)
            s_ent[(cnt_k.x + u) * TILE + threadIdx.x] = nbr[(size_t)(M - 1 - u) * ld + k];
    }
    double e_site = 0.0;
    R w[9];                 // virial of the NEP pair terms (R)
    double wz[9];           // virial of the ZBL pair terms (FP64)
    bool has_zbl = false;
#pragma unroll
    for (int t = 0; t < 9; ++t) { w[t] = R(0); wz[t] = 0.0; }

    if (k < g.n) {
        const typename V4<R>::T pi = pos4[k];
        const int na = cnt_k.x, nro = cnt_k.y;
        // entry s of the list: angular pairs first, then radial-only pairs
        auto entry = [&](int s) -> int {
            if (staged) return s_ent[s * TILE + threadIdx.x];
            const int slot = s < na ? s : M - 1 - (s - na);
            return nbr[(size_t)slot * ld + k];
        };

        // ---------------- descriptor sums ----------------
        R Sb[KR];
        R A[NA][NLM];
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) Sb[kk] = R(0);
#pragma unroll
        for (int n = 0; n < NA; ++n)
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) A[n][lm] = R(0);

        const int total = na + nro;
        // two-stage prefetch: entry s + 2 and position s + 1 are loaded while
        // pair s is computed
        int ent_n = total > 0 ? entry(0) : 0;
        int ent_nn = total > 1 ? entry(1) : 0;
        P4 pj_n = total > 0 ? pos4[ent_n >> 5] : pi;
        for (int s = 0; s < total; ++s) {
            const int ent = ent_n;
            const P4 pj = pj_n;
            ent_n = ent_nn;
            if (s + 1 < total) pj_n = pos4[ent_n >> 5];
            if (s + 2 < total) ent_nn = entry(s + 2);
            const P4 off = s_off[ent & 31];
            R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, ent >> 5, dx, dy, dz, r2);
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            desc_pair<R>(P, dx, dy, dz, r, inv_r, s < na, Sb, A);
        }
        R qR[NR];
        radial_q<R>(P, Sb, qR);

        // ---------------- network and its backward ---------------------------
        R bR[KR], B0;
        const R U = network_adjoint<R>(P, qR, A, bR, B0);

        // ---------------- pair forces --------------------------------------
        typename A_::T fi[3] = {0, 0, 0};
        double ez = 0.0;
        bool bad = !isfinite(U);
        const int i_caller = perm[k];

        ent_n = total > 0 ? entry(0) : 0;
        ent_nn = total > 1 ? entry(1) : 0;
        pj_n = total > 0 ? pos4[ent_n >> 5] : pi;
        for (int s = 0; s < total; ++s) {
            const int ent = ent_n;
            const P4 pj = pj_n;
            ent_n = ent_nn;
            if (s + 1 < total) pj_n = pos4[ent_n >> 5];
            if (s + 2 < total) ent_nn = entry(s + 2);
            const int m = ent >> 5;
            const P4 off = s_off[ent & 31];
            R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, m, dx, dy, dz, r2);
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            const R ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
            R fx, fy, fz;
            force_pair<R>(P, r, inv_r, ux, uy, uz, s < na, A, bR, B0, fx, fy, fz);
            bad |= !isfinite(fx + fy + fz);
            typename A_::T cx = A_::conv(fx), cy = A_::conv(fy), cz = A_::conv(fz);
            // ZBL pair term (Eq. 1-4), FP64 from the FP64 positions
            if (s < na && r < P.zbl_r2) {
                double d64[3];
                if (sizeof(R) == 4) {
                    const int j_caller = perm[m];
                    for (int a = 0; a < 3; ++a) {
                        double t = x64[a * g.n + j_caller] - x64[a * g.n + i_caller];
                        if (!g.tric && g.pbc[a]) t -= g.L[a] * rint(t * g.invL[a]);
                        d64[a] = t;
                    }
                    if (g.tric) min_image_tric(g, d64);
                } else {
                    d64[0] = (double)dx; d64[1] = (double)dy; d64[2] = (double)dz;
                }
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
                    has_zbl = true;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) wz[3 * a + b] -= f3[a] * d64[b];
                }
            }
            fi[0] += cx; fi[1] += cy; fi[2] += cz;
            A_::add(&facc[m], -cx);
            A_::add(&facc[ld + m], -cy);
            A_::add(&facc[2 * ld + m], -cz);
            w[0] -= fx * dx; w[1] -= fx * dy; w[2] -= fx * dz;
            w[3] -= fy * dx; w[4] -= fy * dy; w[5] -= fy * dz;
            w[6] -= fz * dx; w[7] -= fz * dy; w[8] -= fz * dz;
        }
        A_::add(&facc[k], fi[0]);
        A_::add(&facc[ld + k], fi[1]);
        A_::add(&facc[2 * ld + k], fi[2]);
        e_site = (double)U + ez;
        if (site_energy) site_energy[i_caller] = e_site;
        if (bad) atomicOr(status, ST_NONFINITE);
    }

    // ---------------- per-tile energy and virial (fixed order) ----------------
    // energy: FP64 over the warp; NEP virial: R over the warp (32 atoms), then
    // FP64; ZBL virial: FP64, only in warps that have a ZBL pair
    __shared__ double red[TILE / 32][NPART];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_site += __shfl_xor_sync(0xffffffffu, e_site, o);
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[t] += __shfl_xor_sync(0xffffffffu, w[t], o);
    if (__any_sync(0xffffffffu, has_zbl)) {
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wz[t] += __shfl_xor_sync(0xffffffffu, wz[t], o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = e_site;
#pragma unroll
        for (int t = 0; t < 9; ++t) red[threadIdx.x >> 5][1 + t] = (double)w[t] + wz[t];
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        double s = 0.0;
#pragma unroll
        for (int wi = 0; wi < TILE / 32; ++wi) s += red[wi][threadIdx.x];
        partials[(size_t)blockIdx.x * NPART + threadIdx.x] = s;
    }
}

// ----------------------------------------------------------------------------
// The force evaluation split by register footprint.  Only the ~14 angular
// pairs of an atom need its 120 angular accumulators; the ~58 radial terms
// need 9.  So:
//   k_radial_q     all pairs  -> q_n (radial descriptor)            small state
//   k_nep_ang      angular pairs -> A_nlm, network, adjoint, angular and ZBL
//                  pair forces, energy                              large state
//   k_radial_force all pairs  -> radial pair forces from b_k        small state
// All three scatter into the same fixed-point sums (order independent).
// ----------------------------------------------------------------------------

__device__ __forceinline__ int list_slot(int s, int na, int M)
{
    return s < na ? s : M - 1 - (s - na);
}

// With a Verlet skin (act_nbr != nullptr) the kernel also writes this step's
// lists of the pairs within r_c (angular ones from the front, radial-only ones
// from the back, same layout as nbr), so the angular and radial-force kernels
// never branch over pairs beyond the cutoffs.
// MS (several species): basis sums per neighbour species, Sb[t][k] =
// sum_{j of species t} f_c T_k, contracted per atom with the coefficients of
// the pairs (t_i, t) from coef.
template <typename R, bool MS>
__global__ void __launch_bounds__(128) k_radial_q(const Model<R> P, const Grid g,
                                                  const typename V4<R>::T* __restrict__ pos4,
                                                  const int* __restrict__ nbr,
                                                  const int2* __restrict__ cnt,
                                                  R* __restrict__ qr,
                                                  int* __restrict__ act_nbr,
                                                  int2* __restrict__ act_cnt,
                                                  const R* __restrict__ coef,
                                                  const int* __restrict__ perm,
                                                  const double* __restrict__ x64,
                                                  int* __restrict__ status,
                                                  int* __restrict__ tflag = nullptr)
{
    using P4 = typename V4<R>::T;
    constexpr int NTS = MS ? NT_MAX : 1;
    __shared__ P4 s_off[27];
    fill_stencil<R>(s_off, g);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const size_t ld = (size_t)g.ld;
    const int2 c2 = cnt[k];
    const int na = c2.x, total = c2.x + c2.y, M = g.M;
    const P4 pi = pos4[k];
    const int T = MS ? P.ntypes : 1;
    R Sb[NTS][KR];
#pragma unroll
    for (int t = 0; t < NTS; ++t)
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) Sb[t][kk] = R(0);
    int a_na = 0, a_nro = 0;
    bool close = false;
    // two-stage prefetch: entry s + 2 and position s + 1 in flight during pair s
    int ent_n = total > 0 ? nbr[(size_t)list_slot(0, na, M) * ld + k] : 0;
    int ent_nn = total > 1 ? nbr[(size_t)list_slot(1, na, M) * ld + k] : 0;
    P4 pj_n = total > 0 ? pos4[ent_n >> 5] : pi;
    for (int s = 0; s < total; ++s) {
        const int ent = ent_n;
        const P4 pj = pj_n;
        ent_n = ent_nn;
        if (s + 1 < total) pj_n = pos4[ent_n >> 5];
        if (s + 2 < total) ent_nn = nbr[(size_t)list_slot(s + 2, na, M) * ld + k];
        const P4 off = s_off[ent & 31];
        R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
        R r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rcR2) continue;   // beyond r_c (lists built with a skin)
        if (act_nbr) {
            if (r2 < P.rcA2) act_nbr[(size_t)(a_na++) * ld + k] = ent;
            else act_nbr[(size_t)(M - 1 - a_nro++) * ld + k] = ent;
        }
        close |= r2 < P.zbl_r2 * P.zbl_r2;
        close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, ent >> 5, dx, dy, dz, r2);
        const R r = r2 * nepm::nep_rsqrt(r2);
        R Tk[KR], dT[KR], fc, dfc, dxdr;
        nepm::cheb<KR, false>(r, P.inv_rcR, Tk, dT, fc, dfc, dxdr);
        if constexpr (MS) {
            const int tj = (int)pj.w;
#pragma unroll
            for (int t = 0; t < NTS; ++t) {
                if (t < T) {
                    const R wt = tj == t ? fc : R(0);
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) Sb[t][kk] += wt * Tk[kk];
                }
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) Sb[0][kk] += fc * Tk[kk];
        }
    }
    if (act_cnt) act_cnt[k] = make_int2(a_na, a_nro);
    if (tflag) {
        // this tile's kernel choice (blocks of TILE atoms: block = tile)
        const int bits = (close ? TILE_CLOSE : 0) |
                         ((act_cnt ? a_na : na) > TILE_ANG_LIM ? TILE_DENSE : 0);
        if (bits) tile_mark(tflag, (g.n + TILE - 1) / TILE, blockIdx.x, bits);
    }
    R q[NR];
    if constexpr (MS) {
        const int ti = (int)pi.w;
#pragma unroll
        for (int n = 0; n < NR; ++n) q[n] = R(0);
#pragma unroll
        for (int t = 0; t < NTS; ++t) {
            if (t < T) {
                const R* c = coef + (size_t)(ti * T + t) * CSTR + C_RAD;
#pragma unroll
                for (int n = 0; n < NR; ++n) {
                    R acc = c[NR * KR + n] * Sb[t][0];
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) acc += c[n * KR + kk] * Sb[t][kk];
                    q[n] += acc;
                }
            }
        }
    } else {
        radial_q<R>(P, Sb[0], q);
    }
#pragma unroll
    for (int n = 0; n < NR; ++n) qr[(size_t)n * ld + k] = q[n];
}

// Angular part of dU_i/dd_ij for one angular neighbour (no radial term).
// cs: the pair's angular coefficients (h [0, 45), C [45, 50)) with several
// species, nullptr for the model's own (one species).
template <typename R>
__device__ __forceinline__ void force_pair_ang(const Model<R>& P, R r, R inv_r, R ux, R uy, R uz,
                                               const R (&Ab)[NA][NLM], R& fx, R& fy, R& fz,
                                               const R* cs = nullptr)
{
    R T[KA], dT[KA], fc, dfc, dxdr;
    nepm::cheb<KA, true>(r, P.inv_rcA, T, dT, fc, dfc, dxdr);
    R gn[NA], dgn[NA];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        R a = cs ? cs[NA * KA + n] : P.CA[n], b = R(0);
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            const R h = cs ? cs[n * KA + kk] : P.hA[n * KA + kk];
            a += h * T[kk];
            b += h * dT[kk];
        }
        gn[n] = fc * a;
        dgn[n] = dfc * a + fc * dxdr * b;
    }
    R Y[NLM], G[NLM];
    nepm::harmonics(ux, uy, uz, Y);
    R sang = R(0);
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
        const int l = lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4));
        R gsum = R(0), dsum = R(0);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            gsum += Ab[n][lm] * gn[n];
            dsum += Ab[n][lm] * dgn[n];
        }
        G[lm] = gsum;
        sang += (dsum - R(l) * inv_r * gsum) * Y[lm];
    }
    R vx, vy, vz;
    nepm::harmonics_grad_dot(ux, uy, uz, G, vx, vy, vz);
    fx = sang * ux + vx * inv_r;
    fy = sang * uy + vy * inv_r;
    fz = sang * uz + vz * inv_r;
}

// Per-tile energy and virial partials (fixed order); see k_nep.
template <typename R>
__device__ __forceinline__ void tile_partials(double e_site, R (&w)[9], double (&wz)[9],
                                              bool has_zbl, double* __restrict__ out)
{
    __shared__ double red[TILE / 32][NPART];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_site += __shfl_xor_sync(0xffffffffu, e_site, o);
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[t] += __shfl_xor_sync(0xffffffffu, w[t], o);
    if (__any_sync(0xffffffffu, has_zbl)) {
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wz[t] += __shfl_xor_sync(0xffffffffu, wz[t], o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = e_site;
#pragma unroll
        for (int t = 0; t < 9; ++t) red[threadIdx.x >> 5][1 + t] = (double)w[t] + wz[t];
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        double sum = 0.0;
#pragma unroll
        for (int wi = 0; wi < TILE / 32; ++wi) sum += red[wi][threadIdx.x];
        out[threadIdx.x] = sum;
    }
}

// Close pairs in the register kernel (FP32 path).  A warp runs every pair
// slot for all 32 lanes, and FP64 arithmetic runs at a small fraction of the
// FP32 rate on this part, so an FP64 displacement or ZBL term taken inline
// costs the warp a full FP64 sequence in each slot in which any lane has a
// close pair; in a dense clump (~13 of ~100 angular pairs inside 2 A) that is
// nearly every slot.  Instead each atom lists its close pairs (up to CQ; more
// are taken inline) and the warp does their FP64 work with one pair per lane:
//   before the descriptor pass: the FP64 displacement of each listed pair,
//     rounded once to FP32 (as close_pair_fp64), read back in both passes;
//   after the pair-force pass: the ZBL term (Eq. 2-4) of each listed pair
//     inside the outer radius; the lane that evaluates it adds the
//     neighbour's share of the force, the atom's own lane then adds its
//     energy, force and FP64 virial in slot order, so every sum is the one of
//     the inline form, in the same order.
constexpr int CQ = 32;
// dynamic shared memory of the register kernel behind the staged entries:
// the close-pair lists [CQ][TILE] float4, the ZBL results [9][TILE] double
// and the per-warp prefix counts [TILE] int
constexpr size_t CQ_BYTES = sizeof(float4) * CQ * TILE + sizeof(double) * 9 * TILE + sizeof(int) * TILE;

// The per-lane list lengths of the warp's lanes in mask (lanes 0..nact-1:
// the atoms of a tile that exist) as an inclusive prefix in inc[0..nact-1]
// (the warp's own entries); returns the warp's total.
__device__ __forceinline__ int warp_list_prefix(int cnt, int* __restrict__ inc, unsigned mask)
{
    const int lane = threadIdx.x & 31;
    int v = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(mask, v, o);
        if (lane >= o) v += t;
    }
    inc[lane] = v;
    __syncwarp(mask);
    return __shfl_sync(mask, v, 31 - __clz(mask));
}

// The lane owning entry e of the warp's lists (inc as above, nact lanes) and
// the entry's index c within that lane's list.
__device__ __forceinline__ int warp_entry_owner(const int* __restrict__ inc, int nact, int e, int& c)
{
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (inc[mid] > e) hi = mid;
        else lo = mid + 1;
    }
    c = e - (lo > 0 ? inc[lo - 1] : 0);
    return lo;
}

// cd[c * TILE + t] = (dx, dy, dz, slot) of the c-th listed pair of the
// block's atom t: on entry the slot (int bits), on return also the FP64
// displacement rounded to FP32.  Collective over the lanes in mask (see
// warp_list_prefix); nc = this lane's count.
__device__ __forceinline__ void close_refine_warp(const Grid& g, const double* __restrict__ x64,
                                                  const int* __restrict__ perm,
                                                  const int* __restrict__ s_ent, bool staged,
                                                  const int* __restrict__ nbr, size_t ld,
                                                  int tile, float4* __restrict__ cd,
                                                  int* __restrict__ inc, int nc, unsigned mask)
{
    const int total = warp_list_prefix(nc, inc, mask);
    const int lane = threadIdx.x & 31, wb = threadIdx.x & ~31, nact = __popc(mask);
    for (int e = lane; e < total; e += nact) {
        int c;
        const int t = wb + warp_entry_owner(inc, nact, e, c);
        const int ko = tile * TILE + t;
        float4 v = cd[c * TILE + t];
        const int s = __float_as_int(v.w);
        const int ent = staged ? s_ent[s * TILE + t] : nbr[(size_t)s * ld + ko];
        double d[3];
        disp64(g, x64, perm[ko], perm[ent >> 5], d);
        v.x = (float)d[0];
        v.y = (float)d[1];
        v.z = (float)d[2];
        cd[c * TILE + t] = v;
    }
    __syncwarp(mask);
}

// The ZBL terms of the listed pairs: cd[c * TILE + t].w = neighbour m (int
// bits) of the c-th pair of atom t with r < outer radius; zr [9][TILE]
// doubles of scratch.  Collective over the lanes in mask; nz = this lane's
// count; ez, fi, wz, bad, has_zbl are this lane's atom's sums, continued as
// the inline form would.
template <bool MS>
__device__ __forceinline__ void zbl_warp(const Model<float>& P, const Grid& g,
                                         const double* __restrict__ x64,
                                         const int* __restrict__ perm,
                                         const float4* __restrict__ pos4,
                                         long long* __restrict__ facc, size_t ld, int tile,
                                         const float4* __restrict__ cd, double* __restrict__ zr,
                                         int* __restrict__ inc, int nz, unsigned mask,
                                         double& ez, long long (&fi)[3], double (&wz)[9],
                                         bool& bad, bool& has_zbl)
{
    using A_ = Acc<float>;
    const int total = warp_list_prefix(nz, inc, mask);
    const int lane = threadIdx.x & 31, wb = threadIdx.x & ~31, nact = __popc(mask);
    const int start = inc[lane] - nz;
    for (int b0 = 0; b0 < total; b0 += nact) {
        const int e = b0 + lane;
        if (e < total) {
            int c;
            const int t = wb + warp_entry_owner(inc, nact, e, c);
            const int ko = tile * TILE + t;
            const int m = __float_as_int(cd[c * TILE + t].w);
            double d64[3];
            disp64(g, x64, perm[ko], perm[m], d64);
            const double r64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
            double in = 0.0, uh = 0.0, cc = 0.0, f3[3] = {0.0, 0.0, 0.0};
            if (r64 < P.zbl_rr2) {
                double Uz, dUz;
                const int pz = MS ? (int)pos4[ko].w * P.ntypes + (int)pos4[m].w : 0;
                zbl_pair(r64, MS ? P.zbl_kp[pz] : P.zbl_k, MS ? P.zbl_inv_ap[pz] : P.zbl_inv_a,
                         P.zbl_r1, P.zbl_rr2, Uz, dUz);
                in = 1.0;
                uh = 0.5 * Uz;
                cc = 0.5 * dUz / r64;
#pragma unroll
                for (int a = 0; a < 3; ++a) f3[a] = cc * d64[a];
                A_::add(&facc[m], -A_::convd(f3[0]));
                A_::add(&facc[ld + m], -A_::convd(f3[1]));
                A_::add(&facc[2 * ld + m], -A_::convd(f3[2]));
            }
            zr[threadIdx.x] = in;
            zr[TILE + threadIdx.x] = uh;
            zr[2 * TILE + threadIdx.x] = cc;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                zr[(3 + a) * TILE + threadIdx.x] = f3[a];
                zr[(6 + a) * TILE + threadIdx.x] = d64[a];
            }
        }
        __syncwarp(mask);
        // this lane's entries among the batch, in slot order
        const int lo = start > b0 ? start : b0;
        const int hi = start + nz < b0 + nact ? start + nz : b0 + nact;
        for (int e2 = lo; e2 < hi; ++e2) {
            const int q = wb + (e2 - b0);
            if (zr[q] != 0.0) {
                ez += zr[TILE + q];
                const double cc = zr[2 * TILE + q];
                const double f3[3] = {zr[3 * TILE + q], zr[4 * TILE + q], zr[5 * TILE + q]};
                const double d64[3] = {zr[6 * TILE + q], zr[7 * TILE + q], zr[8 * TILE + q]};
                fi[0] += A_::convd(f3[0]);
                fi[1] += A_::convd(f3[1]);
                fi[2] += A_::convd(f3[2]);
                bad |= !isfinite(cc);
                has_zbl = true;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) wz[3 * a + b] -= f3[a] * d64[b];
            }
        }
        __syncwarp(mask);
    }
}

// MS (several species): the coefficient table of all ordered species pairs
// is copied to shared memory ahead of the staged entries; each angular pair
// reads its own block, and the radial adjoint is written once per neighbour
// species (br[(k * T + t) * 3]).
// FP32: the close pairs' FP64 work warp-wide (see CQ) in shared memory
// behind the staged entries.
template <typename R, bool MS>
__global__ void __launch_bounds__(TILE) k_nep_ang(const Model<R> P, const Grid g,
                                                  const typename V4<R>::T* __restrict__ pos4,
                                                  const int* __restrict__ nbr,
                                                  const int2* __restrict__ cnt,
                                                  const int* __restrict__ perm,
                                                  const double* __restrict__ x64,
                                                  const R* __restrict__ qr,
                                                  typename V4<R>::T* __restrict__ br,
                                                  typename Acc<R>::T* __restrict__ facc,
                                                  double* __restrict__ partials,
                                                  double* __restrict__ site_energy,
                                                  int* __restrict__ status, int stage_slots,
                                                  const R* __restrict__ coef,
                                                  const int* __restrict__ tflag = nullptr,
                                                  int* __restrict__ ntiles_done = nullptr,
                                                  int tmask = 0)
{
    // with tflag: this launch takes only the tiles with a bit of tmask in their
    // flag (k_nep_ang_tm takes the others) and counts them
    using A_ = Acc<R>;
    using P4 = typename V4<R>::T;
    __shared__ P4 s_off[27];
    __shared__ int s_max;
    // dynamic: [T * T * CSTR] coefficients (MS only), then [stage_slots][TILE]
    // angular entries, then (FP32) the close-pair lists (see CQ)
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int T = MS ? P.ntypes : 1;
    R* s_coef = reinterpret_cast<R*>(s_dyn);
    int* s_ent = reinterpret_cast<int*>(s_dyn + (MS ? sizeof(R) * T * T * CSTR : 0));
    constexpr bool CW = sizeof(R) == 4;   // close pairs warp-wide
    float4* s_cd = reinterpret_cast<float4*>(s_ent + (size_t)stage_slots * TILE);
    double* s_zr = reinterpret_cast<double*>(s_cd + CQ * TILE);
    int* s_inc = reinterpret_cast<int*>(s_zr + 9 * TILE) + (threadIdx.x & ~31);
    if constexpr (MS) {
        for (int t = threadIdx.x; t < T * T * CSTR; t += TILE) s_coef[t] = coef[t];
    }
    __shared__ __align__(16) R s_w[H * WROW];
    fill_network_rows<R>(s_w, P);
    fill_stencil<R>(s_off, g);
    // one tile of TILE cell-ordered atoms per iteration (one iteration per
    // block unless the launch uses fewer blocks than tiles)
    const int ntiles = (g.n + TILE - 1) / TILE;
    // with tflag: the listed tiles (see tile_mark)
    const int nlist = tflag ? tflag[ntiles] : ntiles;
    for (int it = blockIdx.x; it < nlist; it += gridDim.x) {
    const int tile = tflag ? tflag[ntiles + 1 + it] : it;
    if (tflag) {
        if (!(tflag[tile] & tmask)) continue;   // the whole block: the flag is the tile's
        if (threadIdx.x == 0) atomicAdd(ntiles_done, 1);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int k = tile * TILE + threadIdx.x;
    const size_t ld = (size_t)g.ld;
    const int na = k < g.n ? cnt[k].x : 0;
    atomicMax(&s_max, na);
    __syncthreads();
    const bool staged = s_max <= stage_slots;
    if (staged)
        for (int s = 0; s < na; ++s) s_ent[s * TILE + threadIdx.x] = nbr[(size_t)s * ld + k];
    double e_site = 0.0;
    R w[9];
    double wz[9];
    bool has_zbl = false;
#pragma unroll
    for (int t = 0; t < 9; ++t) { w[t] = R(0); wz[t] = 0.0; }
    const unsigned vmask = __ballot_sync(0xffffffffu, k < g.n);   // a prefix of the warp

    if (k < g.n) {
        const P4 pi = pos4[k];
        const int ti = MS ? (int)pi.w : 0;
        auto entry = [&](int s) -> int {
            return staged ? s_ent[s * TILE + threadIdx.x] : nbr[(size_t)s * ld + k];
        };
        // FP32: the slots of this atom's close pairs (r^2 below the squared
        // outer ZBL radius, in the passes' own FP32 form), the first CQ listed
        // with their FP64 displacements (warp-wide, see CQ); from slot s_inl
        // on (more than CQ) the passes refine close pairs inline
        int ncq = 0, s_inl = 0x7fffffff;
        if constexpr (CW) {
            int nc = 0;
            int ent_c = na > 0 ? entry(0) : 0;
            P4 pj_c = na > 0 ? pos4[ent_c >> 5] : pi;
            for (int s = 0; s < na; ++s) {
                const int ent = ent_c;
                const P4 pj = pj_c;
                if (s + 1 < na) {
                    ent_c = entry(s + 1);
                    pj_c = pos4[ent_c >> 5];
                }
                const P4 off = s_off[ent & 31];
                const R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
                const R r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < P.zbl_r2 * P.zbl_r2) {
                    if (nc < CQ) s_cd[nc * TILE + threadIdx.x] = make_float4(0.f, 0.f, 0.f, __int_as_float(s));
                    else if (nc == CQ) s_inl = s;
                    ++nc;
                }
            }
            ncq = nc < CQ ? nc : CQ;
            close_refine_warp(g, x64, perm, s_ent, staged, nbr, ld, tile, s_cd, s_inc, ncq, vmask);
        }
        // the next listed close pair (its slot; -1: none left)
        int ci = 0;
        auto listed_slot = [&](int c) -> int {
            return c < ncq ? __float_as_int(s_cd[c * TILE + threadIdx.x].w) : -1;
        };
        int next_s = CW ? listed_slot(0) : -1;
        R A[NA][NLM];
#pragma unroll
        for (int n = 0; n < NA; ++n)
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) A[n][lm] = R(0);
        int ent_n = na > 0 ? entry(0) : 0;
        P4 pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
        for (int s = 0; s < na; ++s) {
            const int ent = ent_n;
            const P4 pj = pj_n;
            if (s + 1 < na) {
                ent_n = entry(s + 1);
                pj_n = pos4[ent_n >> 5];
            }
            const P4 off = s_off[ent & 31];
            R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            bool listed = false;
            if (CW && s == next_s) {
                const float4 v = s_cd[ci * TILE + threadIdx.x];
                dx = v.x; dy = v.y; dz = v.z;
                r2 = dx * dx + dy * dy + dz * dz;
                listed = true;
                next_s = listed_slot(++ci);
            }
            if (r2 >= P.rcA2) continue;   // beyond r_c^A (lists built with a skin)
            if (!CW || (!listed && s >= s_inl))
                close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, ent >> 5, dx, dy, dz, r2);
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            R Tk[KA], dT[KA], fc, dfc, dxdr;
            nepm::cheb<KA, false>(r, P.inv_rcA, Tk, dT, fc, dfc, dxdr);
            R Y[NLM];
            nepm::harmonics(dx * inv_r, dy * inv_r, dz * inv_r, Y);
            const R* cs = MS ? s_coef + ((size_t)ti * T + (int)pj.w) * CSTR + C_ANG : nullptr;
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                R acc = MS ? cs[NA * KA + n] : P.CA[n];
#pragma unroll
                for (int kk = 0; kk < KA; ++kk) acc += (MS ? cs[n * KA + kk] : P.hA[n * KA + kk]) * Tk[kk];
                const R gn = fc * acc;
#pragma unroll
                for (int lm = 0; lm < NLM; ++lm) A[n][lm] += gn * Y[lm];
            }
        }
        R qR[NR];
#pragma unroll
        for (int n = 0; n < NR; ++n) qR[n] = qr[(size_t)n * ld + k];
        R U;
        auto store_b = [&](const R (&bR)[KR], R B0, size_t slot) {
            P4 b0v, b1v, b2v;
            b0v.x = bR[0]; b0v.y = bR[1]; b0v.z = bR[2]; b0v.w = bR[3];
            b1v.x = bR[4]; b1v.y = bR[5]; b1v.z = bR[6]; b1v.w = bR[7];
            b2v.x = bR[8]; b2v.y = B0; b2v.z = R(0); b2v.w = R(0);
            br[3 * slot] = b0v;
            br[3 * slot + 1] = b1v;
            br[3 * slot + 2] = b2v;
        };
        if constexpr (MS) {
            R aR[NR];
            U = network_adjoint_core_rolled<R>(P, s_w, qR, A, aR);
            for (int t = 0; t < T; ++t) {
                const R* c = s_coef + ((size_t)ti * T + t) * CSTR + C_RAD;
                R bR[KR], B0 = R(0);
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) bR[kk] = R(0);
#pragma unroll
                for (int nu = 0; nu < NR; ++nu) {
                    B0 += aR[nu] * c[NR * KR + nu];
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) bR[kk] += aR[nu] * c[nu * KR + kk];
                }
                store_b(bR, B0, (size_t)k * T + t);
            }
        } else {
            // one species: the record the radial-force kernel gathers per
            // neighbour, (x, y, z, b_8), (b_0 + B0, b_1, b_2, b_3), (b_4..b_7)
            // (T_0 = 1 and T_0' = 0, so B0 folds into b_0)
            R bR[KR], B0 = R(0);
            {
                R aR[NR];
                U = network_adjoint_core_rolled<R>(P, s_w, qR, A, aR);
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) bR[kk] = R(0);
#pragma unroll
                for (int nu = 0; nu < NR; ++nu) {
                    B0 += aR[nu] * P.CR[nu];
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) bR[kk] += aR[nu] * P.hR[nu * KR + kk];
                }
            }
            P4 r0, r1, r2;
            r0.x = pi.x; r0.y = pi.y; r0.z = pi.z; r0.w = bR[8];
            r1.x = bR[0] + B0; r1.y = bR[1]; r1.z = bR[2]; r1.w = bR[3];
            r2.x = bR[4]; r2.y = bR[5]; r2.z = bR[6]; r2.w = bR[7];
            br[3 * (size_t)k] = r0;
            br[3 * (size_t)k + 1] = r1;
            br[3 * (size_t)k + 2] = r2;
        }

        typename A_::T fi[3] = {0, 0, 0};
        double ez = 0.0;
        bool bad = !isfinite(U);
        const int i_caller = perm[k];
        ent_n = na > 0 ? entry(0) : 0;
        pj_n = na > 0 ? pos4[ent_n >> 5] : pi;
        // listed close pairs again in slot order; those with a ZBL term are
        // queued in the consumed list entries (nz <= ci) for zbl_warp
        ci = 0;
        next_s = CW ? listed_slot(0) : -1;
        int nz = 0;
        for (int s = 0; s < na; ++s) {
            const int ent = ent_n;
            const P4 pj = pj_n;
            if (s + 1 < na) {
                ent_n = entry(s + 1);
                pj_n = pos4[ent_n >> 5];
            }
            const int m = ent >> 5;
            const P4 off = s_off[ent & 31];
            R dx = pj.x - pi.x + off.x, dy = pj.y - pi.y + off.y, dz = pj.z - pi.z + off.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            bool listed = false;
            if (CW && s == next_s) {
                const float4 v = s_cd[ci * TILE + threadIdx.x];
                dx = v.x; dy = v.y; dz = v.z;
                r2 = dx * dx + dy * dy + dz * dz;
                listed = true;
                next_s = listed_slot(++ci);
            }
            if (r2 >= P.rcA2) continue;
            // close pair (FP32 path) not listed: the FP64 displacement, formed
            // once for the NEP terms (rounded, see close_pair_fp64) and the ZBL
            // term
            double d64[3];
            const bool close = sizeof(R) == 4 && !listed && (!CW || s >= s_inl) &&
                               r2 < P.zbl_r2 * P.zbl_r2;
            if (close) {
                disp64(g, x64, i_caller, perm[m], d64);
                dx = (R)d64[0];
                dy = (R)d64[1];
                dz = (R)d64[2];
                r2 = dx * dx + dy * dy + dz * dz;
            }
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            R fx, fy, fz;
            force_pair_ang<R>(P, r, inv_r, dx * inv_r, dy * inv_r, dz * inv_r, A, fx, fy, fz,
                              MS ? s_coef + ((size_t)ti * T + (int)pj.w) * CSTR + C_ANG
                                 : nullptr);
            bad |= !isfinite(fx + fy + fz);
            typename A_::T cx = A_::conv(fx), cy = A_::conv(fy), cz = A_::conv(fz);
            if (CW && listed && r < P.zbl_r2) {
                s_cd[nz * TILE + threadIdx.x].w = __int_as_float(m);
                ++nz;
            } else if (r < P.zbl_r2) {
                if (sizeof(R) == 4) {
                    if (!close) disp64(g, x64, i_caller, perm[m], d64);
                } else {
                    d64[0] = (double)dx; d64[1] = (double)dy; d64[2] = (double)dz;
                }
                const double r64 = sqrt(d64[0] * d64[0] + d64[1] * d64[1] + d64[2] * d64[2]);
                if (r64 < P.zbl_rr2) {
                    double Uz, dUz;
                    const int pz = MS ? ti * T + (int)pj.w : 0;
                    zbl_pair(r64, MS ? P.zbl_kp[pz] : P.zbl_k, MS ? P.zbl_inv_ap[pz] : P.zbl_inv_a,
                             P.zbl_r1, P.zbl_rr2, Uz, dUz);
                    ez += 0.5 * Uz;
                    const double c = 0.5 * dUz / r64;
                    const double f3[3] = {c * d64[0], c * d64[1], c * d64[2]};
                    cx += A_::convd(f3[0]);
                    cy += A_::convd(f3[1]);
                    cz += A_::convd(f3[2]);
                    bad |= !isfinite(c);
                    has_zbl = true;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) wz[3 * a + b] -= f3[a] * d64[b];
                }
            }
            fi[0] += cx; fi[1] += cy; fi[2] += cz;
            A_::add(&facc[m], -cx);
            A_::add(&facc[ld + m], -cy);
            A_::add(&facc[2 * ld + m], -cz);
            w[0] -= fx * dx; w[1] -= fx * dy; w[2] -= fx * dz;
            w[3] -= fy * dx; w[4] -= fy * dy; w[5] -= fy * dz;
            w[6] -= fz * dx; w[7] -= fz * dy; w[8] -= fz * dz;
        }
        if constexpr (CW)
            zbl_warp<MS>(P, g, x64, perm, pos4, facc, ld, tile, s_cd, s_zr, s_inc, nz, vmask, ez,
                         fi, wz, bad, has_zbl);
        A_::add(&facc[k], fi[0]);
        A_::add(&facc[ld + k], fi[1]);
        A_::add(&facc[2 * ld + k], fi[2]);
        e_site = (double)U + ez;
        if (site_energy) site_energy[i_caller] = e_site;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    tile_partials<R>(e_site, w, wz, has_zbl, partials + (size_t)tile * NPART);
    __syncthreads();   // the staged entries and shared sums are reused by the next tile
    }
}

// Radial pair forces by gathering: with the radial adjoint of both atoms,
//   f_ij - f_ji = [f_c' (B0_i + B0_j + sum_k (b_i + b_j)_k T_k)
//                  + f_c x' sum_k (b_i + b_j)_k T'_k] u_ij,
// so each atom sums its own radial force from its neighbours' packed adjoint
// without atomics; the virial is -1/2 sum_i sum_j (f_ij - f_ji) (x) d_ij.
// One species: bp[3k..3k+2] = (x, y, z, b_8), (b_0 + B0, b_1..b_3), (b_4..b_7)
// (position and adjoint in one gathered record); several species: pos4 and
// bp[(k T + t) * 3] = (b_0..b_3), (b_4..b_7), (b_8, B0, 0, 0).
// MS (several species): the pair (i, j) adds atom i's adjoint for neighbour
// species t_j and atom j's for species t_i (bp[(k * T + t) * 3]).
template <typename R, bool MS, bool CLOSE = true>
__global__ void __launch_bounds__(TILE, sizeof(R) == 4 && !MS ? 7 : 1) k_radial_force(const Model<R> P, const Grid g,
                                                       const typename V4<R>::T* __restrict__ pos4,
                                                       const int* __restrict__ nbr,
                                                       const int2* __restrict__ cnt,
                                                       const typename V4<R>::T* __restrict__ bp,
                                                       typename Acc<R>::T* __restrict__ facc,
                                                       double* __restrict__ partials,
                                                       int* __restrict__ status,
                                                       const int* __restrict__ perm,
                                                       const double* __restrict__ x64,
                                                       const int* __restrict__ tflag = nullptr)
{
    using A_ = Acc<R>;
    using P4 = typename V4<R>::T;
    // with tflag (FP32, one species): both instantiations are launched, the
    // one without the close-pair branch takes the tiles without TILE_CLOSE
    __shared__ StencilSplit<R> s_off;
    fill_stencil_split<R>(s_off, g);
    // FP32, several species: the atom's own adjoints in shared memory (a
    // gathered 16-byte load per neighbour each otherwise)
    constexpr bool OWN = MS && sizeof(R) == 4;
    __shared__ P4 s_own[OWN ? NT_MAX * 3 * TILE : 1];
    // one tile of TILE cell-ordered atoms per iteration (one iteration per
    // block unless the launch uses fewer blocks than tiles)
    const int ntiles = (g.n + TILE - 1) / TILE;
    // with tflag, the close-pair variant takes the listed tiles (see tile_mark)
    const bool listed = tflag && CLOSE;
    const int nlist = listed ? tflag[ntiles] : ntiles;
    for (int it = blockIdx.x; it < nlist; it += gridDim.x) {
    const int tile = listed ? tflag[ntiles + 1 + it] : it;
    if (tflag && (((tflag[tile] & TILE_CLOSE) != 0) != CLOSE)) continue;   // whole block
    const int k = tile * TILE + threadIdx.x;
    const size_t ld = (size_t)g.ld;
    R w[9];
    double wz[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) { w[t] = R(0); wz[t] = 0.0; }
    if (!MS && k < g.n) {
        // one species: three 16-byte loads per neighbour (position and adjoint
        // in one record written by the angular kernel)
        const int2 c2 = cnt[k];
        const int na = c2.x, total = c2.x + c2.y, M = g.M;
        // the record of atom m (see rec_store)
        auto record = [&](size_t m, P4& r0, P4& r1, P4& r2) {
            r0 = bp[3 * m]; r1 = bp[3 * m + 1]; r2 = bp[3 * m + 2];
        };
        P4 ri0, ri1, ri2;
        record((size_t)k, ri0, ri1, ri2);
        R fx = R(0), fy = R(0), fz = R(0);
        int ent_n = total > 0 ? nbr[(size_t)list_slot(0, na, M) * ld + k] : 0;
        int ent_nn = total > 1 ? nbr[(size_t)list_slot(1, na, M) * ld + k] : 0;
        P4 rj0_n = ri0, rj1_n = ri1, rj2_n = ri2;
        if (total > 0) record((size_t)(ent_n >> 5), rj0_n, rj1_n, rj2_n);
        for (int s = 0; s < total; ++s) {
            const int ent = ent_n;
            const P4 rj0 = rj0_n, rj1 = rj1_n, rj2 = rj2_n;
            ent_n = ent_nn;
            if (s + 1 < total) record((size_t)(ent_n >> 5), rj0_n, rj1_n, rj2_n);
            if (s + 2 < total) ent_nn = nbr[(size_t)list_slot(s + 2, na, M) * ld + k];
            const int code = ent & 31;
            R dx = rj0.x - ri0.x + s_off.x[code], dy = rj0.y - ri0.y + s_off.y[code],
              dz = rj0.z - ri0.z + s_off.z[code];
            R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= P.rcR2) continue;   // beyond r_c (lists built with a skin)
            if constexpr (CLOSE)
                close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, ent >> 5, dx, dy, dz, r2);
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            R T[KR], dT[KR], fc, dfc, dxdr;
            nepm::cheb<KR, true>(r, P.inv_rcR, T, dT, fc, dfc, dxdr);
            R s1, s2;
            if constexpr (sizeof(R) == 4) {
                // packed pairs of adjacent k: (b_k, b_k+1) (T_k, T_k+1) and
                // (b_k, b_k+1) (T'_k, T'_k+1), with T_0 = 1, T'_0 = 0, T'_1 = 1
                const float2 b01 = __fadd2_rn(make_float2(ri1.x, ri1.y), make_float2(rj1.x, rj1.y));
                const float2 b23 = __fadd2_rn(make_float2(ri1.z, ri1.w), make_float2(rj1.z, rj1.w));
                const float2 b45 = __fadd2_rn(make_float2(ri2.x, ri2.y), make_float2(rj2.x, rj2.y));
                const float2 b67 = __fadd2_rn(make_float2(ri2.z, ri2.w), make_float2(rj2.z, rj2.w));
                const float b8 = ri0.w + rj0.w;
                float2 a1 = __fmul2_rn(b01, make_float2(1.f, T[1]));
                a1 = __ffma2_rn(b23, make_float2(T[2], T[3]), a1);
                a1 = __ffma2_rn(b45, make_float2(T[4], T[5]), a1);
                a1 = __ffma2_rn(b67, make_float2(T[6], T[7]), a1);
                float2 a2 = make_float2(0.f, b01.y);
                a2 = __ffma2_rn(b23, make_float2(dT[2], dT[3]), a2);
                a2 = __ffma2_rn(b45, make_float2(dT[4], dT[5]), a2);
                a2 = __ffma2_rn(b67, make_float2(dT[6], dT[7]), a2);
                s1 = (a1.x + a1.y) + b8 * T[8];
                s2 = (a2.x + a2.y) + b8 * dT[8];
            } else {
                const R b[KR] = {ri1.x + rj1.x, ri1.y + rj1.y, ri1.z + rj1.z, ri1.w + rj1.w,
                                 ri2.x + rj2.x, ri2.y + rj2.y, ri2.z + rj2.z, ri2.w + rj2.w,
                                 ri0.w + rj0.w};
                s1 = b[0];
                s2 = R(0);
#pragma unroll
                for (int kk = 1; kk < KR; ++kk) {
                    s1 += b[kk] * T[kk];
                    s2 += b[kk] * dT[kk];
                }
            }
            const R fs = (dfc * s1 + fc * dxdr * s2) * inv_r;   // (f_ij - f_ji) = fs d
            const R gx = fs * dx, gy = fs * dy, gz = fs * dz;
            fx += gx; fy += gy; fz += gz;
            // fs d (x) d is symmetric: six products (expanded after the loop)
            w[0] -= gx * dx; w[4] -= gy * dy; w[8] -= gz * dz;
            w[1] -= gx * dy; w[2] -= gx * dz; w[5] -= gy * dz;
        }
        w[3] = w[1]; w[6] = w[2]; w[7] = w[5];
        if (!isfinite(fx + fy + fz)) atomicOr(status, ST_NONFINITE);
        A_::add(&facc[k], A_::conv(fx));
        A_::add(&facc[ld + k], A_::conv(fy));
        A_::add(&facc[2 * ld + k], A_::conv(fz));
#pragma unroll
        for (int t = 0; t < 9; ++t) w[t] *= R(0.5);
    }
    if (MS && k < g.n) {
        const int2 c2 = cnt[k];
        const int na = c2.x, total = c2.x + c2.y, M = g.M;
        const P4 pi = pos4[k];
        const int T = MS ? P.ntypes : 1;
        const int ti = MS ? (int)pi.w : 0;
        P4 bi0 = bp[3 * (size_t)k], bi1 = bp[3 * (size_t)k + 1], bi2 = bp[3 * (size_t)k + 2];
        if constexpr (OWN) {
            // this atom's adjoints for every neighbour species, in this thread's
            // column of shared memory (read by this thread only)
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int p = 0; p < 3; ++p)
                    s_own[(t * 3 + p) * TILE + threadIdx.x] = bp[3 * ((size_t)k * T + t) + p];
        }
        R fx = R(0), fy = R(0), fz = R(0);
        // two-stage prefetch: entry s + 2, position and adjoint s + 1 in flight
        int ent_n = total > 0 ? nbr[(size_t)list_slot(0, na, M) * ld + k] : 0;
        int ent_nn = total > 1 ? nbr[(size_t)list_slot(1, na, M) * ld + k] : 0;
        P4 pj_n = pi, bj0_n = bi0, bj1_n = bi1, bj2_n = bi2;
        if (total > 0) {
            const size_t m0 = (size_t)(ent_n >> 5) * T + ti;
            pj_n = pos4[ent_n >> 5];
            bj0_n = bp[3 * m0]; bj1_n = bp[3 * m0 + 1]; bj2_n = bp[3 * m0 + 2];
        }
        for (int s = 0; s < total; ++s) {
            const int ent = ent_n;
            const P4 pj = pj_n, bj0 = bj0_n, bj1 = bj1_n, bj2 = bj2_n;
            ent_n = ent_nn;
            if (s + 1 < total) {
                const size_t m1 = (size_t)(ent_n >> 5) * T + ti;
                pj_n = pos4[ent_n >> 5];
                bj0_n = bp[3 * m1]; bj1_n = bp[3 * m1 + 1]; bj2_n = bp[3 * m1 + 2];
            }
            if constexpr (OWN) {
                // this atom's adjoint for the neighbour's species
                const int o = (int)pj.w * 3 * TILE + threadIdx.x;
                bi0 = s_own[o]; bi1 = s_own[o + TILE]; bi2 = s_own[o + 2 * TILE];
            } else if constexpr (MS) {
                // this atom's adjoint for the neighbour's species (L1-resident)
                const size_t mi = (size_t)k * T + (int)pj.w;
                bi0 = bp[3 * mi]; bi1 = bp[3 * mi + 1]; bi2 = bp[3 * mi + 2];
            }
            if (s + 2 < total) ent_nn = nbr[(size_t)list_slot(s + 2, na, M) * ld + k];
            const int code = ent & 31;
            R dx = pj.x - pi.x + s_off.x[code], dy = pj.y - pi.y + s_off.y[code],
              dz = pj.z - pi.z + s_off.z[code];
            R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= P.rcR2) continue;   // beyond r_c (lists built with a skin)
            close_pair_fp64<R>(P.zbl_r2 * P.zbl_r2, g, x64, perm, k, ent >> 5, dx, dy, dz, r2);
            const R inv_r = nepm::nep_rsqrt(r2);
            const R r = r2 * inv_r;
            R T[KR], dT[KR], fc, dfc, dxdr;
            nepm::cheb<KR, true>(r, P.inv_rcR, T, dT, fc, dfc, dxdr);
            const R b[KR] = {bi0.x + bj0.x, bi0.y + bj0.y, bi0.z + bj0.z, bi0.w + bj0.w,
                             bi1.x + bj1.x, bi1.y + bj1.y, bi1.z + bj1.z, bi1.w + bj1.w,
                             bi2.x + bj2.x};
            R s1 = bi2.y + bj2.y, s2 = R(0);
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) {
                s1 += b[kk] * T[kk];
                s2 += b[kk] * dT[kk];
            }
            const R fs = (dfc * s1 + fc * dxdr * s2) * inv_r;   // (f_ij - f_ji) = fs d
            const R gx = fs * dx, gy = fs * dy, gz = fs * dz;
            fx += gx; fy += gy; fz += gz;
            w[0] -= gx * dx; w[1] -= gx * dy; w[2] -= gx * dz;
            w[3] -= gy * dx; w[4] -= gy * dy; w[5] -= gy * dz;
            w[6] -= gz * dx; w[7] -= gz * dy; w[8] -= gz * dz;
        }
        if (!isfinite(fx + fy + fz)) atomicOr(status, ST_NONFINITE);
        A_::add(&facc[k], A_::conv(fx));
        A_::add(&facc[ld + k], A_::conv(fy));
        A_::add(&facc[2 * ld + k], A_::conv(fz));
#pragma unroll
        for (int t = 0; t < 9; ++t) w[t] *= R(0.5);
    }
    tile_partials<R>(0.0, w, wz, false, partials + (size_t)tile * NPART);
    __syncthreads();   // tile_partials' shared sums are reused by the next tile
    }
}

// Forces back to caller order (FP64), one thread per caller index: the
// writes are coalesced and the reads gathered through invperm (caller index
// -> cell-ordered slot).  The accumulators are cleared before the next
// evaluation by a memset.
template <typename R>
__global__ void k_forces_gather(int n, int ld, const int* __restrict__ invperm,
                                const typename Acc<R>::T* __restrict__ facc,
                                double* __restrict__ F, int* __restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = invperm[i];
    if constexpr (sizeof(R) == 4) {
        // fixed point (2^-32 eV/A) -> double: convert the integer, then take
        // 32 from the exponent (exact: a nonzero int64 is at least 1 in
        // magnitude); integer sums are always finite
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long q = facc[(size_t)a * ld + k];
            long long b = __double_as_longlong(__ll2double_rn(q));
            if (q != 0) b -= 32LL << 52;
            F[(size_t)a * n + i] = __longlong_as_double(b);
        }
    } else {
        bool bad = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double f = Acc<R>::value(facc[(size_t)a * ld + k]);
            bad |= !isfinite(f);
            F[(size_t)a * n + i] = f;
        }
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

// Forces back to caller order (FP64), accumulators reset to zero.
template <typename R>
__global__ void k_forces_out(int n, int ld, const int* __restrict__ perm,
                             typename Acc<R>::T* __restrict__ facc, double* __restrict__ F,
                             int* __restrict__ status)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm[k];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = Acc<R>::value(facc[(size_t)a * ld + k]);
        facc[(size_t)a * ld + k] = 0;
        bad |= !isfinite(f);
        F[(size_t)a * n + i] = f;
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

// Stage 1 of the energy/virial sum: block b adds the tiles
// [b * chunk, (b + 1) * chunk) in a fixed order; out[b * NPART + c].
constexpr int RED1_MAX = 512;
static __global__ void __launch_bounds__(256) k_reduce_stage1(const double* __restrict__ partials,
                                                       int ntiles, int chunk,
                                                       double* __restrict__ out)
{
    __shared__ double sh[256];
    const int t0 = blockIdx.x * chunk;
    const int t1 = min(ntiles, t0 + chunk);
    for (int c = 0; c < NPART; ++c) {
        double s = 0.0;
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) s += partials[(size_t)t * NPART + c];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(size_t)blockIdx.x * NPART + c] = sh[0];
        __syncthreads();
    }
}

// One block: sums the per-tile partials in a fixed order into out[0..NPART).
static __global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partials,
                                                         int ntiles, double* __restrict__ out)
{
    __shared__ double sh[256];
    for (int c = 0; c < NPART; ++c) {
        double s = 0.0;
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s += partials[(size_t)t * NPART + c];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sh[0];
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Velocity Verlet (Sec. II.B), FP64
// ----------------------------------------------------------------------------

// thermo layout (device doubles): [0] dt of the current step, [1] time,
// [2] step count, [3] KE, [4] vmax, [5] dt_max, [6] d_max, [7] last dt,
// [8..10] sum_i m_i v_ia^2 (eV) for a = x, y, z, [11] thermostat scale of the
// last chain sweep, [12] thermostat energy, [13..15] barostat scale mu_a
// [16..19] half kick dt/2 acc_t of each species for the current dt
constexpr int TH_DT = 0, TH_TIME = 1, TH_STEP = 2, TH_KE = 3, TH_VMAX = 4, TH_DTMAX = 5,
              TH_DMAX = 6, TH_DTLAST = 7, TH_KXX = 8, TH_NHC_S = 11, TH_ENHC = 12,
              TH_MU = 13, TH_HKICK = 16, TH_N = 20;
// per-block partials of k_kick_thermo: sum m v^2, max |v|^2, sum m v_x^2, v_y^2, v_z^2
constexpr int KT_PART = 5;

// Masses of the species: m[t] (amu) and acc[t] = (1 eV/amu in A^2/fs^2) / m[t].
struct MassTab {
    int ntypes;
    double m[NT_MAX];
    double acc[NT_MAX];
};

__device__ __forceinline__ int species_of(const MassTab& mt, const int32_t* types, int i)
{
    if (mt.ntypes == 1) return 0;
    const int t = types[i];
    return t < 0 ? 0 : (t >= mt.ntypes ? mt.ntypes - 1 : t);   // flagged by k_cell_finalize
}

// v += dt/2 F/m ; x += dt v ; wrap periodic coordinates into [0, L).  The
// half kick dt/2 acc_t comes from thermo (k_thermo_step); the wrap is skipped
// by an integer range test when the coordinate is already inside the box.
static __global__ void k_kick_drift(Grid g, MassTab mt, const int32_t* __restrict__ types,
                             const double* __restrict__ thermo,
                             double* __restrict__ x, double* __restrict__ v,
                             const double* __restrict__ F)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const double dt = thermo[TH_DT];
    const double hk = thermo[TH_HKICK + species_of(mt, types, i)];
    double xn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        size_t o = (size_t)a * g.n + i;
        double vv = v[o] + hk * F[o];
        double xx = x[o] + dt * vv;
        if (!g.tric && g.pbc[a] && !in_box_bits(xx, g.L[a])) xx = wrap_slow(xx, g.L[a], g.invL[a]);
        v[o] = vv;
        xn[a] = xx;
    }
    if (g.tric) {
        // x -= sum_a floor(s_a) h_a over periodic a
        double f[3];
        to_frac(g, xn, f);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!g.pbc[a]) continue;
            const double k = floor(f[a]);
            if (k != 0.0)
#pragma unroll
                for (int b = 0; b < 3; ++b) xn[b] -= k * g.h[3 * a + b];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) x[(size_t)a * g.n + i] = xn[a];
}

// v += dt/2 F/m and per-block (sum m v^2, max |v|^2, and with `tensor` the
// per-dimension sums m v_a^2 the barostat needs; zeros otherwise).  The half
// kick comes from thermo; max |v|^2 is reduced on the bit patterns of the
// (non-negative) doubles.  LOWSUM (FP32 path): sum m v^2 over a warp in FP32
// (the per-warp sums and everything after them in FP64).  HALF: apply the
// half kick; TENSOR: the per-dimension sums (compile-time, so that no FP64
// work of an unused branch issues).
template <bool LOWSUM, bool HALF, bool TENSOR>
__global__ void __launch_bounds__(256) k_kick_thermo(int n, MassTab mt,
                                                     const int32_t* __restrict__ types,
                                                     const double* __restrict__ thermo,
                                                     double* __restrict__ v,
                                                     const double* __restrict__ F,
                                                     double* __restrict__ part)
{
    constexpr bool half_kick = HALF, tensor = TENSOR;
    double v2 = 0.0, va[3] = {0.0, 0.0, 0.0};
    long long vmb = 0;   // bit pattern of max |v|^2
    // grid-stride over the atoms (the grid is a few blocks per SM, so that
    // k_thermo_step reduces a few hundred partials, not one per 256 atoms);
    // each thread's atoms are summed in a fixed order
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = species_of(mt, types, i);
        double vm = 0.0, vv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            size_t o = (size_t)a * n + i;
            vv[a] = v[o];
            if constexpr (half_kick) {
                vv[a] += thermo[TH_HKICK + t] * F[o];
                v[o] = vv[a];
            }
            vm += vv[a] * vv[a];
        }
        v2 += mt.m[t] * vm;
        const long long b = __double_as_longlong(vm);
        vmb = b > vmb ? b : vmb;
        if constexpr (tensor)
#pragma unroll
            for (int a = 0; a < 3; ++a) va[a] += mt.m[t] * vv[a] * vv[a];
    }
    __shared__ double sh[KT_PART][8];
    if constexpr (LOWSUM) {
        float v2f = (float)v2;
        for (int o = 16; o > 0; o >>= 1) v2f += __shfl_xor_sync(0xffffffffu, v2f, o);
        v2 = (double)v2f;
    } else {
        for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long u = __shfl_xor_sync(0xffffffffu, vmb, o);
        vmb = u > vmb ? u : vmb;
    }
    if constexpr (tensor) {
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) va[a] += __shfl_xor_sync(0xffffffffu, va[a], o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = v2;
        sh[1][threadIdx.x >> 5] = __longlong_as_double(vmb);
        for (int a = 0; a < 3; ++a) sh[2 + a][threadIdx.x >> 5] = tensor ? va[a] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[KT_PART] = {0.0, 0.0, 0.0, 0.0, 0.0};
        long long mb = 0;
        for (int w = 0; w < 8; ++w) {
            r[0] += sh[0][w];
            const long long u = __double_as_longlong(sh[1][w]);
            mb = u > mb ? u : mb;
            if constexpr (tensor)
                for (int a = 0; a < 3; ++a) r[2 + a] += sh[2 + a][w];
        }
        r[1] = __longlong_as_double(mb);
        for (int c = 0; c < KT_PART; ++c) part[KT_PART * blockIdx.x + c] = r[c];
    }
}

// One block: KE, max|v|, time bookkeeping and the next step's dt
// (dt = min(dt_max, d_max / max|v|) when d_max > 0).
static __global__ void __launch_bounds__(256) k_thermo_step(const double* __restrict__ part, int nb,
                                                     double ev_amu,
                                                     double* __restrict__ thermo,
                                                     int advance, MassTab mt,
                                                     int* __restrict__ gate = nullptr)
{
    if (gate && threadIdx.x == 0) *gate = 0;   // lists are current after this step
    __shared__ double sa[256], sb[256], sk[3][256];
    double a = 0.0, b = 0.0, k3[3] = {0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        a += part[KT_PART * t];
        b = fmax(b, part[KT_PART * t + 1]);
        for (int c = 0; c < 3; ++c) k3[c] += part[KT_PART * t + 2 + c];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    for (int c = 0; c < 3; ++c) sk[c][threadIdx.x] = k3[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] = fmax(sb[threadIdx.x], sb[threadIdx.x + o]);
            for (int c = 0; c < 3; ++c) sk[c][threadIdx.x] += sk[c][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) thermo[TH_KXX + c] = sk[c][0] / ev_amu;
        const double ke = 0.5 * sa[0] / ev_amu;
        const double vmax = sqrt(sb[0]);
        if (advance) {
            thermo[TH_TIME] += thermo[TH_DT];
            thermo[TH_STEP] += 1.0;
            thermo[TH_DTLAST] = thermo[TH_DT];
        }
        thermo[TH_KE] = ke;
        thermo[TH_VMAX] = vmax;
        double dt = thermo[TH_DTMAX];
        const double dmax = thermo[TH_DMAX];
        if (dmax > 0.0 && vmax > 0.0 && dmax / vmax < dt) dt = dmax / vmax;
        thermo[TH_DT] = dt;
        for (int t = 0; t < NT_MAX; ++t) thermo[TH_HKICK + t] = 0.5 * dt * mt.acc[t];
    }
}

// ----------------------------------------------------------------------------
// Cascade protocol pieces (Sec. II.B): Nose-Hoover chain thermostat on a
// group of atoms, Berendsen barostat, PKA launch
// ----------------------------------------------------------------------------

constexpr int NHC_MAX = 8;
// nhc state (device doubles): [0, 8) v_j, [8, 16) xi_j, [16] N_f (3 x group size)
constexpr int NHC_V = 0, NHC_XI = 8, NHC_NF = 16, NHC_N = 17;

struct NhcParams {
    int M;          // chain length
    double kT;      // eV
    double tau2;    // tau^2 (fs^2): Q_1 = N_f kT tau^2, Q_j = kT tau^2
};

// 3 x the number of group atoms (group == nullptr: every atom).
static __global__ void k_group_count(int n, const uint8_t* __restrict__ group,
                                     double* __restrict__ nhc)
{
    __shared__ int sc[256];
    int c = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) c += group ? (group[i] != 0) : 1;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sc[threadIdx.x] += sc[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) nhc[NHC_NF] = 3.0 * sc[0];
}

// Per-block sums of 1/2 m v^2 (eV) over the group.
static __global__ void __launch_bounds__(256) k_group_ke(int n, MassTab mt,
                                                        const int32_t* __restrict__ types,
                                                        const uint8_t* __restrict__ group,
                                                        const double* __restrict__ v,
                                                        double ev_amu, double* __restrict__ part)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double k = 0.0;
    if (i < n && (!group || group[i])) {
        const double m = mt.m[species_of(mt, types, i)];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double vv = v[(size_t)a * n + i];
            k += 0.5 * m * vv * vv / ev_amu;
        }
    }
    __shared__ double sh[8];
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

// One chain sweep NHC(d), d = dt/2 (Martyna-Tuckerman-Tobias-Klein splitting):
// reduces the group's kinetic energy, advances the chain, stores the group's
// velocity scale in thermo[TH_NHC_S] and the thermostat energy in
// thermo[TH_ENHC].  One block.
static __global__ void __launch_bounds__(256) k_nhc_chain(const double* __restrict__ part, int nb,
                                                         NhcParams np, double* __restrict__ nhc,
                                                         double* __restrict__ thermo)
{
    __shared__ double sh[256];
    double a = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) a += part[t];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double Kg = sh[0];
    const int M = np.M;
    const double d = 0.5 * thermo[TH_DT];
    const double Nf = nhc[NHC_NF];
    double Q[NHC_MAX], v[NHC_MAX];
    for (int j = 0; j < M; ++j) {
        Q[j] = (j == 0 ? (Nf > 0.0 ? Nf : 1.0) : 1.0) * np.kT * np.tau2;
        v[j] = nhc[NHC_V + j];
    }
    auto G = [&](int j) {
        return j == 0 ? (2.0 * Kg - Nf * np.kT) / Q[0]
                      : (Q[j - 1] * v[j - 1] * v[j - 1] - np.kT) / Q[j];
    };
    auto sub = [&](int j) {
        if (j + 1 < M) v[j] *= exp(-0.25 * d * v[j + 1]);
        v[j] += 0.5 * d * G(j);
        if (j + 1 < M) v[j] *= exp(-0.25 * d * v[j + 1]);
    };
    for (int j = M - 1; j >= 0; --j) sub(j);
    const double s = exp(-d * v[0]);
    Kg *= s * s;
    for (int j = 0; j < M; ++j) nhc[NHC_XI + j] += d * v[j];
    for (int j = 0; j < M; ++j) sub(j);
    double e = 0.0;
    for (int j = 0; j < M; ++j) {
        nhc[NHC_V + j] = v[j];
        e += 0.5 * Q[j] * v[j] * v[j];
    }
    e += Nf * np.kT * nhc[NHC_XI];
    for (int j = 1; j < M; ++j) e += np.kT * nhc[NHC_XI + j];
    thermo[TH_NHC_S] = s;
    thermo[TH_ENHC] = e;
}

// Group velocities *= thermo[TH_NHC_S].
static __global__ void k_group_scale(int n, const uint8_t* __restrict__ group,
                                     const double* __restrict__ thermo, double* __restrict__ v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (group && !group[i])) return;
    const double s = thermo[TH_NHC_S];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[(size_t)a * n + i] *= s;
}

// Berendsen barostat (one thread): with P_aa = (sum m v_a^2 + W_aa) / V,
// mu_a = [1 - beta (dt / tau_p) (p0 - P_aa)]^(1/3) for periodic a, 1 otherwise;
// box[a] *= mu_a.  result = (E, W[9]) of the current positions.
static __global__ void k_barostat(const double* __restrict__ result, double* __restrict__ thermo,
                                  double* __restrict__ box, int3 pbc, double p0, double tau_p,
                                  double beta)
{
    if (threadIdx.x != 0) return;
    const double V = box[0] * box[1] * box[2];
    const int per[3] = {pbc.x, pbc.y, pbc.z};
    const double dt = thermo[TH_DT];
    for (int a = 0; a < 3; ++a) {
        double mu = 1.0;
        if (per[a]) {
            const double P = (thermo[TH_KXX + a] + result[1 + 4 * a]) / V;
            mu = cbrt(1.0 - beta * (dt / tau_p) * (p0 - P));
        }
        thermo[TH_MU + a] = mu;
    }
    for (int a = 0; a < 3; ++a) box[a] *= thermo[TH_MU + a];
}

// x_a *= mu_a.
static __global__ void k_scale_positions(int n, const double* __restrict__ thermo,
                                         double* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) x[(size_t)a * n + i] *= thermo[TH_MU + a];
}

// PKA: per-block nearest atom to p (minimum image in periodic dimensions),
// ties to the lowest index; out[2 * b] = d^2, out[2 * b + 1] = index.
static __global__ void __launch_bounds__(256) k_nearest(int n, const double* __restrict__ x,
                                                       double3 p, const Grid g,
                                                       double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double best = 1e300;
    int bi = n;
    if (i < n) {
        const double c[3] = {p.x, p.y, p.z};
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = x[(size_t)a * n + i] - c[a];
        if (g.tric) {
            min_image_tric(g, d);
        } else {
            for (int a = 0; a < 3; ++a)
                if (g.pbc[a]) d[a] -= g.L[a] * rint(d[a] / g.L[a]);
        }
        best = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        bi = i;
    }
    __shared__ double sd[256];
    __shared__ int si[256];
    sd[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double d2 = sd[threadIdx.x + o];
            const int i2 = si[threadIdx.x + o];
            if (d2 < sd[threadIdx.x] || (d2 == sd[threadIdx.x] && i2 < si[threadIdx.x])) {
                sd[threadIdx.x] = d2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = sd[0];
        out[2 * blockIdx.x + 1] = (double)si[0];
    }
}

// Picks the nearest atom from the block results (fixed order) and gives it
// the velocity of kinetic energy e (eV) along the unit vector u:
// |v| = sqrt(2 e / m); result index in *atom.
static __global__ void k_pka_set(const double* __restrict__ part, int nb, int n, MassTab mt,
                                 const int32_t* __restrict__ types, double e, double3 u,
                                 double ev_amu, double* __restrict__ v,
                                 long long* __restrict__ atom)
{
    if (threadIdx.x != 0) return;
    double best = 1e300;
    int bi = n;
    for (int b = 0; b < nb; ++b) {
        const double d2 = part[2 * b];
        const int i2 = (int)part[2 * b + 1];
        if (d2 < best || (d2 == best && i2 < bi)) { best = d2; bi = i2; }
    }
    *atom = bi;
    if (bi >= n) return;
    const double m = mt.m[species_of(mt, types, bi)];
    const double sp = sqrt(2.0 * e / m * ev_amu);
    v[bi] = sp * u.x;
    v[(size_t)n + bi] = sp * u.y;
    v[2 * (size_t)n + bi] = sp * u.z;
}

}  // namespace nepk
