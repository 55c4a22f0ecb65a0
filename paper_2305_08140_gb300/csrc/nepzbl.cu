// nepzbl.cu -- C ABI of the NEP-ZBL library: context, scratch memory, one
// force evaluation and graph-captured velocity-Verlet MD (see nepzbl.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/nepzbl.h"
#include "nep_batch.cuh"
#include "nep_batch_launch.h"
#include "nep_tmem.cuh"

using namespace nepk;

namespace {

// e^2 / (4 pi eps0) in eV*A (CODATA), prefactor of Eq. 2
constexpr double COULOMB_EV_A = 14.39964547;
// 1 eV/amu in A^2/fs^2
constexpr double EV_AMU = 1.602176634e-19 / 1.66053906660e-27 * 1e-10;
// Boltzmann constant (eV/K) and 1 eV/A^3 in GPa (CODATA)
constexpr double KB_EV = 8.617333262e-5;
constexpr double EV_A3_GPA = 160.21766208;
// longest neighbour list (slots) the force kernel stages in shared memory
constexpr int STAGE_MAX_SLOTS = 32;
// the one-species FP32 angular kernel keeps its per-atom angular state in Tensor Memory
// except in the tiles (TILE atoms) with an atom of more than TMEM_MAX_ANG angular
// neighbours (dense clumps, where the register kernel measured faster) or with a
// pair inside the outer ZBL radius: both kernels are launched and each takes the
// tiles the radial-descriptor pass marked for it, so the choice depends on the
// data of this evaluation only
constexpr bool USE_TMEM_ANG = true;
constexpr int TMEM_MAX_ANG = TILE_ANG_LIM;
// device status words of a context
constexpr int NSTATUS = 4;

thread_local std::string g_init_error;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    int steps = 0;
};

}  // namespace

struct nep_ctx {
    int precision = NEP_FP32;
    int device = 0;
    int sm_count = 0;                // multiprocessors of the device
    Model<float> mf;
    Model<double> md;
    nep_params hp;                   // hyperparameters, Z and masses (pointers cleared)
    std::vector<double> scaler;
    int ntypes = 1;
    MassTab mt;
    float* coef_f = nullptr;         // several species: [T * T][CSTR] pair coefficients
    double* coef_d = nullptr;
    double rcR = 0.0;
    std::string err;

    // capacities
    int ld = 0;        // atoms
    int M = 0;         // neighbour slots per atom
    int ccap = 0;      // cells
    // scratch (device)
    int *cell_of = nullptr, *slot_of = nullptr, *perm = nullptr, *cell_sorted = nullptr;
    int* invperm = nullptr;          // caller index -> cell-ordered slot
    void* pos4 = nullptr;
    void* rel4 = nullptr;            // cell-relative position by caller index (binning)
    int2* cnt = nullptr;
    int* nbr = nullptr;
    void* facc = nullptr;
    double* partials = nullptr;      // 2 x tiles x NPART
    double* partials2 = nullptr;     // RED1_MAX x NPART
    void* qr = nullptr;              // radial descriptor [NR][ld] (R)
    void* br = nullptr;              // radial adjoint (b_0..b_8, B0, 0, 0) per atom: 3 x V4
    double* vpart = nullptr;
    int *count = nullptr, *start = nullptr, *scan_sums = nullptr;
    double* backup = nullptr;        // x, v, F copies for MD rollback
    // device mirror of a host MD state (md_step_host)
    double* hm_x = nullptr;
    double* hm_v = nullptr;
    double* hm_f = nullptr;
    int32_t* hm_t = nullptr;
    int64_t hm_cap = 0;
    double* thermo = nullptr;        // TH_N doubles
    double* thermo_backup = nullptr;
    double* result = nullptr;        // NPART doubles (E, W)
    int* status = nullptr;           // [0] status bits, [1..2] max counts, [3] tiles
                                     // of the register angular kernel (dispatch)
    int* tflag = nullptr;            // per-tile kernel choice (TILE_CLOSE, TILE_DENSE)
    unsigned long long* pairs = nullptr;
    // pinned host mirrors
    double* h_result = nullptr;      // NPART + TH_N
    int* h_status = nullptr;         // NSTATUS
    unsigned long long* h_pairs = nullptr;

    cudaStream_t cap_stream = nullptr;
    std::map<int, GraphEntry> graphs;
    const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
    int graph_n = -1;
    Grid graph_grid;

    // options and counters
    int timing = 0;
    int chunk = 10;
    int64_t launches = 0;
    int64_t timed_launches = 0;
    double timed_ms = 0.0;
    std::vector<cudaEvent_t> events;   // pairs (start, stop)
    int last_max_total = 0, last_max_ang = 0;
    long long last_pairs_r = 0, last_pairs_a = 0;
    bool capturing = false;
    int capture_kernels = 0;
    int capture_timed = 0;
    int nep_smem_set[4] = {0, 0, 0, 0};
    int radial_q_fused = 0;          // last evaluation summed q in the neighbour kernel
    int ang_tmem = 0;                // last evaluation ran the Tensor-Memory angular kernel
    int last_tiles = 0;              // tiles (TILE atoms) of the last evaluation
    long long ang_tiles = 0, ang_reg_tiles = 0;   // of the last call / graph chunk
    int ang_dispatch = 0;            // last evaluation launched both angular kernels
    int tm_dyn = -1;                 // k_nep_ang_tm dynamic shared memory (-1: not set)
    int tm_blocks = 0;               // its resident blocks per SM
    int tm_dyn_close = -1, tm_blocks_close = 0;   // the same for k_nep_ang_tm<true, false>
    int rf_close_blocks = 0;         // resident blocks per SM of k_radial_force<float, false, true>
    int tm_dyn_ms[2] = {-1, -1}, tm_blocks_ms[2] = {0, 0};   // <false / true, true>
    // Nose-Hoover chain thermostat on a group, Berendsen barostat (MD)
    int nhc_on = 0;
    NhcParams nhc_p;
    const uint8_t* nhc_group = nullptr;   // caller's device flags (nullptr: all atoms)
    double* nhc = nullptr;                // device state [NHC_N]
    double* nhc_backup = nullptr;
    int nhc_counted = -1;                 // atom count the group size was taken for
    int baro_on = 0;
    double baro_p0 = 0.0, baro_tau = 0.0, baro_beta = 0.0;   // eV/A^3, fs, A^3/eV
    double* d_box = nullptr;              // device box lengths [3]
    double* pka_part = nullptr;           // [2 * blocks] nearest-atom search
    long long* pka_atom = nullptr;
    size_t pka_cap = 0;
    // neighbour search tiling (orthorhombic cells): z slices per cell and
    // candidates per unrolled chunk
    int nbr_zs = 1;
    int nbr_chw = 16;
    // Verlet skin for MD (0: rebuild every step)
    double skin = 0.0;
    double* xref = nullptr;          // positions at the last list build (3 x ld)
    int* nbr_act = nullptr;          // this step's pairs within r_c (skin runs) [M][ld]
    int2* cnt_act = nullptr;
    int* gate = nullptr;             // device: 1 = rebuild the lists this step
    unsigned long long* nrebuild = nullptr;
    long long rebuilds = 0;

    // batched configurations (small periodic boxes)
    long long b_ntot_cap = 0;
    int b_S_cap = 0;
    int b_M = 0;
    int* b_nbr = nullptr;
    int2* b_cnt = nullptr;
    void* b_scr = nullptr;
    double* b_gpart = nullptr;
    double* b_lpart = nullptr;
    double* b_E = nullptr;
    double* b_F = nullptr;
    double* b_W = nullptr;           // [S][9] virials
    unsigned char* b_hv = nullptr;   // [S] has-virial mask of the last loss call
    int b_hv_cap = 0;
    long long* b_off = nullptr;
    int* b_order = nullptr;
    double* b_box = nullptr;
    int* b_queue = nullptr;
    // population evaluation (SNES)
    double* p_thetas = nullptr;      // [n_pop][n_params]
    void* p_tables = nullptr;        // several species: n_pop pair tables
    size_t p_tables_cap = 0;
    void* p_models = nullptr;        // n_pop models
    double* p_out = nullptr;         // [n_pop][S][3]
    double* p_util = nullptr;        // [1024]
    double* d_scaler = nullptr;      // [D] FP64 descriptor scaler
    size_t p_thetas_cap = 0, p_models_cap = 0, p_out_cap = 0;
    int b_bt = 128;          // threads per CTA
    int b_per_sm = 0;        // CTAs per SM (0: as many as fit)
    int b_tuned = 0;
    nep_tune_table b_table{};   // the last batched autotune
};

static int fail(nep_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_init_error = buf;
    return code;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, NEP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void count_launch(nep_ctx* ctx)
{
    if (ctx->capturing) ctx->capture_kernels++;
    else ctx->launches++;
}

template <typename T>
static void free_dev(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

static void drop_graphs(nep_ctx* ctx)
{
    for (auto& kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
}

static void free_scratch(nep_ctx* ctx)
{
    drop_graphs(ctx);
    free_dev(ctx->cell_of); free_dev(ctx->slot_of); free_dev(ctx->perm);
    free_dev(ctx->cell_sorted); free_dev(ctx->invperm); free_dev(ctx->pos4); free_dev(ctx->rel4); free_dev(ctx->cnt); free_dev(ctx->nbr);
    free_dev(ctx->facc); free_dev(ctx->partials); free_dev(ctx->partials2); free_dev(ctx->tflag);
    free_dev(ctx->qr); free_dev(ctx->br); free_dev(ctx->xref); free_dev(ctx->nbr_act);
    free_dev(ctx->cnt_act);
    free_dev(ctx->vpart); free_dev(ctx->backup);
    ctx->ld = 0;
    ctx->M = 0;
}

// Atom-sized buffers for n atoms with M neighbour slots.
static int ensure_atoms(nep_ctx* ctx, int n, int M)
{
    if (n <= ctx->ld && M <= ctx->M && ctx->nbr) return NEP_OK;
    int ld = n > ctx->ld ? n + n / 16 + 128 : ctx->ld;
    int MM = M > ctx->M ? M : ctx->M;
    cudaDeviceSynchronize();
    free_scratch(ctx);
    size_t acc = ctx->precision == NEP_FP32 ? sizeof(long long) : sizeof(double);
    size_t p4 = ctx->precision == NEP_FP32 ? sizeof(float4) : sizeof(double4_32a);
    int tiles = (ld + TILE - 1) / TILE;
    int vb = (ld + 255) / 256;
    CK(cudaMalloc(&ctx->cell_of, sizeof(int) * ld));
    CK(cudaMalloc(&ctx->slot_of, sizeof(int) * ld));
    CK(cudaMalloc(&ctx->perm, sizeof(int) * ld));
    CK(cudaMalloc(&ctx->cell_sorted, sizeof(int) * ld));
    CK(cudaMalloc(&ctx->invperm, sizeof(int) * ld));
    // NB_CHUNK - 1 entries of slack: the chunked neighbour search reads past
    // the last atom (those reads are masked off)
    CK(cudaMalloc(&ctx->pos4, p4 * (ld + NB_CHUNK)));
    CK(cudaMemset(ctx->pos4, 0, p4 * (ld + NB_CHUNK)));
    CK(cudaMalloc(&ctx->rel4, p4 * ld));
    CK(cudaMalloc(&ctx->cnt, sizeof(int2) * ld));
    CK(cudaMalloc(&ctx->nbr, sizeof(int) * (size_t)ld * MM));
    CK(cudaMalloc(&ctx->facc, acc * 3 * (size_t)ld));
    CK(cudaMemset(ctx->facc, 0, acc * 3 * (size_t)ld));
    CK(cudaMalloc(&ctx->partials, sizeof(double) * NPART * 2 * (size_t)tiles));
    CK(cudaMalloc(&ctx->tflag, sizeof(int) * (2 * (size_t)tiles + 1)));   // flags, count, list
    const size_t rsz = ctx->precision == NEP_FP32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&ctx->qr, rsz * NR * (size_t)ld));
    CK(cudaMalloc(&ctx->br, rsz * 12 * (size_t)ctx->ntypes * ld));
    CK(cudaMalloc(&ctx->partials2, sizeof(double) * NPART * (size_t)RED1_MAX));
    CK(cudaMalloc(&ctx->vpart, sizeof(double) * KT_PART * (size_t)vb));
    CK(cudaMalloc(&ctx->backup, sizeof(double) * 9 * (size_t)ld));
    CK(cudaMalloc(&ctx->xref, sizeof(double) * 3 * (size_t)ld));
    if (ctx->skin > 0.0) {
        CK(cudaMalloc(&ctx->nbr_act, sizeof(int) * (size_t)ld * MM));
        CK(cudaMalloc(&ctx->cnt_act, sizeof(int2) * (size_t)ld));
    }
    ctx->ld = ld;
    ctx->M = MM;
    return NEP_OK;
}

static int ensure_cells(nep_ctx* ctx, int ncell)
{
    if (ncell <= ctx->ccap) return NEP_OK;
    int cap = ncell + ncell / 8 + 64;
    if (ncell > (1 << 27))
        return fail(ctx, NEP_ERR_BOX, "cell grid too large (%d sub-cells)", ncell);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    free_dev(ctx->count); free_dev(ctx->start); free_dev(ctx->scan_sums);
    CK(cudaMalloc(&ctx->count, sizeof(int) * (size_t)(cap + 1)));
    CK(cudaMalloc(&ctx->start, sizeof(int) * (size_t)(cap + 1)));
    CK(cudaMalloc(&ctx->scan_sums, sizeof(int) * (size_t)SCAN_B));
    ctx->ccap = cap;
    return NEP_OK;
}

// Cell grid for a diagonal box; periodic dims need >= 3 cells of >= rc_R.
static int make_grid(nep_ctx* ctx, int64_t n, const double box[9], const int32_t pbc[3], Grid& g,
                     double rcell = 0.0)
{
    const double rc_cell = rcell > 0.0 ? rcell : ctx->rcR;
    memset(&g, 0, sizeof(Grid));
    for (int t = 0; t < 9; ++t)
        if (!isfinite(box[t])) return fail(ctx, NEP_ERR_BOX, "non-finite cell entry");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && box[3 * a + b] != 0.0) g.tric = 1;
    // H (rows = cell vectors), its inverse, and the perpendicular widths V / |h_b x h_c|
    const double* h = box;
    const double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8],
                 c02 = h[3] * h[7] - h[4] * h[6];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(det > 0.0)) return fail(ctx, NEP_ERR_BOX, "cell volume det(H) = %g must be positive", det);
    for (int t = 0; t < 9; ++t) g.h[t] = h[t];
    g.hinv[0] = c00 / det;
    g.hinv[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    g.hinv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    g.hinv[3] = c01 / det;
    g.hinv[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    g.hinv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    g.hinv[6] = c02 / det;
    g.hinv[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    g.hinv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    for (int a = 0; a < 3; ++a) {
        const double* u = h + 3 * ((a + 1) % 3);
        const double* v = h + 3 * ((a + 2) % 3);
        const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
                     cz = u[0] * v[1] - u[1] * v[0];
        // width along lattice direction a (the box length for a diagonal H)
        const double W = g.tric ? det / sqrt(cx * cx + cy * cy + cz * cz) : box[4 * a];
        if (!(W > 0.0)) return fail(ctx, NEP_ERR_BOX, "cell width %d is %g", a, W);
        int nc = (int)floor(W / rc_cell);
        if (pbc[a]) {
            if (nc < 3)
                return fail(ctx, NEP_ERR_BOX,
                            "periodic cell width %g < 3 x %g A (cell-list path; small boxes go "
                            "through the batched entry points)", W, rc_cell);
        } else if (nc < 1) {
            nc = 1;
        }
        if (nc > 1024) nc = 1024;
        const double L = box[4 * a];
        g.nc[a] = nc;
        g.pbc[a] = pbc[a] ? 1 : 0;
        g.lc[a] = L / nc;
        g.inv_lc[a] = nc / L;
        g.L[a] = L;
        g.invL[a] = 1.0 / L;
    }
    g.n = (int)n;
    g.ntypes = ctx->ntypes;
    g.zs = g.tric ? 1 : ctx->nbr_zs;
    return NEP_OK;
}

// Sub-cells of a grid (cells x z slices): the length of count[] and start[].
static int sub_cells(const Grid& g)
{
    return g.nc[0] * g.nc[1] * g.nc[2] * (g.zs > 1 ? g.zs : 1);
}

static int check_device_ptr(nep_ctx* ctx, const void* p, const char* what)
{
    if (!p) return fail(ctx, NEP_ERR_INVALID_ARG, "%s is NULL", what);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, NEP_ERR_INVALID_ARG, "%s is not a CUDA pointer", what);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(ctx, NEP_ERR_INVALID_ARG, "%s must be device memory", what);
    return NEP_OK;
}

// Dynamic shared memory of k_nep_ang_tm<CLOSE, MS>, set once per context: at
// least what the kernel uses, padded until no more than TM_BLOCKS_PER_SM
// blocks can be resident on an SM (each holds TM_COLS of the 512 Tensor Memory
// columns, so a further block's allocation would wait for one of them to
// finish).  Returns 0 when the kernel cannot be made resident that way (then
// the register kernel takes its tiles).
template <bool CLOSE, bool MS>
static int tmem_dyn_for(nep_ctx* ctx, int& dyn_out, int& blocks_out)
{
    if (dyn_out >= 0) return dyn_out;
    dyn_out = 0;
    int dev_max = 0;
    if (cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_nep_ang_tm<CLOSE, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dev_max - 8192) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t lo = tm_dyn_min<CLOSE, MS>();
    for (size_t dyn = lo; dyn + 8192 <= (size_t)dev_max; dyn += 4096) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_nep_ang_tm<CLOSE, MS>, TILE, dyn) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        if (nb < 1) return 0;
        if (nb <= TM_BLOCKS_PER_SM) {
            dyn_out = (int)dyn;
            blocks_out = nb;
            return dyn_out;
        }
    }
    return 0;
}
static int tmem_dyn_bytes(nep_ctx* ctx, bool ms = false)
{
    return ms ? tmem_dyn_for<false, true>(ctx, ctx->tm_dyn_ms[0], ctx->tm_blocks_ms[0])
              : tmem_dyn_for<false, false>(ctx, ctx->tm_dyn, ctx->tm_blocks);
}
static int tmem_dyn_bytes_close(nep_ctx* ctx, bool ms = false)
{
    return ms ? tmem_dyn_for<true, true>(ctx, ctx->tm_dyn_ms[1], ctx->tm_blocks_ms[1])
              : tmem_dyn_for<true, false>(ctx, ctx->tm_dyn_close, ctx->tm_blocks_close);
}

// The orthorhombic neighbour-search kernel for a chunk width (4, 8, 16).
template <typename R>
static auto neighbor_kernel(bool fuse_q, int chw)
{
    if (chw == 4) return fuse_q ? k_neighbors<R, true, false, true, 4> : k_neighbors<R, false, false, true, 4>;
    if (chw == 16) return fuse_q ? k_neighbors<R, true, false, true, 16> : k_neighbors<R, false, false, true, 16>;
    return fuse_q ? k_neighbors<R, true, false, true, 8> : k_neighbors<R, false, false, true, 8>;
}

// Launches one force evaluation on stream s (no synchronisation).
// Kernels: bin count, 3-kernel scan, scatter, cell finalize, neighbours,
// force kernel, forces out, reduction.
template <typename R>
static int launch_eval(nep_ctx* ctx, const Grid& g0, const double* x, const int32_t* types,
                       double* F, double* site_energy, cudaStream_t s, int timed_slot,
                       int* gate)
{
    Grid g = g0;
    g.ld = ctx->ld;
    g.M = ctx->M;
    const int n = g.n;
    const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
    const int nsub = sub_cells(g);   // cells x z slices (count[], start[])
    const Model<R>* Pp;
    if constexpr (sizeof(R) == 4) Pp = &ctx->mf;
    else Pp = &ctx->md;
    const Model<R>& P = *Pp;
    if (n == 0) return NEP_OK;
    const int tb = 256;
    const int nb = (n + tb - 1) / tb;
    // list cutoffs: r_c, or r_c + skin when the lists are reused between steps
    const double sk = gate ? ctx->skin : 0.0;
    const double rl = ctx->rcR + sk, ra = sqrt(ctx->md.rcA2) + sk;
    if (gate) {
        // rebuild only when an atom moved more than skin/2 since the last build
        k_skin_check<<<nb, tb, 0, s>>>(g, x, ctx->xref, 0.25 * sk * sk, gate);
        count_launch(ctx);
        const int np = std::max(nsub + 1, 3 * n);
        k_skin_rebuild_prep<<<(np + tb - 1) / tb, tb, 0, s>>>(ctx->count, nsub, x, ctx->xref,
                                                             3 * n, gate, ctx->nrebuild);
        count_launch(ctx);
    } else {
        CK(cudaMemsetAsync(ctx->count, 0, sizeof(int) * (size_t)(nsub + 1), s));
        CK(cudaMemsetAsync(ctx->pairs, 0, sizeof(unsigned long long) * 2, s));
    }
    k_bin_count<R><<<nb, tb, 0, s>>>(g, x, ctx->cell_of, ctx->slot_of, ctx->count, ctx->status, gate,
                                     (typename V4<R>::T*)ctx->rel4);
    count_launch(ctx);
    const int sb = (nsub + SCAN_B - 1) / SCAN_B;
    k_scan_blocks<<<sb, SCAN_T, 0, s>>>(ctx->count, nsub, ctx->start, ctx->scan_sums, gate);
    count_launch(ctx);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(ctx->scan_sums, sb, ctx->start, nsub, gate);
    count_launch(ctx);
    k_scan_add<<<(nsub + tb - 1) / tb, tb, 0, s>>>(ctx->start, nsub, ctx->scan_sums, gate);
    count_launch(ctx);
    k_bin_scatter<<<nb, tb, 0, s>>>(n, ctx->cell_of, ctx->slot_of, ctx->start, ctx->perm, gate);
    count_launch(ctx);
    // one warp per cell (the positions relative to the cells from k_bin_count)
    k_cell_finalize_w<R><<<(int)(((size_t)ncell * 32 + 255) / 256), 256, 0, s>>>(
        g, ncell, ctx->start, ctx->perm, types, (typename V4<R>::T*)ctx->pos4, ctx->cell_sorted,
        ctx->status, gate, ctx->invperm, (const typename V4<R>::T*)ctx->rel4);
    count_launch(ctx);
    // one species, lists rebuilt every step, FP32: the neighbour kernel also
    // sums the radial descriptor (no separate radial-descriptor pass); the
    // FP64 path keeps the separate pass (FP64 arithmetic in the divergent hit
    // branch of the search costs more than the pass)
    const bool ms = ctx->ntypes > 1;
    // (several species: the orthorhombic search with chunks of 16, basis sums
    // per neighbour species)
    const bool fuse_q = !gate && sizeof(R) == 4 && (!ms || (!g.tric && ctx->nbr_chw == 16));
    RadCoef<R> rq;
    rq.inv_rcR = P.inv_rcR;
    for (int t = 0; t < NR * KR; ++t) rq.hR[t] = P.hR[t];
    for (int t = 0; t < NR; ++t) rq.CR[t] = P.CR[t];
    rq.close2 = P.zbl_r2 * P.zbl_r2;
    // FP32: the angular kernels (and, with one species, the radial-force
    // kernels) are chosen tile by tile; the radial-descriptor pass (here or in
    // k_radial_q) marks the tiles in tflag (blocks of TILE atoms = tiles)
    const bool tiled = sizeof(R) == 4;
    const bool dispatch = tiled && USE_TMEM_ANG && tmem_dyn_bytes(ctx, ms) > 0;
    const int tiles = (n + TILE - 1) / TILE;
    int* tfl = tiled ? ctx->tflag : nullptr;
    if (tiled) CK(cudaMemsetAsync(ctx->tflag, 0, sizeof(int) * ((size_t)tiles + 1), s));
    // chunked candidate tests (pos4 holds NB_CHUNK - 1 readable entries past
    // the last atom, see ensure_atoms)
    auto kn = g.tric ? (fuse_q ? k_neighbors<R, true, true, true> : k_neighbors<R, false, true, true>)
                     : neighbor_kernel<R>(fuse_q, ctx->nbr_chw);
    if (fuse_q && ms)
        kn = ctx->ntypes <= 2 ? k_neighbors<R, true, false, true, 16, 2>
                              : k_neighbors<R, true, false, true, 16, 4>;
    const R* coefR;
    if constexpr (sizeof(R) == 4) coefR = ctx->coef_f;
    else coefR = ctx->coef_d;
    kn<<<(n + 127) / 128, 128, 0, s>>>(
        g, (R)(rl * rl), (R)(ra * ra), (const typename V4<R>::T*)ctx->pos4, ctx->cell_sorted,
        ctx->start, ctx->nbr, ctx->cnt, ctx->status, ctx->status + 1, ctx->pairs, gate, rq,
        (R*)ctx->qr, ctx->perm, x, fuse_q ? tfl : nullptr, ms ? coefR : nullptr);
    count_launch(ctx);
    ctx->radial_q_fused = fuse_q ? 1 : 0;
    if (gate) {
        // cell-relative positions of this step (cells as of the last build)
        k_refresh_pos4<R><<<nb, tb, 0, s>>>(g, ctx->perm, ctx->cell_sorted, x,
                                           (typename V4<R>::T*)ctx->pos4);
        count_launch(ctx);
    }
    // force accumulators start at zero (the forces are gathered out of them)
    CK(cudaMemsetAsync(ctx->facc, 0, sizeof(typename Acc<R>::T) * 3 * (size_t)ctx->ld, s));
    // the force kernels are timed together when timing is on
    if (timed_slot >= 0) {
        if (ctx->capturing)
            CK(cudaEventRecordWithFlags(ctx->events[2 * timed_slot], s, cudaEventRecordExternal));
        else
            CK(cudaEventRecord(ctx->events[2 * timed_slot], s));
    }
    // radial descriptor (all pairs, small state)
    const typename V4<R>::T* p4 = (const typename V4<R>::T*)ctx->pos4;
    typename Acc<R>::T* fa = (typename Acc<R>::T*)ctx->facc;
    // with a skin: this step's lists within r_c go to nbr_act / cnt_act
    int* lnbr = gate ? ctx->nbr_act : ctx->nbr;
    int2* lcnt = gate ? ctx->cnt_act : ctx->cnt;
    const R* coef;
    if constexpr (sizeof(R) == 4) coef = ctx->coef_f;
    else coef = ctx->coef_d;
    if (!fuse_q) {
        (ms ? k_radial_q<R, true> : k_radial_q<R, false>)<<<(n + 127) / 128, 128, 0, s>>>(
            P, g, p4, ctx->nbr, ctx->cnt, (R*)ctx->qr, gate ? ctx->nbr_act : nullptr,
            gate ? ctx->cnt_act : nullptr, coef, ctx->perm, x, ctx->status, tfl);
        count_launch(ctx);
    }
    // angular part, network, ZBL (the block's angular entries staged in shared
    // memory when they fit; with several species the pair coefficients first)
    const int stage_slots = ctx->M < STAGE_MAX_SLOTS ? ctx->M : STAGE_MAX_SLOTS;
    const size_t coef_bytes = ms ? sizeof(R) * (size_t)ctx->ntypes * ctx->ntypes * CSTR : 0;
    // (FP32: the close-pair lists behind them, see CQ)
    const size_t stage_bytes = coef_bytes + sizeof(int) * (size_t)stage_slots * TILE +
                               (sizeof(R) == 4 ? CQ_BYTES : 0);
    auto kang = ms ? k_nep_ang<R, true> : k_nep_ang<R, false>;
    const int ks = (sizeof(R) == 4 ? 0 : 2) + (ms ? 1 : 0);
    if (!ctx->nep_smem_set[ks]) {
        CK(cudaFuncSetAttribute(kang, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(R) * NT_MAX * NT_MAX * CSTR +
                                      sizeof(int) * STAGE_MAX_SLOTS * TILE +
                                      (sizeof(R) == 4 ? CQ_BYTES : 0))));
        ctx->nep_smem_set[ks] = 1;
    }
    ctx->ang_dispatch = dispatch ? 1 : 0;
    ctx->last_tiles = tiles;
    // tiles with a close pair: the Tensor-Memory kernel with the close-pair
    // and ZBL branches when it can be made resident, else the register kernel
    const bool tm_close = dispatch && tmem_dyn_bytes_close(ctx, ms) > 0;
    if constexpr (sizeof(R) == 4) {
        // (few tiles have close pairs: a grid of a few blocks per SM loops over
        // the listed tiles and takes those)
        const int cg = tiles < TM_BLOCKS_PER_SM * ctx->sm_count ? tiles
                                                                 : TM_BLOCKS_PER_SM * ctx->sm_count;
        const float* cf = ctx->coef_f;
        if (dispatch) {
            // FP32: the angular state in Tensor Memory
            (ms ? k_nep_ang_tm<false, true> : k_nep_ang_tm<false, false>)
                <<<tiles, TILE, (size_t)tmem_dyn_bytes(ctx, ms), s>>>(
                    P, g, p4, lnbr, lcnt, ctx->perm, x, (const float*)ctx->qr, (float4*)ctx->br,
                    fa, ctx->partials, site_energy, ctx->status, stage_slots, ctx->tflag, cf);
            count_launch(ctx);
        }
        if (tm_close) {
            (ms ? k_nep_ang_tm<true, true> : k_nep_ang_tm<true, false>)
                <<<cg, TILE, (size_t)tmem_dyn_bytes_close(ctx, ms), s>>>(
                    P, g, p4, lnbr, lcnt, ctx->perm, x, (const float*)ctx->qr, (float4*)ctx->br,
                    fa, ctx->partials, site_energy, ctx->status, stage_slots, ctx->tflag, cf);
            count_launch(ctx);
        }
    }
    // with the dispatch the register kernel rarely runs on lattices: a grid of a
    // few blocks per SM, looping over the tiles, makes its early return cheap
    const int ang_grid = dispatch && tiles > 4 * ctx->sm_count ? 4 * ctx->sm_count : tiles;
    kang<<<ang_grid, TILE, stage_bytes, s>>>(P, g, p4, lnbr, lcnt, ctx->perm, x, (const R*)ctx->qr,
                                          (typename V4<R>::T*)ctx->br, fa, ctx->partials,
                                          site_energy, ctx->status, stage_slots, coef,
                                          dispatch ? ctx->tflag : nullptr, ctx->status + 3,
                                          tm_close ? TILE_DENSE : TILE_DENSE | TILE_CLOSE);
    count_launch(ctx);
    // radial pair forces (all pairs, small state); FP32 one species: the
    // variant without the close-pair branch on the tiles without a pair inside
    // the outer ZBL radius, the other on the rest (both launched)
    if (tiled && !ms) {
        k_radial_force<R, false, false><<<tiles, TILE, 0, s>>>(
            P, g, p4, lnbr, lcnt, (const typename V4<R>::T*)ctx->br, fa,
            ctx->partials + (size_t)tiles * NPART, ctx->status, ctx->perm, x, tfl);
        count_launch(ctx);
        // (the close-pair variant loops over the listed tiles on a grid of as
        // many blocks as are resident at once: cheap when the list is empty,
        // at full occupancy when it is long)
        if (ctx->rf_close_blocks == 0) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_radial_force<R, false, true>,
                                                              TILE, 0) != cudaSuccess ||
                nb < 1) {
                cudaGetLastError();
                nb = 4;
            }
            ctx->rf_close_blocks = nb;
        }
        const int close_cap = ctx->rf_close_blocks * ctx->sm_count;
        const int close_grid = tiles < close_cap ? tiles : close_cap;
        k_radial_force<R, false, true><<<close_grid > 0 ? close_grid : 1, TILE, 0, s>>>(
            P, g, p4, lnbr, lcnt, (const typename V4<R>::T*)ctx->br, fa,
            ctx->partials + (size_t)tiles * NPART, ctx->status, ctx->perm, x, tfl);
        count_launch(ctx);
    } else {
        (ms ? k_radial_force<R, true> : k_radial_force<R, false>)<<<tiles, TILE, 0, s>>>(
            P, g, p4, lnbr, lcnt, (const typename V4<R>::T*)ctx->br, fa,
            ctx->partials + (size_t)tiles * NPART, ctx->status, ctx->perm, x, nullptr);
        count_launch(ctx);
    }
    if (timed_slot >= 0) {
        if (ctx->capturing)
            CK(cudaEventRecordWithFlags(ctx->events[2 * timed_slot + 1], s, cudaEventRecordExternal));
        else
            CK(cudaEventRecord(ctx->events[2 * timed_slot + 1], s));
    }
    k_forces_gather<R><<<nb, tb, 0, s>>>(n, ctx->ld, ctx->invperm,
                                         (const typename Acc<R>::T*)ctx->facc, F, ctx->status);
    count_launch(ctx);
    {
        // two-stage fixed-order sum of the per-tile energy/virial partials
        const int nt = 2 * tiles;   // angular/energy tiles, then radial tiles
        const int chunk = (nt + RED1_MAX - 1) / RED1_MAX > 64 ? (nt + RED1_MAX - 1) / RED1_MAX : 64;
        const int nb1 = (nt + chunk - 1) / chunk;
        k_reduce_stage1<<<nb1, 256, 0, s>>>(ctx->partials, nt, chunk, ctx->partials2);
        count_launch(ctx);
        k_reduce_partials<<<1, 256, 0, s>>>(ctx->partials2, nb1, ctx->result);
        count_launch(ctx);
    }
    CK(cudaGetLastError());
    return NEP_OK;
}

static int eval(nep_ctx* ctx, const Grid& g, const double* x, const int32_t* types, double* F,
                double* site_energy, cudaStream_t s, int timed_slot, int* gate = nullptr)
{
    return ctx->precision == NEP_FP32
               ? launch_eval<float>(ctx, g, x, types, F, site_energy, s, timed_slot, gate)
               : launch_eval<double>(ctx, g, x, types, F, site_energy, s, timed_slot, gate);
}

static int ensure_events(nep_ctx* ctx, int pairs)
{
    while ((int)ctx->events.size() < 2 * pairs) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->events.push_back(e);
    }
    return NEP_OK;
}

static int collect_timing(nep_ctx* ctx, int count)
{
    for (int t = 0; t < count; ++t) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->events[2 * t], ctx->events[2 * t + 1]));
        ctx->timed_ms += ms;
        ctx->timed_launches++;
    }
    return NEP_OK;
}

// Reads status, counters and results to pinned host memory and waits.
static int readback(nep_ctx* ctx, cudaStream_t s, int evals = 1)
{
    CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int) * NSTATUS, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_pairs, ctx->pairs, sizeof(unsigned long long) * 2,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_result, ctx->result, sizeof(double) * NPART, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_result + NPART, ctx->thermo, sizeof(double) * TH_N,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->last_max_total = ctx->h_status[1];
    ctx->last_max_ang = ctx->h_status[2];
    // angular tiles of these evaluations, and those the register kernel took
    ctx->ang_tiles = (long long)ctx->last_tiles * evals;
    ctx->ang_reg_tiles = ctx->ang_dispatch ? ctx->h_status[3] : ctx->ang_tiles;
    ctx->ang_tmem = ctx->ang_dispatch && ctx->ang_reg_tiles < ctx->ang_tiles ? 1 : 0;
    ctx->last_pairs_r = (long long)ctx->h_pairs[0];
    ctx->last_pairs_a = (long long)ctx->h_pairs[1];
    return NEP_OK;
}

static int grown_capacity(int needed) { return needed + needed / 4 + 8; }

template <typename R>
static void build_model(Model<R>& P, const nep_params* p)
{
    const int Dd = D, Hh = H;
    const double* w0 = p->params;
    const double* b0 = w0 + Hh * Dd;
    const double* w1 = b0 + Hh;
    const double* b1 = w1 + Hh;
    const double* cR = b1 + 1;
    const double* cA = cR + NR * KR;
    for (int mu = 0; mu < Hh; ++mu)
        for (int nu = 0; nu < Dd; ++nu) P.w0[mu * Dd + nu] = (R)(w0[mu * Dd + nu] * p->q_scaler[nu]);
    for (int mu = 0; mu < Hh; ++mu) {
        P.b0[mu] = (R)b0[mu];
        P.w1[mu] = (R)w1[mu];
    }
    P.b1 = (R)b1[0];
    for (int n = 0; n < NR; ++n) {
        double s = 0.0;
        for (int k = 0; k < KR; ++k) {
            P.hR[n * KR + k] = (R)(0.5 * cR[n * KR + k]);
            s += 0.5 * cR[n * KR + k];
        }
        P.CR[n] = (R)s;
    }
    for (int n = 0; n < NA; ++n) {
        double s = 0.0;
        for (int k = 0; k < KA; ++k) {
            P.hA[n * KA + k] = (R)(0.5 * cA[n * KA + k]);
            s += 0.5 * cA[n * KA + k];
        }
        P.CA[n] = (R)s;
    }
    for (int nu = 0; nu < Dd; ++nu) P.sc[nu] = (R)p->q_scaler[nu];
    P.rcR2 = (R)(p->rc_radial * p->rc_radial);
    P.rcA2 = (R)(p->rc_angular * p->rc_angular);
    P.inv_rcR = (R)(1.0 / p->rc_radial);
    P.inv_rcA = (R)(1.0 / p->rc_angular);
    P.zbl_r2 = (R)p->zbl_r_outer;
    const double Z = (double)p->z[0];
    P.zbl_k = COULOMB_EV_A * Z * Z;
    P.zbl_inv_a = (pow(Z, 0.23) + pow(Z, 0.23)) / 0.46848;
    P.zbl_r1 = p->zbl_r_inner;
    P.zbl_rr2 = p->zbl_r_outer;
    // ZBL prefactor and screening length of every ordered species pair (Eq. 2, 4)
    const int T = p->n_types < 1 ? 1 : p->n_types;
    P.ntypes = T;
    for (int a = 0; a < NT_MAX * NT_MAX; ++a) { P.zbl_kp[a] = 0.0; P.zbl_inv_ap[a] = 0.0; }
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const double Za = (double)p->z[a], Zb = (double)p->z[b];
            P.zbl_kp[a * T + b] = COULOMB_EV_A * Za * Zb;
            P.zbl_inv_ap[a * T + b] = (pow(Za, 0.23) + pow(Zb, 0.23)) / 0.46848;
        }
}

// Number of model parameters for T species.
static int64_t n_params_for(int T)
{
    return (int64_t)H * D + 2 * H + 1 + (int64_t)T * T * (NR * KR + NA * KA);
}

// Pair coefficient table [T * T][CSTR] (h = c/2 and C = sum_k c/2 of every
// ordered species pair, radial then angular) in precision R.
template <typename R>
static void pair_table(const nep_params* p, std::vector<R>& tab)
{
    const int T = p->n_types;
    const double* cR = p->params + (int64_t)H * D + 2 * H + 1;
    const double* cA = cR + (int64_t)T * T * NR * KR;
    tab.assign((size_t)T * T * CSTR, R(0));
    for (int pr = 0; pr < T * T; ++pr) {
        R* o = tab.data() + (size_t)pr * CSTR;
        for (int n = 0; n < NR; ++n) {
            double sum = 0.0;
            for (int k = 0; k < KR; ++k) {
                const double h = 0.5 * cR[((size_t)pr * NR + n) * KR + k];
                o[C_RAD + n * KR + k] = (R)h;
                sum += h;
            }
            o[C_RAD + NR * KR + n] = (R)sum;
        }
        for (int n = 0; n < NA; ++n) {
            double sum = 0.0;
            for (int k = 0; k < KA; ++k) {
                const double h = 0.5 * cA[((size_t)pr * NA + n) * KA + k];
                o[C_ANG + n * KA + k] = (R)h;
                sum += h;
            }
            o[C_ANG + NA * KA + n] = (R)sum;
        }
    }
}

// Builds both precisions' models and, for several species, the device pair
// tables, from the stored hyperparameters and `params`.
static int setup_model(nep_ctx* ctx, const double* params)
{
    nep_params p = ctx->hp;
    p.params = params;
    p.q_scaler = ctx->scaler.data();
    const int T = p.n_types;
    if (T == 1) {
        build_model<float>(ctx->mf, &p);
        build_model<double>(ctx->md, &p);
    } else {
        // the one-species fields hold block (0, 0); the kernels for several
        // species read the pair tables instead
        std::vector<double> one((size_t)n_params_for(1));
        const int64_t head = (int64_t)H * D + 2 * H + 1;
        std::copy(params, params + head, one.begin());
        std::copy(params + head, params + head + NR * KR, one.begin() + head);
        std::copy(params + head + (int64_t)T * T * NR * KR,
                  params + head + (int64_t)T * T * NR * KR + NA * KA,
                  one.begin() + head + NR * KR);
        nep_params p1 = p;
        p1.params = one.data();
        p1.n_params = (int64_t)one.size();
        build_model<float>(ctx->mf, &p1);
        build_model<double>(ctx->md, &p1);
        std::vector<float> tf;
        std::vector<double> td;
        pair_table<float>(&p, tf);
        pair_table<double>(&p, td);
        if (!ctx->coef_f) CK(cudaMalloc(&ctx->coef_f, sizeof(float) * tf.size()));
        if (!ctx->coef_d) CK(cudaMalloc(&ctx->coef_d, sizeof(double) * td.size()));
        CK(cudaMemcpy(ctx->coef_f, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->coef_d, td.data(), sizeof(double) * td.size(), cudaMemcpyHostToDevice));
    }
    return NEP_OK;
}

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

int nep_init(const nep_params* p, int precision, nep_ctx** out)
{
    nep_ctx* ctx = nullptr;
    if (!p || !out) return fail(nullptr, NEP_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (precision != NEP_FP32 && precision != NEP_FP64)
        return fail(nullptr, NEP_ERR_INVALID_ARG, "precision must be NEP_FP32 or NEP_FP64");
    if (p->n_types < 1 || p->n_types > NT_MAX)
        return fail(nullptr, NEP_ERR_UNSUPPORTED, "n_types must be 1..%d", NT_MAX);
    if (p->n_max_radial != NR - 1 || p->n_max_angular != NA - 1 ||
        p->basis_size_radial != KR - 1 || p->basis_size_angular != KA - 1 || p->l_max != LM ||
        p->use_4body != 1 || p->n_hidden != H)
        return fail(nullptr, NEP_ERR_UNSUPPORTED,
                    "this build is compiled for n_max 4/4, basis 8/8, l_max 4, 4-body, 30 neurons");
    const int64_t np = n_params_for(p->n_types);
    if (!p->params || p->n_params != np)
        return fail(nullptr, NEP_ERR_INVALID_ARG, "params must hold %lld values", (long long)np);
    if (!p->q_scaler) return fail(nullptr, NEP_ERR_INVALID_ARG, "q_scaler is NULL");
    for (int64_t i = 0; i < np; ++i)
        if (!isfinite(p->params[i])) return fail(nullptr, NEP_ERR_INVALID_ARG, "non-finite parameter");
    for (int i = 0; i < D; ++i)
        if (!isfinite(p->q_scaler[i])) return fail(nullptr, NEP_ERR_INVALID_ARG, "non-finite scaler");
    if (!(p->rc_radial > 0) || !(p->rc_angular > 0) || p->rc_angular > p->rc_radial ||
        !(p->zbl_r_outer > p->zbl_r_inner) || !(p->zbl_r_inner >= 0) ||
        p->zbl_r_outer > p->rc_angular)
        return fail(nullptr, NEP_ERR_INVALID_ARG,
                    "need 0 <= zbl_r_inner < zbl_r_outer <= rc_angular <= rc_radial");
    for (int t = 0; t < p->n_types; ++t)
        if (!(p->z[t] > 0) || !(p->mass[t] > 0) || !isfinite(p->mass[t]))
            return fail(nullptr, NEP_ERR_INVALID_ARG, "Z and mass of species %d must be positive", t);

    ctx = new (std::nothrow) nep_ctx();
    if (!ctx) return fail(nullptr, NEP_ERR_INVALID_ARG, "out of host memory");
    ctx->precision = precision;
    ctx->rcR = p->rc_radial;
    ctx->hp = *p;
    ctx->hp.params = nullptr;
    ctx->hp.q_scaler = nullptr;
    ctx->scaler.assign(p->q_scaler, p->q_scaler + D);
    ctx->ntypes = p->n_types;
    ctx->mt.ntypes = p->n_types;
    for (int t = 0; t < NT_MAX; ++t) {
        const double m = t < p->n_types ? p->mass[t] : 1.0;
        ctx->mt.m[t] = m;
        ctx->mt.acc[t] = EV_AMU / m;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->thermo, sizeof(double) * TH_N);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->thermo_backup, sizeof(double) * TH_N);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->result, sizeof(double) * NPART);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(int) * NSTATUS);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->pairs, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->gate, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->nrebuild, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->nrebuild, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_result, sizeof(double) * (NPART + TH_N));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, sizeof(int) * NSTATUS);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pairs, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess) e = cudaMemset(ctx->thermo, 0, sizeof(double) * TH_N);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(int) * NSTATUS);
    if (e != cudaSuccess) {
        int rc = fail(nullptr, NEP_ERR_CUDA, "CUDA setup failed: %s", cudaGetErrorString(e));
        nep_free(ctx);
        return rc;
    }
    if (setup_model(ctx, p->params) != NEP_OK) {
        int rc = fail(nullptr, NEP_ERR_CUDA, "%s", ctx->err.c_str());
        nep_free(ctx);
        return rc;
    }
    ctx->M = 0;
    *out = ctx;
    return NEP_OK;
}

static void free_batch(nep_ctx* ctx)
{
    free_dev(ctx->b_nbr); free_dev(ctx->b_cnt); free_dev(ctx->b_scr); free_dev(ctx->b_gpart);
    free_dev(ctx->b_lpart); free_dev(ctx->b_E); free_dev(ctx->b_F); free_dev(ctx->b_off);
    free_dev(ctx->b_order); free_dev(ctx->b_box); free_dev(ctx->b_queue); free_dev(ctx->b_W);
    ctx->b_ntot_cap = 0;
    ctx->b_S_cap = 0;
    ctx->b_M = 0;
}

void nep_free(nep_ctx* ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_scratch(ctx);
    free_batch(ctx);
    free_dev(ctx->count); free_dev(ctx->start); free_dev(ctx->scan_sums);
    free_dev(ctx->thermo); free_dev(ctx->thermo_backup); free_dev(ctx->result);
    free_dev(ctx->status); free_dev(ctx->pairs); free_dev(ctx->gate); free_dev(ctx->nrebuild);
    free_dev(ctx->coef_f); free_dev(ctx->coef_d); free_dev(ctx->b_hv);
    free_dev(ctx->p_thetas); free_dev(ctx->p_models); free_dev(ctx->p_out); free_dev(ctx->p_util);
    free_dev(ctx->p_tables);
    free_dev(ctx->d_scaler);
    free_dev(ctx->nhc); free_dev(ctx->nhc_backup); free_dev(ctx->d_box); free_dev(ctx->pka_part);
    free_dev(ctx->pka_atom);
    free_dev(ctx->hm_x); free_dev(ctx->hm_v); free_dev(ctx->hm_f); free_dev(ctx->hm_t);
    if (ctx->h_result) cudaFreeHost(ctx->h_result);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_pairs) cudaFreeHost(ctx->h_pairs);
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

const char* nep_last_error(const nep_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

int nep_set_option(nep_ctx* ctx, int option, int64_t value)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    switch (option) {
    case NEP_OPT_TIMING:
        ctx->timing = value ? 1 : 0;
        drop_graphs(ctx);
        return NEP_OK;
    case NEP_OPT_GRAPH_CHUNK:
        if (value < 1 || value > 100000) return fail(ctx, NEP_ERR_INVALID_ARG, "bad chunk");
        ctx->chunk = (int)value;
        return NEP_OK;
    case NEP_OPT_SKIN_MILLIANGSTROM:
        if (value < 0 || value > 3000) return fail(ctx, NEP_ERR_INVALID_ARG, "skin must be 0..3 A");
        ctx->skin = value * 1e-3;
        drop_graphs(ctx);
        if (ctx->skin > 0.0 && ctx->ld > 0 && !ctx->nbr_act) {
            cudaDeviceSynchronize();
            const int ld = ctx->ld, M = ctx->M;
            free_scratch(ctx);
            return ensure_atoms(ctx, ld, M);
        }
        return NEP_OK;
    case NEP_OPT_NBR_SLICES:
        if (value != 1 && value != 2 && value != 4 && value != 8)
            return fail(ctx, NEP_ERR_INVALID_ARG, "z slices per cell must be 1, 2, 4 or 8");
        ctx->nbr_zs = (int)value;
        drop_graphs(ctx);
        return NEP_OK;
    case NEP_OPT_NBR_CHUNK:
        if (value != 4 && value != 8 && value != 16)
            return fail(ctx, NEP_ERR_INVALID_ARG, "candidate chunk must be 4, 8 or 16");
        ctx->nbr_chw = (int)value;
        drop_graphs(ctx);
        return NEP_OK;
    case NEP_OPT_NBR_CAPACITY:
        if (value < 1 || value > 1000000) return fail(ctx, NEP_ERR_INVALID_ARG, "bad capacity");
        if (ctx->ld > 0) {
            if (value > ctx->M) return ensure_atoms(ctx, ctx->ld, (int)value);
            return NEP_OK;
        }
        ctx->M = (int)value;
        return NEP_OK;
    default:
        return fail(ctx, NEP_ERR_INVALID_ARG, "unknown option %d", option);
    }
}

int nep_get_stats(const nep_ctx* ctx, nep_stats* out)
{
    if (!ctx || !out) return NEP_ERR_INVALID_ARG;
    out->kernel_launches = ctx->launches;
    out->timed_launches = ctx->timed_launches;
    out->timed_ms = ctx->timed_ms;
    out->pairs_radial = ctx->last_pairs_r;
    out->pairs_angular = ctx->last_pairs_a;
    out->max_nbr_radial = ctx->last_max_total;
    out->max_nbr_angular = ctx->last_max_ang;
    out->nbr_capacity = ctx->M;
    out->graph_chunk = ctx->chunk;
    unsigned long long nb = 0;
    if (ctx->nrebuild && cudaMemcpy(&nb, ctx->nrebuild, sizeof(nb), cudaMemcpyDeviceToHost) != cudaSuccess)
        nb = 0;
    out->list_builds_skin = (int64_t)nb;
    out->radial_q_in_neighbor_kernel = ctx->radial_q_fused;
    out->angular_state_in_tmem = ctx->ang_tmem;
    out->angular_tmem_blocks_per_sm = ctx->tm_blocks;
    out->nbr_z_slices = ctx->nbr_zs;
    out->nbr_chunk = ctx->nbr_chw;
    out->angular_tiles = ctx->ang_tiles;
    out->angular_tiles_register = ctx->ang_reg_tiles;
    return NEP_OK;
}

int nep_reset_stats(nep_ctx* ctx)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    ctx->launches = 0;
    ctx->timed_launches = 0;
    ctx->timed_ms = 0.0;
    return NEP_OK;
}

// One evaluation with growth of the neighbour capacity on overflow.
static int compute_with_retry(nep_ctx* ctx, const Grid& g, const double* x, const int32_t* types,
                              double* F, double* site_energy, cudaStream_t s)
{
    int rc = ensure_cells(ctx, sub_cells(g));
    if (rc) return rc;
    int M = ctx->M > 0 ? ctx->M : 96;
    for (int attempt = 0; attempt < 4; ++attempt) {
        rc = ensure_atoms(ctx, g.n, M);
        if (rc) return rc;
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(int) * NSTATUS, s));
        int slot = -1;
        if (ctx->timing) {
            rc = ensure_events(ctx, 1);
            if (rc) return rc;
            slot = 0;
        }
        rc = eval(ctx, g, x, types, F, site_energy, s, slot);
        if (rc) return rc;
        rc = readback(ctx, s);
        if (rc) return rc;
        if (slot == 0 && g.n > 0) {
            rc = collect_timing(ctx, 1);
            if (rc) return rc;
        }
        if (ctx->h_status[0] & ST_BADTYPE)
            return fail(ctx, NEP_ERR_INVALID_ARG, "species index out of range [0, %d)",
                        ctx->ntypes);
        if (ctx->h_status[0] & ST_OVERFLOW) {
            M = grown_capacity(ctx->h_status[1]);
            continue;
        }
        if (ctx->h_status[0] & ST_NONFINITE)
            return fail(ctx, NEP_ERR_NONFINITE, "non-finite positions, energies or forces");
        return NEP_OK;
    }
    return fail(ctx, NEP_ERR_NBR_OVERFLOW, "neighbour capacity could not be grown enough");
}

int nep_compute(nep_ctx* ctx, int64_t n_atoms, const double* xyz, const double box[9],
                const int32_t* types, const int32_t pbc[3], double* energy, double* forces,
                double* virial, double* site_energy, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (n_atoms < 0 || n_atoms >= (1 << 26))
        return fail(ctx, NEP_ERR_INVALID_ARG, "n_atoms must be in [0, 2^26)");
    if (!box || !pbc || !energy) return fail(ctx, NEP_ERR_INVALID_ARG, "NULL host argument");
    Grid g;
    int rc = make_grid(ctx, n_atoms, box, pbc, g);
    if (rc) return rc;
    if (n_atoms == 0) {
        *energy = 0.0;
        if (virial) for (int t = 0; t < 9; ++t) virial[t] = 0.0;
        return NEP_OK;
    }
    if ((rc = check_device_ptr(ctx, xyz, "xyz")) || (rc = check_device_ptr(ctx, types, "types")) ||
        (rc = check_device_ptr(ctx, forces, "forces")))
        return rc;
    if (site_energy && (rc = check_device_ptr(ctx, site_energy, "site_energy"))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    rc = compute_with_retry(ctx, g, xyz, types, forces, site_energy, s);
    if (rc) return rc;
    *energy = ctx->h_result[0];
    if (virial) for (int t = 0; t < 9; ++t) virial[t] = ctx->h_result[1 + t];
    return NEP_OK;
}

// One chain sweep NHC(dt/2) of the thermostatted group (3 kernels).
static void enqueue_nhc(nep_ctx* ctx, int n, const int32_t* types, double* vel, cudaStream_t s)
{
    const int tb = 256, nb = (n + tb - 1) / tb;
    k_group_ke<<<nb, tb, 0, s>>>(n, ctx->mt, types, ctx->nhc_group, vel, EV_AMU, ctx->vpart);
    count_launch(ctx);
    k_nhc_chain<<<1, 256, 0, s>>>(ctx->vpart, nb, ctx->nhc_p, ctx->nhc, ctx->thermo);
    count_launch(ctx);
    k_group_scale<<<nb, tb, 0, s>>>(n, ctx->nhc_group, ctx->thermo, vel);
    count_launch(ctx);
}

// Kick + kinetic statistics (warp sums of m v^2 in FP32 on the FP32 path;
// the half kick and the per-dimension sums chosen at compile time).
static auto kick_thermo_kernel(const nep_ctx* ctx, int half_kick, int tensor)
    -> decltype(&k_kick_thermo<true, true, true>)
{
    const bool lo = ctx->precision == NEP_FP32;
    if (half_kick)
        return tensor ? (lo ? k_kick_thermo<true, true, true> : k_kick_thermo<false, true, true>)
                      : (lo ? k_kick_thermo<true, true, false> : k_kick_thermo<false, true, false>);
    return tensor ? (lo ? k_kick_thermo<true, false, true> : k_kick_thermo<false, false, true>)
                  : (lo ? k_kick_thermo<true, false, false> : k_kick_thermo<false, false, false>);
}

// One velocity-Verlet step on stream s:
//   [NHC(dt/2)] v += dt/2 F/m, x += dt v; F(x); v += dt/2 F/m [NHC(dt/2)];
//   kinetic energy, max |v| and the next dt.
// Blocks of k_kick_thermo (grid-stride): four per SM at most, so that the
// single-block k_thermo_step reduces a few hundred partials.
static int kick_blocks(const nep_ctx* ctx, int n)
{
    const int full = (n + 255) / 256, cap = 4 * (ctx->sm_count > 0 ? ctx->sm_count : 152);
    return full < cap ? (full > 0 ? full : 1) : cap;
}

static int enqueue_step(nep_ctx* ctx, const Grid& g, nep_md_state* st, cudaStream_t s, int slot)
{
    const int n = g.n;
    const int tb = 256, nb = (n + tb - 1) / tb;
    if (ctx->nhc_on) enqueue_nhc(ctx, n, st->types, st->vel, s);
    k_kick_drift<<<nb, tb, 0, s>>>(g, ctx->mt, st->types, ctx->thermo, st->xyz, st->vel,
                                   st->forces);
    count_launch(ctx);
    int* gate = ctx->skin > 0.0 && !ctx->baro_on ? ctx->gate : nullptr;
    int rc = eval(ctx, g, st->xyz, st->types, st->forces, nullptr, s, slot, gate);
    if (rc) return rc;
    const int nkt = kick_blocks(ctx, n);
    kick_thermo_kernel(ctx, 1, ctx->baro_on)<<<nkt, tb, 0, s>>>(n, ctx->mt, st->types, ctx->thermo,
                                                                st->vel, st->forces, ctx->vpart);
    count_launch(ctx);
    if (ctx->nhc_on) {
        enqueue_nhc(ctx, n, st->types, st->vel, s);
        // kinetic energy and speeds after the thermostat's scaling
        kick_thermo_kernel(ctx, 0, ctx->baro_on)<<<nkt, tb, 0, s>>>(n, ctx->mt, st->types,
                                                                    ctx->thermo, st->vel,
                                                                    st->forces, ctx->vpart);
        count_launch(ctx);
    }
    k_thermo_step<<<1, 256, 0, s>>>(ctx->vpart, nkt, EV_AMU, ctx->thermo, 1, ctx->mt, gate);
    count_launch(ctx);
    return NEP_OK;
}

// Captures `steps` MD steps into a graph (on the context's capture stream).
static int capture_steps(nep_ctx* ctx, const Grid& g, nep_md_state* st, int steps, GraphEntry& ge)
{
    cudaStream_t cs = ctx->cap_stream;
    const int n = g.n;
    const int tb = 256, nb = (n + tb - 1) / tb;
    if (ctx->timing) {
        int rc = ensure_events(ctx, steps);
        if (rc) return rc;
    }
    ctx->capturing = true;
    ctx->capture_kernels = 0;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = NEP_OK;
    (void)n;
    (void)nb;
    for (int t = 0; t < steps && !rc; ++t) rc = enqueue_step(ctx, g, st, cs, ctx->timing ? t : -1);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    ctx->capturing = false;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, NEP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return fail(ctx, NEP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    ge.kernels = ctx->capture_kernels;
    ge.steps = steps;
    return NEP_OK;
}

}  // extern "C"

// MD steps with the Berendsen barostat: the box changes every step, so the
// steps are launched directly (no graph): one step, the barostat scale
// mu_a (device), x_a *= mu_a, then the new box is read back to lay the next
// step's cell grid.  A neighbour overflow restores the step's start, grows
// the capacity and repeats the step.
static int md_steps_barostat(nep_ctx* ctx, nep_md_state* st, int n_steps, cudaStream_t s)
{
    const int64_t n = st->n_atoms;
    const size_t bytes = sizeof(double) * 3 * (size_t)n;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && st->box[3 * a + b] != 0.0)
                return fail(ctx, NEP_ERR_UNSUPPORTED, "the barostat scales orthorhombic boxes only");
    double h_box[3] = {st->box[0], st->box[4], st->box[8]};
    CK(cudaMemcpyAsync(ctx->d_box, h_box, sizeof(h_box), cudaMemcpyHostToDevice, s));
    const int3 pbc = make_int3(st->pbc[0] ? 1 : 0, st->pbc[1] ? 1 : 0, st->pbc[2] ? 1 : 0);
    int retries = 0;
    for (int step = 0; step < n_steps;) {
        Grid g;
        int rc = make_grid(ctx, n, st->box, st->pbc, g);
        if (rc) return rc;
        if ((rc = ensure_cells(ctx, sub_cells(g)))) return rc;
        if ((rc = ensure_atoms(ctx, (int)n, ctx->M > 0 ? ctx->M : 96))) return rc;
        CK(cudaMemcpyAsync(ctx->backup, st->xyz, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->backup + 3 * n, st->vel, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->backup + 6 * n, st->forces, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->thermo_backup, ctx->thermo, sizeof(double) * TH_N,
                           cudaMemcpyDeviceToDevice, s));
        if (ctx->nhc_on)
            CK(cudaMemcpyAsync(ctx->nhc_backup, ctx->nhc, sizeof(double) * NHC_N,
                               cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(int) * NSTATUS, s));
        g.ld = ctx->ld;
        g.M = ctx->M;
        if ((rc = enqueue_step(ctx, g, st, s, -1))) return rc;
        k_barostat<<<1, 32, 0, s>>>(ctx->result, ctx->thermo, ctx->d_box, pbc, ctx->baro_p0,
                                    ctx->baro_tau, ctx->baro_beta);
        count_launch(ctx);
        const int tb = 256;
        k_scale_positions<<<(int)((n + tb - 1) / tb), tb, 0, s>>>((int)n, ctx->thermo, st->xyz);
        count_launch(ctx);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h_box, ctx->d_box, sizeof(h_box), cudaMemcpyDeviceToHost, s));
        rc = readback(ctx, s);
        if (rc) return rc;
        if (ctx->h_status[0] & ST_BADTYPE)
            return fail(ctx, NEP_ERR_INVALID_ARG, "species index out of range [0, %d)",
                        ctx->ntypes);
        if (ctx->h_status[0] & ST_OVERFLOW) {
            if (++retries > 4) return fail(ctx, NEP_ERR_NBR_OVERFLOW, "neighbour overflow persists");
            CK(cudaMemcpyAsync(st->xyz, ctx->backup, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(st->vel, ctx->backup + 3 * n, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(st->forces, ctx->backup + 6 * n, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(ctx->thermo, ctx->thermo_backup, sizeof(double) * TH_N,
                               cudaMemcpyDeviceToDevice, s));
            if (ctx->nhc_on)
                CK(cudaMemcpyAsync(ctx->nhc, ctx->nhc_backup, sizeof(double) * NHC_N,
                                   cudaMemcpyDeviceToDevice, s));
            h_box[0] = st->box[0]; h_box[1] = st->box[4]; h_box[2] = st->box[8];
            CK(cudaMemcpyAsync(ctx->d_box, h_box, sizeof(h_box), cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
            if ((rc = ensure_atoms(ctx, (int)n, grown_capacity(ctx->h_status[1])))) return rc;
            continue;
        }
        if (ctx->h_status[0] & ST_NONFINITE)
            return fail(ctx, NEP_ERR_NONFINITE, "non-finite values during MD");
        st->box[0] = h_box[0];
        st->box[4] = h_box[1];
        st->box[8] = h_box[2];
        ++step;
    }
    return NEP_OK;
}

extern "C" {

int md_step(nep_ctx* ctx, nep_md_state* st, int n_steps, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (!st || n_steps < 0) return fail(ctx, NEP_ERR_INVALID_ARG, "bad state or step count");
    const int64_t n = st->n_atoms;
    if (n <= 0 || n >= (1 << 26)) return fail(ctx, NEP_ERR_INVALID_ARG, "n_atoms must be in [1, 2^26)");
    if (!(st->dt_max > 0) || !isfinite(st->dt_max))
        return fail(ctx, NEP_ERR_INVALID_ARG, "dt_max must be positive");
    int rc;
    if ((rc = check_device_ptr(ctx, st->xyz, "xyz")) || (rc = check_device_ptr(ctx, st->vel, "vel")) ||
        (rc = check_device_ptr(ctx, st->forces, "forces")) ||
        (rc = check_device_ptr(ctx, st->types, "types")))
        return rc;
    Grid g0, g;
    if ((rc = make_grid(ctx, n, st->box, st->pbc, g0))) return rc;
    // with a Verlet skin the MD lists (and cells) use r_c + skin
    if ((rc = make_grid(ctx, n, st->box, st->pbc, g, ctx->rcR + ctx->skin))) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!st->forces_valid) {
        rc = compute_with_retry(ctx, g0, st->xyz, st->types, st->forces, nullptr, s);
        if (rc) return rc;
        st->forces_valid = 1;
        st->potential_energy = ctx->h_result[0];
        for (int t = 0; t < 9; ++t) st->virial[t] = ctx->h_result[1 + t];
    }
    {
        int rc2 = ensure_cells(ctx, sub_cells(g));
        if (rc2) return rc2;
        int need = ctx->M > 0 ? ctx->M : 96;
        if (ctx->last_max_total > 0) {
            // lists with a skin hold ((r_c + skin) / r_c)^3 as many pairs
            const double sc = pow((ctx->rcR + ctx->skin) / ctx->rcR, 3.0);
            const int est = grown_capacity((int)ceil(ctx->last_max_total * sc));
            if (est > need) need = est;
        }
        if ((rc2 = ensure_atoms(ctx, (int)n, need))) return rc2;
    }
    // graphs are bound to the state's pointers and sizes
    if (ctx->graph_key[0] != st->xyz || ctx->graph_key[1] != st->vel ||
        ctx->graph_key[2] != st->forces || ctx->graph_key[3] != st->types || ctx->graph_n != n ||
        memcmp(&ctx->graph_grid, &g, sizeof(Grid)) != 0) {
        drop_graphs(ctx);
        ctx->graph_key[0] = st->xyz; ctx->graph_key[1] = st->vel;
        ctx->graph_key[2] = st->forces; ctx->graph_key[3] = st->types;
        ctx->graph_n = (int)n;
        ctx->graph_grid = g;
    }
    // thermo: dt_max, d_max, time, step; initial dt from the current velocities
    double th[TH_N] = {0};
    th[TH_TIME] = st->time;
    th[TH_STEP] = (double)st->step;
    th[TH_DTMAX] = st->dt_max;
    th[TH_DMAX] = st->d_max;
    th[TH_DTLAST] = st->dt_last;
    CK(cudaMemcpyAsync(ctx->thermo, th, sizeof(th), cudaMemcpyHostToDevice, s));
    {
        const int tb = 256;
        kick_thermo_kernel(ctx, 0, ctx->baro_on)<<<kick_blocks(ctx, (int)n), tb, 0, s>>>(
            (int)n, ctx->mt, st->types, ctx->thermo, st->vel, st->forces, ctx->vpart);
        count_launch(ctx);
        k_thermo_step<<<1, 256, 0, s>>>(ctx->vpart, kick_blocks(ctx, (int)n), EV_AMU, ctx->thermo,
                                        0, ctx->mt);
        count_launch(ctx);
        if (ctx->nhc_on && ctx->nhc_counted != (int)n) {
            k_group_count<<<1, 256, 0, s>>>((int)n, ctx->nhc_group, ctx->nhc);
            count_launch(ctx);
            ctx->nhc_counted = (int)n;
        }
        CK(cudaGetLastError());
    }
    if (ctx->baro_on) {
        rc = md_steps_barostat(ctx, st, n_steps, s);
        if (rc) return rc;
        n_steps = n_steps > 0 ? n_steps : 0;
    }
    int done = ctx->baro_on ? n_steps : 0;
    int retries = 0;
    bool force_rebuild = true;   // the caller may have moved atoms since the last call
    while (done < n_steps) {
        const int len = (n_steps - done) < ctx->chunk ? (n_steps - done) : ctx->chunk;
        auto it = ctx->graphs.find(len);
        if (it == ctx->graphs.end()) {
            GraphEntry ge;
            rc = capture_steps(ctx, g, st, len, ge);
            if (rc) return rc;
            it = ctx->graphs.emplace(len, ge).first;
        }
        // rollback copy of x, v, F and the thermo block
        const size_t bytes = sizeof(double) * 3 * (size_t)n;
        CK(cudaMemcpyAsync(ctx->backup, st->xyz, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->backup + 3 * n, st->vel, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->backup + 6 * n, st->forces, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->thermo_backup, ctx->thermo, sizeof(double) * TH_N,
                           cudaMemcpyDeviceToDevice, s));
        if (ctx->nhc_on)
            CK(cudaMemcpyAsync(ctx->nhc_backup, ctx->nhc, sizeof(double) * NHC_N,
                               cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(int) * NSTATUS, s));
        if (ctx->skin > 0.0 && force_rebuild) {
            const int one = 1;
            CK(cudaMemcpyAsync(ctx->gate, &one, sizeof(int), cudaMemcpyHostToDevice, s));
            force_rebuild = false;
        }
        CK(cudaGraphLaunch(it->second.exec, s));
        ctx->launches += it->second.kernels;
        rc = readback(ctx, s, len);
        if (rc) return rc;
        if (ctx->h_status[0] & ST_BADTYPE)
            return fail(ctx, NEP_ERR_INVALID_ARG, "species index out of range [0, %d)",
                        ctx->ntypes);
        if (ctx->h_status[0] & ST_OVERFLOW) {
            if (++retries > 4) return fail(ctx, NEP_ERR_NBR_OVERFLOW, "neighbour overflow persists");
            CK(cudaMemcpyAsync(st->xyz, ctx->backup, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(st->vel, ctx->backup + 3 * n, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(st->forces, ctx->backup + 6 * n, bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(ctx->thermo, ctx->thermo_backup, sizeof(double) * TH_N,
                               cudaMemcpyDeviceToDevice, s));
            if (ctx->nhc_on)
                CK(cudaMemcpyAsync(ctx->nhc, ctx->nhc_backup, sizeof(double) * NHC_N,
                                   cudaMemcpyDeviceToDevice, s));
            CK(cudaStreamSynchronize(s));
            rc = ensure_atoms(ctx, (int)n, grown_capacity(ctx->h_status[1]));
            if (rc) return rc;
            force_rebuild = true;
            continue;
        }
        if (ctx->timing) {
            rc = collect_timing(ctx, len);
            if (rc) return rc;
        }
        if (ctx->h_status[0] & ST_NONFINITE)
            return fail(ctx, NEP_ERR_NONFINITE, "non-finite values during MD");
        done += len;
    }
    const double* th2 = ctx->h_result + NPART;
    st->time = th2[TH_TIME];
    st->step = (int64_t)llround(th2[TH_STEP]);
    st->dt_last = th2[TH_DTLAST];
    st->kinetic_energy = th2[TH_KE];
    st->thermostat_energy = ctx->nhc_on ? th2[TH_ENHC] : 0.0;
    if (n_steps > 0) {
        st->potential_energy = ctx->h_result[0];
        for (int t = 0; t < 9; ++t) st->virial[t] = ctx->h_result[1 + t];
    }
    return NEP_OK;
}

}  // extern "C"

// Device mirror of an MD state (x, v, F, species) owned by the context: the
// device side of md_step_host and the scratch state of nep_md_autotune.
static int ensure_mirror(nep_ctx* ctx, int64_t n)
{
    if (n <= ctx->hm_cap) return NEP_OK;
    cudaDeviceSynchronize();
    drop_graphs(ctx);   // graphs hold the old mirror's addresses
    free_dev(ctx->hm_x); free_dev(ctx->hm_v); free_dev(ctx->hm_f); free_dev(ctx->hm_t);
    ctx->hm_cap = 0;
    CK(cudaMalloc(&ctx->hm_x, sizeof(double) * 3 * (size_t)n));
    CK(cudaMalloc(&ctx->hm_v, sizeof(double) * 3 * (size_t)n));
    CK(cudaMalloc(&ctx->hm_f, sizeof(double) * 3 * (size_t)n));
    CK(cudaMalloc(&ctx->hm_t, sizeof(int32_t) * (size_t)n));
    ctx->hm_cap = n;
    return NEP_OK;
}

extern "C" {

int md_step_host(nep_ctx* ctx, nep_md_state* st, int n_steps, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (!st || n_steps < 0) return fail(ctx, NEP_ERR_INVALID_ARG, "bad state or step count");
    const int64_t n = st->n_atoms;
    if (n <= 0 || n >= (1 << 26)) return fail(ctx, NEP_ERR_INVALID_ARG, "n_atoms must be in [1, 2^26)");
    const void* arrays[4] = {st->xyz, st->vel, st->forces, st->types};
    const char* names[4] = {"xyz", "vel", "forces", "types"};
    CK(cudaSetDevice(ctx->device));
    for (int t = 0; t < 4; ++t) {
        if (!arrays[t]) return fail(ctx, NEP_ERR_INVALID_ARG, "%s is NULL", names[t]);
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, arrays[t]) != cudaSuccess) {
            cudaGetLastError();   // plain host memory unknown to CUDA: accepted
        } else if (at.type == cudaMemoryTypeDevice) {
            return fail(ctx, NEP_ERR_INVALID_ARG,
                        "%s is device memory: md_step_host takes host arrays (md_step takes "
                        "device arrays)", names[t]);
        }
    }
    int rc0 = ensure_mirror(ctx, n);
    if (rc0) return rc0;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b3 = sizeof(double) * 3 * (size_t)n;
    CK(cudaMemcpyAsync(ctx->hm_x, st->xyz, b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->hm_v, st->vel, b3, cudaMemcpyHostToDevice, s));
    if (st->forces_valid) CK(cudaMemcpyAsync(ctx->hm_f, st->forces, b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->hm_t, st->types, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    nep_md_state d = *st;
    d.xyz = ctx->hm_x;
    d.vel = ctx->hm_v;
    d.forces = ctx->hm_f;
    d.types = ctx->hm_t;
    int rc = md_step(ctx, &d, n_steps, stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(st->xyz, ctx->hm_x, b3, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(st->vel, ctx->hm_v, b3, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(st->forces, ctx->hm_f, b3, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // outputs of the step (the arrays are the caller's again)
    d.xyz = st->xyz;
    d.vel = st->vel;
    d.forces = st->forces;
    d.types = st->types;
    *st = d;
    return NEP_OK;
}

// Median of a few timings.
static double median_ms(std::vector<float> t)
{
    std::sort(t.begin(), t.end());
    const size_t m = t.size();
    return m == 0 ? 0.0 : (m % 2 ? t[m / 2] : 0.5 * ((double)t[m / 2 - 1] + t[m / 2]));
}

int nep_md_autotune(nep_ctx* ctx, const nep_md_state* st, int reps, void* stream,
                    nep_tune_table* tiling, nep_tune_table* chunk)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (!st) return fail(ctx, NEP_ERR_INVALID_ARG, "NULL state");
    const int64_t n = st->n_atoms;
    if (n <= 0 || n >= (1 << 26)) return fail(ctx, NEP_ERR_INVALID_ARG, "n_atoms must be in [1, 2^26)");
    if (reps < 1 || reps > 50) return fail(ctx, NEP_ERR_INVALID_ARG, "reps must be in [1, 50]");
    int rc;
    if ((rc = check_device_ptr(ctx, st->xyz, "xyz")) || (rc = check_device_ptr(ctx, st->vel, "vel")) ||
        (rc = check_device_ptr(ctx, st->forces, "forces")) ||
        (rc = check_device_ptr(ctx, st->types, "types")))
        return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_mirror(ctx, n))) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    nep_tune_table tt;
    memset(&tt, 0, sizeof(tt));
    // 1. neighbour-search tiling: force evaluations of the state's positions
    //    (forces into the context's scratch state)
    const int zss[4] = {1, 2, 4, 8}, chws[3] = {4, 8, 16};
    const int zs0 = ctx->nbr_zs, chw0 = ctx->nbr_chw;
    double best = 1e300;
    int bz = zs0, bc = chw0;
    for (int a = 0; a < 4 && !rc; ++a)
        for (int b = 0; b < 3 && !rc; ++b) {
            ctx->nbr_zs = zss[a];
            ctx->nbr_chw = chws[b];
            Grid g;
            if ((rc = make_grid(ctx, n, st->box, st->pbc, g))) break;
            if (g.tric && (a > 0 || b != 2)) continue;   // triclinic: one kernel
            if ((rc = compute_with_retry(ctx, g, st->xyz, st->types, ctx->hm_f, nullptr, s))) break;
            std::vector<float> t;
            for (int r = 0; r < reps && !rc; ++r) {
                CK(cudaEventRecord(e0, s));
                rc = eval(ctx, g, st->xyz, st->types, ctx->hm_f, nullptr, s, -1);
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                t.push_back(ms);
            }
            if (rc) break;
            CK(cudaStreamSynchronize(s));
            CK(cudaMemcpy(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
            if (ctx->h_status[0] & ST_OVERFLOW) continue;   // capacity grew meanwhile
            const double m = median_ms(t);
            if (tt.n < 32) {
                tt.a[tt.n] = zss[a]; tt.b[tt.n] = chws[b]; tt.ms[tt.n] = m;
                if (m < best) { best = m; bz = zss[a]; bc = chws[b]; tt.best = tt.n; }
                ++tt.n;
            }
        }
    ctx->nbr_zs = rc ? zs0 : bz;
    ctx->nbr_chw = rc ? chw0 : bc;
    drop_graphs(ctx);
    if (tiling) *tiling = tt;
    // 2. steps per captured graph: 50 MD steps of a copy of the state for
    //    each candidate (NVE only: a thermostat or barostat keeps its state in
    //    the context, which trial steps would advance)
    nep_tune_table tc;
    memset(&tc, 0, sizeof(tc));
    if (!rc && !ctx->nhc_on && !ctx->baro_on) {
        const int chunks[3] = {10, 25, 50};
        const int chunk0 = ctx->chunk;
        const size_t b3 = sizeof(double) * 3 * (size_t)n;
        double bestc = 1e300;
        int bch = chunk0;
        for (int c = 0; c < 3 && !rc; ++c) {
            ctx->chunk = chunks[c];
            nep_md_state d = *st;
            d.xyz = ctx->hm_x; d.vel = ctx->hm_v; d.forces = ctx->hm_f; d.types = ctx->hm_t;
            std::vector<float> t;
            for (int r = 0; r <= reps && !rc; ++r) {   // r = 0: capture (not timed)
                CK(cudaMemcpyAsync(ctx->hm_x, st->xyz, b3, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(ctx->hm_v, st->vel, b3, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(ctx->hm_f, st->forces, b3, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(ctx->hm_t, st->types, sizeof(int32_t) * (size_t)n,
                                   cudaMemcpyDeviceToDevice, s));
                nep_md_state d2 = d;
                CK(cudaEventRecord(e0, s));
                rc = md_step(ctx, &d2, 50, stream);
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (r > 0) t.push_back(ms / 50.0f);
            }
            if (rc) break;
            const double m = median_ms(t);
            tc.a[tc.n] = chunks[c]; tc.b[tc.n] = 0; tc.ms[tc.n] = m;
            if (m < bestc) { bestc = m; bch = chunks[c]; tc.best = tc.n; }
            ++tc.n;
        }
        ctx->chunk = rc ? chunk0 : bch;
        drop_graphs(ctx);
    }
    if (chunk) *chunk = tc;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"

// ============================================================================
// Batches of small periodic configurations
// ============================================================================

// Grows a device buffer to at least `bytes`.
static int grow(nep_ctx* ctx, void** p, size_t& cap, size_t bytes, cudaStream_t s)
{
    if (bytes <= cap && *p) return NEP_OK;
    CK(cudaStreamSynchronize(s));
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    CK(cudaMalloc(p, bytes));
    cap = bytes;
    return NEP_OK;
}

static int batch_buffers(nep_ctx* ctx, long long ntot, int S, int M)
{
    if (ntot <= ctx->b_ntot_cap && S <= ctx->b_S_cap && M <= ctx->b_M && ctx->b_nbr) return NEP_OK;
    cudaDeviceSynchronize();
    const long long nc = std::max(ntot, ctx->b_ntot_cap);
    const int Sc = std::max(S, ctx->b_S_cap);
    const int Mc = std::max(M, ctx->b_M);
    free_batch(ctx);
    const size_t rsz = ctx->precision == NEP_FP32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&ctx->b_nbr, sizeof(int) * (size_t)nc * Mc));
    CK(cudaMalloc(&ctx->b_cnt, sizeof(int2) * (size_t)nc));
    CK(cudaMalloc(&ctx->b_scr, rsz * (size_t)nc * BSTRIDE));
    CK(cudaMalloc(&ctx->b_F, sizeof(double) * 3 * (size_t)nc));
    CK(cudaMalloc(&ctx->b_gpart, sizeof(double) * (size_t)Sc * n_params_for(ctx->ntypes)));
    CK(cudaMalloc(&ctx->b_lpart, sizeof(double) * 3 * (size_t)Sc));
    CK(cudaMalloc(&ctx->b_E, sizeof(double) * (size_t)Sc));
    CK(cudaMalloc(&ctx->b_W, sizeof(double) * 9 * (size_t)Sc));
    CK(cudaMalloc(&ctx->b_off, sizeof(long long) * (size_t)(Sc + 1)));
    CK(cudaMalloc(&ctx->b_order, sizeof(int) * (size_t)Sc));
    CK(cudaMalloc(&ctx->b_box, sizeof(double) * 3 * (size_t)Sc));
    CK(cudaMalloc(&ctx->b_queue, sizeof(int)));
    ctx->b_ntot_cap = nc;
    ctx->b_S_cap = Sc;
    ctx->b_M = Mc;
    return NEP_OK;
}

// Validates a batch, uploads its offsets/boxes/order and fills b.
static int batch_prepare(nep_ctx* ctx, const nep_batch* bt, cudaStream_t s, Batch& b)
{
    if (!bt || bt->n_configs < 1 || !bt->offsets || !bt->boxes)
        return fail(ctx, NEP_ERR_INVALID_ARG, "batch needs n_configs >= 1, offsets and boxes");
    const int S = bt->n_configs;
    if (bt->offsets[0] != 0 || bt->offsets[S] != bt->n_atoms || bt->n_atoms >= (1LL << 31))
        return fail(ctx, NEP_ERR_INVALID_ARG, "offsets must start at 0 and end at n_atoms");
    std::vector<int> order(S);
    for (int c = 0; c < S; ++c) {
        const long long n = bt->offsets[c + 1] - bt->offsets[c];
        if (n < 1 || n > BMAXA)
            return fail(ctx, NEP_ERR_INVALID_ARG, "configuration %d has %lld atoms (1..%d)", c, n,
                        BMAXA);
        for (int a = 0; a < 3; ++a) {
            const double L = bt->boxes[3 * c + a];
            if (!(L >= ctx->rcR) || !isfinite(L))
                return fail(ctx, NEP_ERR_BOX, "configuration %d: box length %g < r_c^R", c, L);
        }
        order[c] = c;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return bt->offsets[a + 1] - bt->offsets[a] > bt->offsets[c + 1] - bt->offsets[c];
    });
    int rc;
    if ((rc = check_device_ptr(ctx, bt->xyz, "batch xyz"))) return rc;
    if (ctx->ntypes > 1 && (rc = check_device_ptr(ctx, bt->types, "batch types"))) return rc;
    int M = ctx->b_M > 0 ? ctx->b_M : 112;
    if ((rc = batch_buffers(ctx, bt->n_atoms, S, M))) return rc;
    std::vector<long long> off(bt->offsets, bt->offsets + S + 1);
    CK(cudaMemcpyAsync(ctx->b_off, off.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->b_box, bt->boxes, sizeof(double) * 3 * S, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->b_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    memset(&b, 0, sizeof(b));
    b.S = S;
    b.ntot = bt->n_atoms;
    b.off = ctx->b_off;
    b.order = ctx->b_order;
    b.box = ctx->b_box;
    b.x = bt->xyz;
    b.queue = ctx->b_queue;
    b.status = ctx->status;
    b.lpart = ctx->b_lpart;
    b.gpart = ctx->b_gpart;
    b.T = ctx->ntypes;
    b.np = (int)n_params_for(ctx->ntypes);
    b.types = bt->types;
    if (ctx->precision == NEP_FP32) b.coef = ctx->coef_f;
    else b.coef = ctx->coef_d;
    return NEP_OK;
}

// Runs one batched launch (with neighbour-capacity growth) and waits.
// uE, uF, uW: the caller's outputs, or nullptr for the context's scratch
// (re-pointed after a reallocation).
static int batch_launch(nep_ctx* ctx, Batch& b, int mode, double* grad, cudaStream_t s,
                        double* uE = nullptr, double* uF = nullptr, double* uW = nullptr)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int bt = ctx->precision == NEP_FP32 ? ctx->b_bt : 128;
    for (int attempt = 0; attempt < 4; ++attempt) {
        b.M = ctx->b_M;
        b.nbr = ctx->b_nbr;
        b.cnt = ctx->b_cnt;
        b.scr = ctx->b_scr;
        b.gpart = ctx->b_gpart;
        b.lpart = ctx->b_lpart;
        b.off = ctx->b_off;
        b.order = ctx->b_order;
        b.box = ctx->b_box;
        b.queue = ctx->b_queue;
        b.E = uE ? uE : ctx->b_E;
        b.F = uF ? uF : ctx->b_F;
        b.W = uW ? uW : ctx->b_W;
        int per_sm = ctx->b_per_sm > 0 ? ctx->b_per_sm
                                        : batch_blocks_per_sm(ctx->precision, mode, bt);
        int grid = std::min(b.S, std::max(1, per_sm * sms));
        CK(cudaMemsetAsync(ctx->b_queue, 0, sizeof(int), s));
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(int) * NSTATUS, s));
        CK(launch_batch(ctx->precision, mode, bt, grid, ctx->mf, ctx->md, b, grad, s));
        ctx->launches += (mode == MODE_BACKWARD || mode == MODE_LOSS) ? 2 : 1;
        CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int) * NSTATUS, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (ctx->h_status[0] & ST_OVERFLOW) {
            // keep the batch description: reallocation must not lose offsets/boxes/order
            std::vector<long long> off(b.S + 1);
            std::vector<double> box(3 * (size_t)b.S);
            std::vector<int> order(b.S);
            CK(cudaMemcpy(off.data(), ctx->b_off, sizeof(long long) * (b.S + 1), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(box.data(), ctx->b_box, sizeof(double) * 3 * b.S, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(order.data(), ctx->b_order, sizeof(int) * b.S, cudaMemcpyDeviceToHost));
            const int need = grown_capacity(ctx->h_status[1]);
            int rc = batch_buffers(ctx, b.ntot, b.S, need);
            if (rc) return rc;
            CK(cudaMemcpy(ctx->b_off, off.data(), sizeof(long long) * (b.S + 1), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(ctx->b_box, box.data(), sizeof(double) * 3 * b.S, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(ctx->b_order, order.data(), sizeof(int) * b.S, cudaMemcpyHostToDevice));
            continue;
        }
        if (ctx->h_status[0] & ST_BADTYPE)
            return fail(ctx, NEP_ERR_INVALID_ARG, "species index out of range [0, %d)",
                        ctx->ntypes);
        if (ctx->h_status[0] & ST_NONFINITE)
            return fail(ctx, NEP_ERR_NONFINITE, "non-finite values in the batch");
        return NEP_OK;
    }
    return fail(ctx, NEP_ERR_NBR_OVERFLOW, "neighbour capacity could not be grown enough");
}

extern "C" {

int nep_set_params(nep_ctx* ctx, const double* params, int64_t n_params)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    const int64_t np = n_params_for(ctx->ntypes);
    if (!params || n_params != np)
        return fail(ctx, NEP_ERR_INVALID_ARG, "params must hold %lld values", (long long)np);
    for (int64_t i = 0; i < np; ++i)
        if (!isfinite(params[i])) return fail(ctx, NEP_ERR_INVALID_ARG, "non-finite parameter");
    // rebuild both models (and pair tables) from the new parameters and the
    // stored hyperparameters and scaler; graphs hold the old model by value
    CK(cudaDeviceSynchronize());
    int rc = setup_model(ctx, params);
    if (rc) return rc;
    drop_graphs(ctx);
    return NEP_OK;
}

int nep_batch_forward(nep_ctx* ctx, const nep_batch* batch, double* energies, double* forces,
                      double* virials, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = check_device_ptr(ctx, energies, "energies")) ||
        (rc = check_device_ptr(ctx, forces, "forces")))
        return rc;
    if (virials && (rc = check_device_ptr(ctx, virials, "virials"))) return rc;
    Batch b;
    if ((rc = batch_prepare(ctx, batch, s, b))) return rc;
    return batch_launch(ctx, b, MODE_FORWARD, nullptr, s, energies, forces, virials);
}

int nep_batch_backward(nep_ctx* ctx, const nep_batch* batch, const double* dL_dE,
                       const double* dL_dF, const double* dL_dW, double* grad, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = check_device_ptr(ctx, dL_dE, "dL_dE")) || (rc = check_device_ptr(ctx, dL_dF, "dL_dF")) ||
        (rc = check_device_ptr(ctx, grad, "grad")))
        return rc;
    if (dL_dW && (rc = check_device_ptr(ctx, dL_dW, "dL_dW"))) return rc;
    Batch b;
    if ((rc = batch_prepare(ctx, batch, s, b))) return rc;
    b.dLdE = dL_dE;
    b.dLdF = dL_dF;
    b.dLdW = dL_dW;
    return batch_launch(ctx, b, MODE_BACKWARD, grad, s);
}

// Uploads the has-virial mask (all ones when NULL) and returns how many
// configurations have a virial target.
static int upload_virial_mask(nep_ctx* ctx, const nep_targets* t, int S, cudaStream_t s, int* nv)
{
    *nv = 0;
    if (!t->virial) return NEP_OK;
    int rc = check_device_ptr(ctx, t->virial, "virial targets");
    if (rc) return rc;
    if (S > ctx->b_hv_cap) {
        CK(cudaStreamSynchronize(s));
        free_dev(ctx->b_hv);
        CK(cudaMalloc(&ctx->b_hv, (size_t)S));
        ctx->b_hv_cap = S;
    }
    std::vector<unsigned char> hv(S);
    for (int c = 0; c < S; ++c) {
        hv[c] = t->has_virial ? (t->has_virial[c] ? 1 : 0) : 1;
        *nv += hv[c];
    }
    CK(cudaMemcpyAsync(ctx->b_hv, hv.data(), (size_t)S, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return NEP_OK;
}

int nep_batch_loss_grad(nep_ctx* ctx, const nep_batch* batch, const nep_targets* t,
                        const nep_loss_weights* w, double* loss, double* grad, double* energies,
                        double* forces, double* virials, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (!loss || !t || !w) return fail(ctx, NEP_ERR_INVALID_ARG, "loss, targets or weights is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = check_device_ptr(ctx, t->energy, "energy targets")) ||
        (rc = check_device_ptr(ctx, t->forces, "force targets")) ||
        (rc = check_device_ptr(ctx, grad, "grad")))
        return rc;
    if (energies && (rc = check_device_ptr(ctx, energies, "energies"))) return rc;
    if (forces && (rc = check_device_ptr(ctx, forces, "forces"))) return rc;
    if (virials && (rc = check_device_ptr(ctx, virials, "virials"))) return rc;
    Batch b;
    if ((rc = batch_prepare(ctx, batch, s, b))) return rc;
    int nv = 0;
    if ((rc = upload_virial_mask(ctx, t, b.S, s, &nv))) return rc;
    b.Et = t->energy;
    b.Ft = t->forces;
    b.Wt = nv > 0 ? t->virial : nullptr;
    b.hv = ctx->b_hv;
    b.nv = nv;
    b.we = w->energy;
    b.wf = w->force;
    b.wv = w->virial;
    if ((rc = batch_launch(ctx, b, MODE_LOSS, grad, s, energies, forces, virials))) return rc;
    std::vector<double> lp(3 * (size_t)b.S);
    CK(cudaMemcpy(lp.data(), ctx->b_lpart, sizeof(double) * 3 * b.S, cudaMemcpyDeviceToHost));
    double terms[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < b.S; ++c)
        for (int k = 0; k < 3; ++k) terms[k] += lp[3 * (size_t)c + k];
    loss[0] = terms[0] + terms[1] + terms[2];
    loss[1] = terms[0];
    loss[2] = terms[1];
    loss[3] = terms[2];
    return NEP_OK;
}

int nep_batch_autotune(nep_ctx* ctx, const nep_batch* batch, const nep_targets* t,
                       const nep_loss_weights* w, void* stream, int* best_threads,
                       int* best_per_sm)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* grad = nullptr;
    CK(cudaMalloc(&grad, sizeof(double) * n_params_for(ctx->ntypes)));
    const int bts[3] = {64, 128, 256};
    const int nbt = ctx->precision == NEP_FP32 ? 3 : 1;
    double best = 1e300;
    int bb = ctx->b_bt, bs = ctx->b_per_sm;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = NEP_OK;
    nep_tune_table tab;
    memset(&tab, 0, sizeof(tab));
    for (int a = 0; a < nbt && !rc; ++a) {
        for (int per = 1; per <= 4 && !rc; per *= 2) {
            ctx->b_bt = ctx->precision == NEP_FP32 ? bts[a] : 128;
            ctx->b_per_sm = per;
            double L[4];
            rc = nep_batch_loss_grad(ctx, batch, t, w, L, grad, nullptr, nullptr, nullptr,
                                     stream);   // warm-up
            if (rc) break;
            // median of three launches (one launch alone is too noisy to rank
            // candidates a few per cent apart)
            std::vector<float> tm;
            for (int r = 0; r < 3 && !rc; ++r) {
                cudaEventRecord(e0, s);
                rc = nep_batch_loss_grad(ctx, batch, t, w, L, grad, nullptr, nullptr, nullptr,
                                         stream);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tm.push_back(ms);
            }
            if (rc) break;
            const double m = median_ms(tm);
            tab.a[tab.n] = ctx->b_bt; tab.b[tab.n] = per; tab.ms[tab.n] = m;
            if (m < best) { best = m; bb = ctx->b_bt; bs = per; tab.best = tab.n; }
            ++tab.n;
        }
    }
    ctx->b_table = tab;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(grad);
    ctx->b_bt = bb;
    ctx->b_per_sm = bs;
    ctx->b_tuned = 1;
    if (best_threads) *best_threads = bb;
    if (best_per_sm) *best_per_sm = bs;
    return rc;
}

int nep_batch_autotune_table(const nep_ctx* ctx, nep_tune_table* out)
{
    if (!ctx || !out) return NEP_ERR_INVALID_ARG;
    *out = ctx->b_table;
    return NEP_OK;
}


// Loss terms of n_pop parameter vectors (device thetas [n_pop][NP]) over the
// batch: one list-building launch, the models, one population launch, one
// loss launch; losses (device) [n_pop][6].
static int population_eval(nep_ctx* ctx, const nep_batch* batch, const nep_targets* t,
                           const nep_loss_weights* w, int n_pop, const double* thetas,
                           double* losses, cudaStream_t s)
{
    int rc;
    if ((rc = check_device_ptr(ctx, t->energy, "energy targets")) ||
        (rc = check_device_ptr(ctx, t->forces, "force targets")))
        return rc;
    Batch b;
    if ((rc = batch_prepare(ctx, batch, s, b))) return rc;
    int nv = 0;
    if ((rc = upload_virial_mask(ctx, t, b.S, s, &nv))) return rc;
    // neighbour lists of every configuration (capacity grows on overflow)
    if ((rc = batch_launch(ctx, b, MODE_LISTS, nullptr, s))) return rc;
    b.Et = t->energy;
    b.Ft = t->forces;
    b.Wt = nv > 0 ? t->virial : nullptr;
    b.hv = ctx->b_hv;
    b.nv = nv;
    if (!ctx->d_scaler) {
        CK(cudaMalloc(&ctx->d_scaler, sizeof(double) * D));
        CK(cudaMemcpy(ctx->d_scaler, ctx->scaler.data(), sizeof(double) * D, cudaMemcpyHostToDevice));
    }
    if ((rc = grow(ctx, &ctx->p_models, ctx->p_models_cap, model_bytes(ctx->precision) * n_pop, s)) ||
        (rc = grow(ctx, (void**)&ctx->p_out, ctx->p_out_cap,
                   sizeof(double) * 3 * (size_t)n_pop * b.S, s)))
        return rc;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long items = (long long)n_pop * b.S;
    const int grid = (int)std::min<long long>(items, (long long)population_blocks_per_sm(ctx->precision) * sms);
    CK(cudaMemsetAsync(ctx->b_queue, 0, sizeof(int), s));
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int) * NSTATUS, s));
    if (b.T > 1) {
        const size_t rsz = ctx->precision == NEP_FP32 ? sizeof(float) : sizeof(double);
        if ((rc = grow(ctx, &ctx->p_tables, ctx->p_tables_cap,
                       rsz * (size_t)b.T * b.T * CSTR * n_pop, s)))
            return rc;
    }
    CK(launch_population(ctx->precision, n_pop, ctx->mf, ctx->md, ctx->d_scaler, thetas,
                         ctx->p_models, ctx->p_tables, b, ctx->p_out, grid, s));
    CK(launch_population_loss(n_pop, ctx->p_out, thetas, b.S, b.ntot, (double)nv, w->energy,
                              w->force, w->virial, w->l1, w->l2, losses, b.np, s));
    ctx->launches += 3;
    CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int) * NSTATUS, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->h_status[0] & ST_BADTYPE)
        return fail(ctx, NEP_ERR_INVALID_ARG, "species index out of range [0, %d)", ctx->ntypes);
    if (ctx->h_status[0] & ST_NONFINITE)
        return fail(ctx, NEP_ERR_NONFINITE, "non-finite values in the population");
    return NEP_OK;
}

static int population_args(nep_ctx* ctx, const nep_targets* t, const nep_loss_weights* w,
                           int n_pop)
{
    if (!t || !w) return fail(ctx, NEP_ERR_INVALID_ARG, "targets or weights is NULL");
    if (n_pop < 1 || n_pop > 1024) return fail(ctx, NEP_ERR_INVALID_ARG, "n_pop must be 1..1024");
    if ((long long)n_pop * n_params_for(ctx->ntypes) > (1LL << 31))
        return fail(ctx, NEP_ERR_INVALID_ARG, "population too large");
    return NEP_OK;
}

int nep_population_loss(nep_ctx* ctx, const nep_batch* batch, const nep_targets* t,
                        const nep_loss_weights* w, int n_pop, const double* thetas,
                        double* losses, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    int rc;
    if ((rc = population_args(ctx, t, w, n_pop))) return rc;
    if ((rc = check_device_ptr(ctx, thetas, "thetas")) || (rc = check_device_ptr(ctx, losses, "losses")))
        return rc;
    return population_eval(ctx, batch, t, w, n_pop, thetas, losses, (cudaStream_t)stream);
}

int nep_snes_generation(nep_ctx* ctx, const nep_batch* batch, const nep_targets* t,
                        const nep_loss_weights* w, int n_pop, double* mu, double* sigma,
                        const double* samples, double eta_mu, double eta_sigma, double* losses,
                        void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    int rc;
    if ((rc = population_args(ctx, t, w, n_pop))) return rc;
    if ((rc = check_device_ptr(ctx, mu, "mu")) || (rc = check_device_ptr(ctx, sigma, "sigma")) ||
        (rc = check_device_ptr(ctx, samples, "samples")) ||
        (rc = check_device_ptr(ctx, losses, "losses")))
        return rc;
    if (!isfinite(eta_mu) || !isfinite(eta_sigma))
        return fail(ctx, NEP_ERR_INVALID_ARG, "learning rates must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = (int)n_params_for(ctx->ntypes);
    if ((rc = grow(ctx, (void**)&ctx->p_thetas, ctx->p_thetas_cap,
                   sizeof(double) * np * (size_t)n_pop, s)))
        return rc;
    if (!ctx->p_util) CK(cudaMalloc(&ctx->p_util, sizeof(double) * 1024));
    CK(launch_snes_sample(mu, sigma, samples, n_pop, np, ctx->p_thetas, s));
    ctx->launches += 1;
    if ((rc = population_eval(ctx, batch, t, w, n_pop, ctx->p_thetas, losses, s))) return rc;
    CK(launch_snes_update(mu, sigma, samples, losses, ctx->p_util, n_pop, np, eta_mu, eta_sigma,
                          s));
    ctx->launches += 2;
    CK(cudaStreamSynchronize(s));
    return NEP_OK;
}

}  // extern "C"

// ============================================================================
// Force evaluation without any allocation: scratch in a fixed device array
// ============================================================================
//
// For callers that cannot call cudaMalloc at the point where they need forces
// (for example a plugin inside a host program whose device memory is all owned
// by the host's own pool or fixed budget, so that components may not allocate
// behind its back).  All scratch of one FP32 evaluation
// lives in g_static_scratch below, a file-scope __device__ array that every GPU
// loading this library holds until the process exits.

namespace {

constexpr int ST_MAX_ATOMS = 8192;   // largest system of the fixed-scratch path
constexpr int ST_SLOTS = 96;         // neighbour slots per atom
constexpr int ST_MAX_CELLS = 8192;   // largest cell grid
constexpr int ST_TILES = (ST_MAX_ATOMS + TILE - 1) / TILE;

constexpr size_t st_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t ST_OFF_CELL_OF = 0;
constexpr size_t ST_OFF_SLOT_OF = ST_OFF_CELL_OF + st_align(sizeof(int) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_PERM = ST_OFF_SLOT_OF + st_align(sizeof(int) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_CELL_SORTED = ST_OFF_PERM + st_align(sizeof(int) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_POS4 = ST_OFF_CELL_SORTED + st_align(sizeof(int) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_CNT = ST_OFF_POS4 + st_align(sizeof(float4) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_NBR = ST_OFF_CNT + st_align(sizeof(int2) * ST_MAX_ATOMS);
constexpr size_t ST_OFF_FACC = ST_OFF_NBR + st_align(sizeof(int) * (size_t)ST_MAX_ATOMS * ST_SLOTS);
constexpr size_t ST_OFF_PART = ST_OFF_FACC + st_align(sizeof(long long) * 3 * ST_MAX_ATOMS);
constexpr size_t ST_OFF_PART2 = ST_OFF_PART + st_align(sizeof(double) * NPART * ST_TILES);
constexpr size_t ST_OFF_COUNT = ST_OFF_PART2 + st_align(sizeof(double) * NPART * RED1_MAX);
constexpr size_t ST_OFF_START = ST_OFF_COUNT + st_align(sizeof(int) * (ST_MAX_CELLS + 1));
constexpr size_t ST_OFF_SCAN = ST_OFF_START + st_align(sizeof(int) * (ST_MAX_CELLS + 1));
constexpr size_t ST_OFF_RESULT = ST_OFF_SCAN + st_align(sizeof(int) * SCAN_B);
constexpr size_t ST_OFF_STATUS = ST_OFF_RESULT + st_align(sizeof(double) * NPART);
constexpr size_t ST_OFF_PAIRS = ST_OFF_STATUS + st_align(sizeof(int) * 3);
constexpr size_t ST_BYTES = ST_OFF_PAIRS + st_align(sizeof(unsigned long long) * 2);

constexpr int ST_MAX_DEVICES = 64;
std::mutex g_static_mutex;
unsigned char* g_static_ptr[ST_MAX_DEVICES] = {nullptr};

}  // namespace

// About 3.8 MB.  Host code must not use this name as an address: the device
// address comes from cudaGetSymbolAddress (static_scratch_address below).
static __device__ __align__(256) unsigned char g_static_scratch[ST_BYTES];

// Device address of g_static_scratch on the current device; looked up once per
// device (first call on that device) and cached.
static int static_scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(nullptr, NEP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= ST_MAX_DEVICES)
        return fail(nullptr, NEP_ERR_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, NEP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_static_ptr[dev] = (unsigned char*)p;
    }
    *out = g_static_ptr[dev];
    return NEP_OK;
}

extern "C" int nep_compute_static(const nep_params* p, int64_t n_atoms, const double* xyz,
                                  const double box[9], const int32_t* types,
                                  const int32_t pbc[3], double* energy, double* forces,
                                  double* virial, double* site_energy, void* stream)
{
    nep_ctx* ctx = nullptr;   // errors go to nep_last_error(NULL)
    if (!p || !box || !pbc || !energy) return fail(nullptr, NEP_ERR_INVALID_ARG, "NULL argument");
    if (n_atoms < 0 || n_atoms > ST_MAX_ATOMS)
        return fail(nullptr, NEP_ERR_INVALID_ARG,
                    "nep_compute_static handles at most %d atoms (got %lld)", ST_MAX_ATOMS,
                    (long long)n_atoms);
    if (p->n_types != 1 || p->n_max_radial != NR - 1 || p->n_max_angular != NA - 1 ||
        p->basis_size_radial != KR - 1 || p->basis_size_angular != KA - 1 || p->l_max != LM ||
        p->use_4body != 1 || p->n_hidden != H)
        return fail(nullptr, NEP_ERR_UNSUPPORTED, "model sizes not supported by this build");
    const int64_t np = (int64_t)H * D + 2 * H + 1 + NR * KR + NA * KA;
    if (!p->params || p->n_params != np || !p->q_scaler)
        return fail(nullptr, NEP_ERR_INVALID_ARG, "params must hold %lld values and a scaler",
                    (long long)np);
    if (!(p->rc_radial > 0) || !(p->rc_angular > 0) || p->rc_angular > p->rc_radial ||
        !(p->zbl_r_outer > p->zbl_r_inner) || p->zbl_r_outer > p->rc_angular || !(p->z[0] > 0))
        return fail(nullptr, NEP_ERR_INVALID_ARG, "bad cutoffs or nuclear charge");
    // cell grid (diagonal box; periodic dims need >= 3 cells of >= rc_R)
    Grid g;
    memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && box[3 * a + b] != 0.0)
                return fail(nullptr, NEP_ERR_BOX, "only diagonal boxes are supported");
    for (int a = 0; a < 3; ++a) {
        const double L = box[4 * a];
        if (!(L > 0.0) || !isfinite(L)) return fail(nullptr, NEP_ERR_BOX, "box length %g", L);
        int nc = (int)floor(L / p->rc_radial);
        if (pbc[a] && nc < 3) return fail(nullptr, NEP_ERR_BOX, "periodic box shorter than 3 r_c");
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        g.nc[a] = nc;
        g.pbc[a] = pbc[a] ? 1 : 0;
        g.lc[a] = L / nc;
        g.inv_lc[a] = nc / L;
        g.L[a] = L;
        g.invL[a] = 1.0 / L;
    }
    const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
    if (ncell > ST_MAX_CELLS)
        return fail(nullptr, NEP_ERR_BOX, "cell grid of %d cells exceeds %d", ncell, ST_MAX_CELLS);
    const int n = (int)n_atoms;
    g.n = n;
    g.ld = ST_MAX_ATOMS;
    g.M = ST_SLOTS;
    g.ntypes = 1;
    g.zs = 1;
    if (n == 0) {
        *energy = 0.0;
        if (virial) for (int t = 0; t < 9; ++t) virial[t] = 0.0;
        return NEP_OK;
    }
    // site_energy is optional; when given, the kernels store to it, so it is
    // checked like the required arrays
    const void* dev_args[4] = {xyz, types, forces, site_energy};
    const char* dev_names[4] = {"xyz", "types", "forces", "site_energy"};
    for (int a = 0; a < 4; ++a) {
        const void* q = dev_args[a];
        if (a == 3 && !q) continue;
        cudaPointerAttributes at;
        if (!q || cudaPointerGetAttributes(&at, q) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(nullptr, NEP_ERR_INVALID_ARG,
                        "%s must be device memory (inputs and outputs are device arrays)",
                        dev_names[a]);
        }
    }
    unsigned char* base = nullptr;
    int rc = static_scratch_address(&base);
    if (rc) return rc;
    int* cell_of = (int*)(base + ST_OFF_CELL_OF);
    int* slot_of = (int*)(base + ST_OFF_SLOT_OF);
    int* perm = (int*)(base + ST_OFF_PERM);
    int* cell_sorted = (int*)(base + ST_OFF_CELL_SORTED);
    float4* pos4 = (float4*)(base + ST_OFF_POS4);
    int2* cnt = (int2*)(base + ST_OFF_CNT);
    int* nbr = (int*)(base + ST_OFF_NBR);
    long long* facc = (long long*)(base + ST_OFF_FACC);
    double* partials = (double*)(base + ST_OFF_PART);
    double* partials2 = (double*)(base + ST_OFF_PART2);
    int* count = (int*)(base + ST_OFF_COUNT);
    int* start = (int*)(base + ST_OFF_START);
    int* scan_sums = (int*)(base + ST_OFF_SCAN);
    double* result = (double*)(base + ST_OFF_RESULT);
    int* status = (int*)(base + ST_OFF_STATUS);
    unsigned long long* pairs = (unsigned long long*)(base + ST_OFF_PAIRS);

    Model<float> P;
    build_model<float>(P, p);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear what must start at zero
    CK(cudaMemsetAsync(facc, 0, sizeof(long long) * 3 * ST_MAX_ATOMS, s));
    CK(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(ncell + 1), s));
    CK(cudaMemsetAsync(status, 0, sizeof(int) * 3, s));
    CK(cudaMemsetAsync(pairs, 0, sizeof(unsigned long long) * 2, s));
    const int tb = 256, nb = (n + tb - 1) / tb;
    k_bin_count<float><<<nb, tb, 0, s>>>(g, xyz, cell_of, slot_of, count, status);
    const int sb = (ncell + SCAN_B - 1) / SCAN_B;
    k_scan_blocks<<<sb, SCAN_T, 0, s>>>(count, ncell, start, scan_sums);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(scan_sums, sb, start, ncell);
    k_scan_add<<<(ncell + tb - 1) / tb, tb, 0, s>>>(start, ncell, scan_sums);
    k_bin_scatter<<<nb, tb, 0, s>>>(n, cell_of, slot_of, start, perm);
    k_cell_finalize<float><<<(ncell + 127) / 128, 128, 0, s>>>(g, ncell, start, perm, xyz, types,
                                                              pos4, cell_sorted, status);
    k_neighbors<float, false><<<(n + 127) / 128, 128, 0, s>>>(g, P.rcR2, P.rcA2, pos4, cell_sorted,
                                                             start, nbr, cnt, status, status + 1,
                                                             pairs, nullptr, RadCoef<float>{},
                                                             nullptr, perm, xyz);
    const int tiles = (n + TILE - 1) / TILE;
    k_nep<float><<<tiles, TILE, 0, s>>>(P, g, pos4, nbr, cnt, perm, xyz, facc, partials,
                                        site_energy, status, 0);
    k_forces_out<float><<<nb, tb, 0, s>>>(n, ST_MAX_ATOMS, perm, facc, forces, status);
    k_reduce_stage1<<<1, 256, 0, s>>>(partials, tiles, tiles, partials2);
    k_reduce_partials<<<1, 256, 0, s>>>(partials2, 1, result);
    CK(cudaGetLastError());
    int st[3];
    double res[NPART];
    CK(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(res, result, sizeof(res), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st[0] & ST_OVERFLOW)
        return fail(nullptr, NEP_ERR_NBR_OVERFLOW,
                    "an atom has %d neighbours within r_c; this path holds %d", st[1], ST_SLOTS);
    if (st[0] & ST_BADTYPE)
        return fail(nullptr, NEP_ERR_INVALID_ARG, "species index out of range (one species)");
    if (st[0] & ST_NONFINITE)
        return fail(nullptr, NEP_ERR_NONFINITE, "non-finite positions, energies or forces");
    *energy = res[0];
    if (virial) for (int t = 0; t < 9; ++t) virial[t] = res[1 + t];
    return NEP_OK;
}

// ============================================================================
// Cascade protocol pieces: thermostat, barostat, PKA launch
// ============================================================================

extern "C" {

int nep_set_thermostat(nep_ctx* ctx, const nep_thermostat* t)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    drop_graphs(ctx);
    if (!t) {
        ctx->nhc_on = 0;
        return NEP_OK;
    }
    if (!(t->temperature > 0) || !(t->tau > 0) || !isfinite(t->temperature) || !isfinite(t->tau) ||
        t->chain_length < 1 || t->chain_length > NHC_MAX)
        return fail(ctx, NEP_ERR_INVALID_ARG, "thermostat needs T > 0, tau > 0, chain 1..%d",
                    NHC_MAX);
    int rc;
    if (t->group && (rc = check_device_ptr(ctx, t->group, "thermostat group"))) return rc;
    if (!ctx->nhc) {
        CK(cudaMalloc(&ctx->nhc, sizeof(double) * NHC_N));
        CK(cudaMalloc(&ctx->nhc_backup, sizeof(double) * NHC_N));
    }
    CK(cudaMemset(ctx->nhc, 0, sizeof(double) * NHC_N));   // chain at rest
    ctx->nhc_p.M = t->chain_length;
    ctx->nhc_p.kT = KB_EV * t->temperature;
    ctx->nhc_p.tau2 = t->tau * t->tau;
    ctx->nhc_group = t->group;
    ctx->nhc_counted = -1;
    ctx->nhc_on = 1;
    return NEP_OK;
}

int nep_set_barostat(nep_ctx* ctx, const nep_barostat* b)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    drop_graphs(ctx);
    if (!b) {
        ctx->baro_on = 0;
        return NEP_OK;
    }
    if (!isfinite(b->pressure) || !(b->tau > 0) || !isfinite(b->tau) ||
        !(b->compressibility >= 0) || !isfinite(b->compressibility))
        return fail(ctx, NEP_ERR_INVALID_ARG, "barostat needs a finite pressure, tau > 0, "
                                              "compressibility >= 0");
    if (!ctx->d_box) CK(cudaMalloc(&ctx->d_box, sizeof(double) * 3));
    ctx->baro_p0 = b->pressure / EV_A3_GPA;
    ctx->baro_tau = b->tau;
    ctx->baro_beta = b->compressibility * EV_A3_GPA;
    ctx->baro_on = 1;
    return NEP_OK;
}

int nep_pka(nep_ctx* ctx, nep_md_state* st, const double point[3], double energy,
            const double direction[3], int64_t* atom, void* stream)
{
    if (!ctx) return NEP_ERR_INVALID_ARG;
    if (!st || !point || !direction || !atom) return fail(ctx, NEP_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = st->n_atoms;
    if (n <= 0 || n >= (1 << 26)) return fail(ctx, NEP_ERR_INVALID_ARG, "n_atoms must be in [1, 2^26)");
    const double un = sqrt(direction[0] * direction[0] + direction[1] * direction[1] +
                           direction[2] * direction[2]);
    if (!(energy >= 0) || !isfinite(energy) || !(un > 0) || !isfinite(un))
        return fail(ctx, NEP_ERR_INVALID_ARG, "PKA needs energy >= 0 and a nonzero direction");
    int rc;
    if ((rc = check_device_ptr(ctx, st->xyz, "xyz")) || (rc = check_device_ptr(ctx, st->vel, "vel")) ||
        (rc = check_device_ptr(ctx, st->types, "types")))
        return rc;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(point[a])) return fail(ctx, NEP_ERR_INVALID_ARG, "bad point");
    cudaStream_t s = (cudaStream_t)stream;
    const int tb = 256, nb = (int)((n + tb - 1) / tb);
    const size_t need = sizeof(double) * 2 * (size_t)nb;
    if (need > ctx->pka_cap) {
        CK(cudaStreamSynchronize(s));
        free_dev(ctx->pka_part);
        CK(cudaMalloc(&ctx->pka_part, need));
        ctx->pka_cap = need;
    }
    if (!ctx->pka_atom) CK(cudaMalloc(&ctx->pka_atom, sizeof(long long)));
    Grid gp;
    if ((rc = make_grid(ctx, n, st->box, st->pbc, gp))) return rc;
    k_nearest<<<nb, tb, 0, s>>>((int)n, st->xyz, make_double3(point[0], point[1], point[2]), gp,
                                ctx->pka_part);
    k_pka_set<<<1, 32, 0, s>>>(ctx->pka_part, nb, (int)n, ctx->mt, st->types, energy,
                               make_double3(direction[0] / un, direction[1] / un, direction[2] / un),
                               EV_AMU, st->vel, ctx->pka_atom);
    ctx->launches += 2;
    CK(cudaGetLastError());
    long long a = 0;
    CK(cudaMemcpyAsync(&a, ctx->pka_atom, sizeof(a), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *atom = a;
    return NEP_OK;
}

}  // extern "C"
