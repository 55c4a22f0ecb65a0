/*
 * nepzbl.h -- C ABI of the GB300 NEP-ZBL library (libnepzbl.so).
 *
 * The library evaluates the NEP-ZBL potential of arXiv:2305.08140 and runs
 * velocity-Verlet molecular dynamics with it on one NVIDIA GPU (sm_103a):
 *
 *   E = sum_i U_i,  U_i = U_i^NEP({q_nu^i}) + 1/2 sum_{j != i} U_ZBL(r_ij)   (Eq. 1)
 *   U_ZBL(r) = e^2/(4 pi eps0) Zi Zj / r * phi(r/a) * f_c(r)                  (Eq. 2)
 *   phi(x) = 0.32825 e^{-2.54931x} + 0.09219 e^{-0.29182x} + 0.58110 e^{-0.59231x}  (Eq. 3)
 *   a = 0.46848 / (Zi^0.23 + Zj^0.23)                                         (Eq. 4)
 *   f_c: Tersoff switch between zbl_r_inner and zbl_r_outer                   (Sec. II.A)
 *
 * U^NEP is a one-hidden-layer tanh network of a descriptor with Chebyshev
 * radial and Legendre angular components (Sec. II.A).  The descriptor read
 * here (the same contract the tests' FP64 CPU checker follows):
 *   f_k(r) = (T_k(2 (r/rc - 1)^2 - 1) + 1)/2 * (1 + cos(pi r/rc))/2,
 *   g_n(r) = sum_k c_nk f_k(r),
 *   q_n    = sum_j g^R_n(r_ij)                                   (n = 0..n_max_radial)
 *   q_nl   = sum_j sum_k g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk) (l = 1..l_max)
 *   q4_n   = tr(T_n^3), T_n = sum_j g^A_n(r_ij) (u_ij u_ij^T - I/3)
 *   U^NEP  = sum_mu w1_mu tanh(sum_nu w0_{mu nu} s_nu q_nu - b0_mu) - b1.
 * Forces F = -dE/dr; virial W_ab = -sum_i sum_j (dU_i/dr_ij)_a (r_ij)_b with
 * r_ij = r_j - r_i (so P = (2 KE + tr W) / (3 V)).
 * Units: A, eV, eV/A, amu, fs.
 *
 * Memory: every array argument documented "device" is a pointer to GPU
 * memory owned by the caller (for example a torch tensor's data_ptr); the
 * library never frees it.  "host" arguments are ordinary CPU memory.  The
 * library owns its context and all scratch memory (cell lists, neighbour
 * lists, accumulators, CUDA graphs) and frees it in nep_free.
 *
 * Streams: all GPU work of a call is issued on the caller's stream
 * (cudaStream_t passed as void*, NULL = legacy default stream) and the call
 * returns after that stream has finished the call's work.  A context must not
 * be used from two threads at once.
 *
 * Errors: every int-returning call returns NEP_OK (0) or a negative
 * NEP_ERR_* code and never aborts the process; nep_last_error gives a
 * message.  GPU-side problems (neighbour overflow, non-finite values) are
 * reported through a device status word read after the stream sync.
 */
#ifndef NEPZBL_H
#define NEPZBL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEP_OK                 0
#define NEP_ERR_INVALID_ARG   (-1)  /* bad pointer, size, or parameter */
#define NEP_ERR_CUDA          (-2)  /* a CUDA runtime call failed */
#define NEP_ERR_NBR_OVERFLOW  (-3)  /* neighbour capacity exceeded and could not grow */
#define NEP_ERR_BOX           (-4)  /* cell with det <= 0, non-finite, or too small */
#define NEP_ERR_NONFINITE     (-5)  /* NaN/Inf in positions, energies or forces */
#define NEP_ERR_ATOM_LOST     (-6)  /* reserved: atom outside any representable cell */
#define NEP_ERR_UNSUPPORTED   (-7)  /* model sizes this build was not compiled for */

/* Arithmetic of the force evaluation. */
#define NEP_FP32  0   /* FP32 descriptors/network/forces; FP64 positions, integrator,
                         energy and virial sums; deterministic fixed-point force sums */
#define NEP_FP64  1   /* every step in FP64 (reference path) */

typedef struct nep_ctx nep_ctx;   /* opaque; created by nep_init */

/* Model definition, copied by nep_init (the caller may free it afterwards).
 * This build supports n_types = 1..4, n_max_radial = n_max_angular = 4,
 * basis_size_radial = basis_size_angular = 8, l_max = 4, use_4body = 1,
 * n_hidden = 30 (descriptor length D = 30; 961 + 90 T^2 parameters for T
 * species, 1051 for one), with zbl_r_outer <= rc_angular <= rc_radial.
 * Several species (the multi-species form of the NEP descriptor, Sec. II.A
 * and the NEP papers it cites): every pair term of the pair (i, j) uses the
 * coefficient block of the ordered species pair (t_i, t_j); the network is
 * shared; the ZBL term of the pair uses Z_{t_i}, Z_{t_j} in Eq. 2 and 4
 * (with the W-W screening function of Eq. 3 for every pair). */
typedef struct nep_params {
    int32_t n_types;                 /* number of species T (1..4) */
    int32_t z[4];                    /* nuclear charge Z per species (Eq. 2, 4) */
    double  mass[4];                 /* mass per species (amu), used by md_step */
    double  rc_radial;               /* r_c^R (A) */
    double  rc_angular;              /* r_c^A (A) */
    double  zbl_r_inner;             /* Tersoff switch inner radius (A) */
    double  zbl_r_outer;             /* Tersoff switch outer radius (A) */
    int32_t n_max_radial;            /* radial functions n = 0..n_max_radial */
    int32_t n_max_angular;           /* angular functions n = 0..n_max_angular */
    int32_t basis_size_radial;       /* Chebyshev k = 0..basis_size_radial */
    int32_t basis_size_angular;      /* Chebyshev k = 0..basis_size_angular */
    int32_t l_max;                   /* Legendre orders l = 1..l_max */
    int32_t use_4body;               /* 1: append q4_n = tr(T_n^3) */
    int32_t n_hidden;                /* hidden tanh neurons */
    const double* params;            /* host, flat: w0[H][D] row-major, b0[H], w1[H], b1,
                                        cR[T][T][nR][KR], cA[T][T][nA][KA] (block
                                        [t_i][t_j]: centre species, neighbour species) */
    int64_t n_params;                /* length of params */
    const double* q_scaler;          /* host, length D: s_nu */
} nep_params;

/* Creates a context for one model.  precision = NEP_FP32 or NEP_FP64.
 * Selects the current CUDA device.  On success *out owns the context. */
int nep_init(const nep_params* p, int precision, nep_ctx** out);

/* Frees the context and all memory it owns (NULL is allowed). */
void nep_free(nep_ctx* ctx);

/* Message of the last error of this context (or of the last failed nep_init
 * when ctx is NULL).  Valid until the next call on the context. */
const char* nep_last_error(const nep_ctx* ctx);

/* One force evaluation (Eq. 1-4 and the descriptor above).
 *   n_atoms      number of atoms (0 allowed; < 2^26)
 *   xyz          device double[3 * n_atoms], SoA: x[0..n), y[0..n), z[0..n) (A)
 *   box          host double[9], row-major 3x3 cell H whose rows are the cell
 *                vectors a, b, c (x = s H for fractional s); det H > 0.  A
 *                diagonal H is an orthorhombic box of lengths H[d][d]; any other
 *                H is a triclinic cell.  A periodic direction needs a
 *                perpendicular cell width >= 3 * rc_radial.  For an open
 *                direction the cell spans fractional [0, 1) over which the cell
 *                grid is laid (atoms outside it are still handled).
 *   types        device int32[n_atoms] species index in [0, n_types); an index
 *                outside is reported as NEP_ERR_INVALID_ARG
 *   pbc          host int32[3], 1 periodic, 0 open
 *   energy       host double[1]: E (eV)
 *   forces       device double[3 * n_atoms], SoA (eV/A), overwritten
 *   virial       host double[9], row-major W (eV), or NULL
 *   site_energy  device double[n_atoms]: U_i (eV), or NULL
 *   stream       cudaStream_t or NULL
 * Grows its neighbour capacity and repeats the evaluation when an atom has
 * more neighbours than fit. */
int nep_compute(nep_ctx* ctx, int64_t n_atoms, const double* xyz, const double box[9],
                const int32_t* types, const int32_t pbc[3], double* energy, double* forces,
                double* virial, double* site_energy, void* stream);

/* State of an MD run.  Pointers are device memory owned by the caller. */
typedef struct nep_md_state {
    int64_t n_atoms;
    double* xyz;            /* device double[3n] SoA positions (A), advanced in place;
                               periodic coordinates are wrapped into [0, L) */
    double* vel;            /* device double[3n] SoA velocities (A/fs) */
    double* forces;         /* device double[3n] SoA forces at xyz (eV/A) */
    const int32_t* types;   /* device int32[n] species in [0, n_types); each atom moves
                               with the mass of its species (nep_params.mass) */
    double box[9];          /* host copy of the cell (see nep_compute) */
    int32_t pbc[3];
    int32_t forces_valid;   /* in/out: 0 = md_step first computes forces at xyz */
    double dt_max;          /* time step or its upper limit (fs) */
    double d_max;           /* > 0: dt = min(dt_max, d_max / max_i |v_i|) before each
                               step (Sec. II.B); <= 0: fixed dt = dt_max */
    /* outputs, updated by md_step */
    double time;            /* accumulated simulated time (fs) */
    int64_t step;           /* accumulated number of steps */
    double dt_last;         /* time step of the last step (fs) */
    double potential_energy;/* E after the last step (eV) */
    double kinetic_energy;  /* KE after the last step (eV) */
    double virial[9];       /* W after the last step (eV) */
    double thermostat_energy;  /* energy of the Nose-Hoover chain after the last step
                                  (eV; 0 without a thermostat): PE + KE + this is
                                  conserved */
} nep_md_state;

/* Advances the state by n_steps velocity-Verlet steps (Sec. II.B):
 *   v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m,
 * NVE unless a thermostat and/or barostat is set (below).
 * Steps are replayed from captured CUDA graphs in chunks; if a chunk
 * overflows the neighbour capacity the chunk is rolled back from a device
 * copy, the capacity grows and the chunk runs again.  With a barostat the box
 * changes every step and the steps are launched directly (box read back after
 * each step; state->box is updated). */
int md_step(nep_ctx* ctx, nep_md_state* state, int n_steps, void* stream);

/* md_step with the state in HOST memory: xyz, vel, forces and types of
 * `state` are host arrays (pinned or pageable; device memory is rejected with
 * NEP_ERR_INVALID_ARG).  The call copies them to device buffers the context
 * owns (allocated on the first call and when n_atoms grows; freed by
 * nep_free), advances n_steps exactly as md_step (Sec. II.B), copies xyz, vel
 * and forces back and updates the outputs of `state`; it returns after the
 * copies have completed (the stream is synchronised).  forces are copied in
 * only when forces_valid is set.  Errors as md_step; on an error the host
 * arrays are left unchanged. */
int md_step_host(nep_ctx* ctx, nep_md_state* state, int n_steps, void* stream);

/* Timings of the candidates of one tuning run (host struct, filled by the
 * library).  Each candidate has two parameters a, b whose meaning the tuning
 * call states, and the median of its timed repetitions in milliseconds. */
typedef struct nep_tune_table {
    int32_t n;            /* candidates timed (at most 32) */
    int32_t a[32], b[32]; /* parameters of each candidate */
    double ms[32];        /* median time of each candidate (ms) */
    int32_t best;         /* index of the candidate kept */
} nep_tune_table;

/* Autotuner of the MD path (an engineering addition; the paper tunes
 * nothing).  On the state's own atoms, box and species it times, with CUDA
 * events on `stream`:
 *   1. every neighbour-search tiling (NEP_OPT_NBR_SLICES 1, 2, 4, 8 x
 *      NEP_OPT_NBR_CHUNK 4, 8, 16) by `reps` force evaluations each, written
 *      into a scratch force array owned by the context; tiling table: a = z
 *      slices, b = chunk width, ms per evaluation (triclinic cells: one
 *      candidate, the fixed search);
 *   2. unless a thermostat or barostat is set, the steps per captured graph
 *      (NEP_OPT_GRAPH_CHUNK 10, 25, 50) by `reps` runs of 50 MD steps of a
 *      copy of the state in context-owned device memory (after one untimed
 *      run that captures the graphs); chunk table: a = steps per graph,
 *      b = 0, ms per MD step;
 * and keeps the fastest of each (median of the repetitions) as the
 * context's options.  The caller's state (xyz, vel, forces, types: device
 * memory) is read, never written.  reps in [1, 50]; either table pointer may
 * be NULL.  The tiling choice does not change which pairs are found.
 * Synchronous. */
int nep_md_autotune(nep_ctx* ctx, const nep_md_state* state, int reps, void* stream,
                    nep_tune_table* tiling, nep_tune_table* chunk);

/* ---------------------------------------------------------------------------
 * Cascade protocol (Sec. II.B): the atoms within 3 a0 of the box boundaries
 * are held at 300 K by a Nose-Hoover chain thermostat, the system is first
 * equilibrated at 300 K and 0 GPa, and the PKA starts with its energy along
 * <135>.
 * --------------------------------------------------------------------------- */

/* Nose-Hoover chain (Martyna, Klein and Tuckerman 1992) on a group of atoms,
 * integrated by the Trotter splitting NHC(dt/2) Verlet NHC(dt/2) (Martyna,
 * Tuckerman, Tobias and Klein 1996): N_f = 3 x group size, Q_1 = N_f k T tau^2,
 * Q_j = k T tau^2.  The chain is set to rest by this call and persists across
 * md_step calls. */
typedef struct nep_thermostat {
    double temperature;      /* K */
    double tau;              /* fs */
    int32_t chain_length;    /* 1..8 */
    const uint8_t* group;    /* device uint8[n_atoms] of the MD state, 1 = thermostatted;
                                NULL = every atom.  Read by later md_step calls. */
} nep_thermostat;
int nep_set_thermostat(nep_ctx* ctx, const nep_thermostat* t);   /* t == NULL: off */

/* Berendsen barostat: after each step, for every periodic dimension a,
 *   P_aa = (sum_i m_i v_ia^2 + W_aa) / V,
 *   mu_a = [1 - compressibility (dt / tau) (pressure - P_aa)]^(1/3),
 * and x_a, L_a are multiplied by mu_a (velocities unchanged); open
 * dimensions keep their extent.  A Verlet skin is not used while it is on. */
typedef struct nep_barostat {
    double pressure;         /* target (GPa) */
    double tau;              /* fs */
    double compressibility;  /* 1/GPa */
} nep_barostat;
int nep_set_barostat(nep_ctx* ctx, const nep_barostat* b);   /* b == NULL: off */

/* PKA launch: the atom nearest to point (A; minimum image in periodic
 * dimensions, lowest index on ties) gets the velocity of kinetic energy
 * `energy` (eV) along `direction` (any nonzero length; the paper uses
 * <135>), replacing its velocity.  *atom receives its index.  Synchronous. */
int nep_pka(nep_ctx* ctx, nep_md_state* state, const double point[3], double energy,
            const double direction[3], int64_t* atom, void* stream);

/* Counters of a context (for benchmarks and tests). */
typedef struct nep_stats {
    int64_t kernel_launches;    /* kernels launched by this context (graph nodes counted) */
    int64_t timed_launches;     /* force-kernel launches timed while timing was on */
    double  timed_ms;           /* their summed duration (CUDA events, ms) */
    int64_t pairs_radial;       /* ordered pairs r < rc_radial in the last evaluation */
    int64_t pairs_angular;      /* ordered pairs r < rc_angular in the last evaluation */
    int32_t max_nbr_radial;     /* largest per-atom count in the last evaluation */
    int32_t max_nbr_angular;
    int32_t nbr_capacity;       /* current neighbour slots per atom */
    int32_t graph_chunk;        /* MD steps per captured graph */
    int64_t list_builds_skin;   /* MD neighbour-list builds with a Verlet skin so far */
    int32_t radial_q_in_neighbor_kernel;  /* 1: the last evaluation summed the radial
                                             descriptor in the neighbour-list kernel (one
                                             species, lists rebuilt every step) */
    int32_t angular_state_in_tmem;        /* 1: the last evaluation (or MD graph chunk)
                                             kept the angular descriptor sums and adjoint
                                             of some of its atoms in Tensor Memory (FP32,
                                             one species: the tiles of 128 cell-ordered
                                             atoms with at most 48 angular neighbours on
                                             every atom and no pair inside the outer ZBL
                                             radius) */
    int32_t angular_tmem_blocks_per_sm;   /* resident blocks per SM of that kernel (from
                                             the occupancy check; 0: not usable) */
    int32_t nbr_z_slices;                 /* NEP_OPT_NBR_SLICES in effect */
    int32_t nbr_chunk;                    /* NEP_OPT_NBR_CHUNK in effect */
    int64_t angular_tiles;                /* tiles of 128 cell-ordered atoms in the last
                                             evaluation (MD: summed over the last graph
                                             chunk's steps) */
    int64_t angular_tiles_register;       /* of those, the tiles the register angular
                                             kernel took: FP32, the tiles with an atom of
                                             more than 48 angular neighbours (and those
                                             with a close pair when the Tensor-Memory
                                             kernel cannot be resident); FP64, all */
} nep_stats;

int nep_get_stats(const nep_ctx* ctx, nep_stats* out);

/* Options: NEP_OPT_TIMING (0/1) times every force evaluation (the three force
 * kernels) with CUDA events, also inside MD graphs; NEP_OPT_GRAPH_CHUNK sets
 * the MD steps per captured graph (>= 1); NEP_OPT_NBR_CAPACITY sets the
 * neighbour slots per atom (grows automatically when exceeded);
 * NEP_OPT_SKIN_MILLIANGSTROM sets a Verlet skin for md_step in units of
 * 0.001 A (0, the default, rebuilds the neighbour lists every step; > 0 builds
 * them with r_c + skin and rebuilds only after some atom moved more than
 * skin / 2 since the last build, which leaves every pair within r_c in the
 * lists); NEP_OPT_NBR_SLICES (1, 2, 4 or 8; default 1) and NEP_OPT_NBR_CHUNK
 * (4, 8 or 16; default 16) tile the neighbour search of orthorhombic cells:
 * the atoms of each cell are grouped into z slices so that only the slices
 * within reach of an atom are searched, and candidates are tested in
 * unrolled chunks of that width.  They change only the order of pairs within
 * a cell's part of a list, never which pairs are found; nep_md_autotune
 * picks them by timing.  Returns NEP_ERR_INVALID_ARG for other values. */
#define NEP_OPT_TIMING               1
#define NEP_OPT_GRAPH_CHUNK          2
#define NEP_OPT_NBR_CAPACITY         3
#define NEP_OPT_SKIN_MILLIANGSTROM   4
#define NEP_OPT_NBR_SLICES           5
#define NEP_OPT_NBR_CHUNK            6
int nep_set_option(nep_ctx* ctx, int option, int64_t value);

/* Resets the counters of nep_stats (launches, timing). */
int nep_reset_stats(nep_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batches of small periodic configurations (training-style workloads)
 *
 * Many independent periodic boxes are evaluated in one persistent launch: a
 * CTA takes whole configurations from a work queue (largest first), builds
 * their neighbour lists over all periodic images (self-images included, so
 * boxes down to r_c^R per side are exact), evaluates energies and forces, and
 * for the gradient entry points the derivative of a loss with respect to all
 * n_params model parameters, including the force term's second derivatives:
 * with e_i = dL/dF_i, eps_s = dL/dE_s and G_s = dL/dW_s (3x3),
 *   dL/dtheta = sum_i d/dtheta [eps U_i - (dU_i/dq_i) . qdot_i],
 *   qdot_i = sum_j (dq_i/dd_ij) . v_ij,  v_ij = (e_j - e_i) + G_s d_ij
 * (the virial W = -sum_ij (dU_i/dd_ij) (x) d_ij enters like a homogeneous
 * deformation of the pair vectors).  Gradient sums are accumulated in FP64
 * and reduced in a fixed order.
 * Virials are 3x3 row-major per configuration (eV); virial targets and the
 * virial loss use the six components xx, yy, zz, yz, zx, xy.
 * --------------------------------------------------------------------------- */
typedef struct nep_batch {
    int32_t n_configs;
    int64_t n_atoms;             /* total atoms */
    const double* xyz;           /* device double[3 * n_atoms] SoA, configurations
                                    concatenated in order */
    const int64_t* offsets;      /* host int64[n_configs + 1]: first atom of each
                                    configuration; offsets[n_configs] = n_atoms */
    const double* boxes;         /* host double[3 * n_configs]: periodic orthorhombic box
                                    lengths, each >= rc_radial */
    const int32_t* types;        /* device int32[n_atoms] species in [0, n_types) (read
                                    only for models of several species) */
} nep_batch;
/* Each configuration holds 1..512 atoms.  With several species the gradient
 * has n_params = 961 + 90 T^2 entries in the layout of nep_params.params
 * (coefficient block (t_i, t_j) of every ordered species pair). */

/* Training targets of a batch (Sec. III.A: every structure has a target
 * energy and forces, some a target virial). */
typedef struct nep_targets {
    const double* energy;        /* device double[n_configs] (eV) */
    const double* forces;        /* device double[3 * n_atoms] SoA (eV/A) */
    const double* virial;        /* device double[6 * n_configs]: xx, yy, zz, yz, zx, xy
                                    per configuration (eV), or NULL (no virial term) */
    const uint8_t* has_virial;   /* host uint8[n_configs]: 1 where the configuration has a
                                    virial target; NULL = every configuration */
} nep_targets;

/* Loss weights: lambda_e, lambda_f, lambda_v of the data terms and lambda_1,
 * lambda_2 of the regularisers (Sec. III.A uses 1, 1, 0.1, 0.05, 0.05). */
typedef struct nep_loss_weights {
    double energy, force, virial;
    double l1, l2;
} nep_loss_weights;

/* Replaces the model parameters (same layout and length as nep_params.params;
 * the descriptor scaler is kept).  Host memory. */
int nep_set_params(nep_ctx* ctx, const double* params, int64_t n_params);

/* Energies (device double[n_configs], eV), forces (device double[3 * n_atoms]
 * SoA, eV/A) and, if virials != NULL, virials (device double[9 * n_configs],
 * eV) of every configuration.  Synchronous on the stream. */
int nep_batch_forward(nep_ctx* ctx, const nep_batch* batch, double* energies, double* forces,
                      double* virials, void* stream);

/* Gradient (device double[n_params]) of a loss L(E, F, W) given its upstream
 * derivatives dL/dE (device double[n_configs]), dL/dF (device
 * double[3 * n_atoms] SoA) and dL/dW (device double[9 * n_configs], or NULL
 * for none), evaluated at the context's current parameters. */
int nep_batch_backward(nep_ctx* ctx, const nep_batch* batch, const double* dL_dE,
                       const double* dL_dF, const double* dL_dW, double* grad, void* stream);

/* One persistent launch for forward, forces, virials, the mean-square loss
 *   L = w.energy * mean_s ((E_s - Et_s) / N_s)^2
 *     + w.force  * mean over the 3 n_atoms components (F - Ft)^2
 *     + w.virial * mean over configurations with a virial target and the six
 *                  components ((W_s - Wt_s) / N_s)^2
 * (FP64 accumulation; w.l1 and w.l2 are not used here) and its gradient
 * (device double[n_params]).  loss: host double[4] = total, energy, force and
 * virial terms.  energies, forces, virials (device) may be NULL. */
int nep_batch_loss_grad(nep_ctx* ctx, const nep_batch* batch, const nep_targets* targets,
                        const nep_loss_weights* w, double* loss, double* grad,
                        double* energies, double* forces, double* virials, void* stream);

/* Times the loss-gradient launch on this batch for each candidate of threads
 * per CTA (atoms of one configuration processed side by side: 64, 128, 256)
 * and CTAs per SM (1, 2, 4), the median of three launches each, and keeps the
 * fastest for later batched calls. */
int nep_batch_autotune(nep_ctx* ctx, const nep_batch* batch, const nep_targets* targets,
                       const nep_loss_weights* w, void* stream, int* best_threads,
                       int* best_per_sm);

/* The timings of the last nep_batch_autotune on this context: a = threads per
 * CTA, b = CTAs per SM, ms per fused launch. */
int nep_batch_autotune_table(const nep_ctx* ctx, nep_tune_table* out);

/* ---------------------------------------------------------------------------
 * Population training (the separable natural evolution strategy, SNES, that
 * Sec. III.A trains the model with; Schaul et al. 2011)
 *
 * The NEP training loss of a parameter vector theta over a batch (Sec. III.A,
 * the terms of Fig. 1(a)):
 *   L = w.energy RMSE_E + w.force RMSE_F + w.virial RMSE_V + L1 + L2,
 *   RMSE_E = sqrt(mean_s ((E_s - Et_s) / N_s)^2),
 *   RMSE_F = sqrt(mean over the 3 n_atoms components (F - Ft)^2),
 *   RMSE_V = sqrt(mean over configurations with a virial target and the six
 *            components ((W_s - Wt_s) / N_s)^2)   (0 without targets),
 *   L1 = w.l1 (1/P) sum_p |theta_p|,  L2 = w.l2 sqrt((1/P) sum_p theta_p^2).
 * The whole population is evaluated in one launch (after one launch that
 * builds the neighbour lists): each work item is one (configuration,
 * individual) pair whose model sits in shared memory.
 * --------------------------------------------------------------------------- */

/* Loss terms of n_pop (1..1024) parameter vectors thetas (device
 * double[n_pop * n_params], host layout of nep_params.params) at the
 * context's hyperparameters and scaler: losses (device double[6 * n_pop]) =
 * total, L1, L2, RMSE_E, RMSE_F, RMSE_V per individual.  Synchronous. */
int nep_population_loss(nep_ctx* ctx, const nep_batch* batch, const nep_targets* targets,
                        const nep_loss_weights* w, int n_pop, const double* thetas,
                        double* losses, void* stream);

/* One SNES generation.  mu, sigma: device double[n_params], updated in place;
 * samples: device double[n_pop * n_params] standard-normal draws supplied by
 * the caller.  Candidates theta_k = mu + sigma * s_k are evaluated with
 * nep_population_loss (losses as there, device double[6 * n_pop]), ranked by
 * total loss (ties by index) and given the utilities
 *   u_r = max(0, ln(n_pop/2 + 1) - ln r) / sum_j max(0, ln(n_pop/2 + 1) - ln j) - 1/n_pop;
 * then mu += eta_mu sigma sum_k u_k s_k and
 * sigma *= exp(eta_sigma / 2 sum_k u_k (s_k^2 - 1)).  The usual rates are
 * eta_mu = 1, eta_sigma = (3 + ln n_params) / (5 sqrt(n_params)).  Synchronous. */
int nep_snes_generation(nep_ctx* ctx, const nep_batch* batch, const nep_targets* targets,
                        const nep_loss_weights* w, int n_pop, double* mu, double* sigma,
                        const double* samples, double eta_mu, double eta_sigma, double* losses,
                        void* stream);

/* Force evaluation that allocates nothing (the paper has no counterpart; it is
 * a deployment convenience).  It is meant for callers that may not allocate
 * GPU memory at the point where they need forces: a plugin inside a host MD
 * or training program that owns all device memory through its own pool or a
 * fixed budget, and forbids its components to call cudaMalloc behind its
 * back (an allocation there can fail or fragment the host's pool mid-run).
 * It takes the model parameters directly
 * (no context: creating one allocates) and computes the same FP32 evaluation
 * as nep_compute with a context created with NEP_FP32; arguments as in
 * nep_compute.
 *   Limits: one species (n_types = 1, else NEP_ERR_UNSUPPORTED; a nonzero
 *   species index gives NEP_ERR_INVALID_ARG), at most 8192 atoms, 96
 *   neighbours per atom within rc_radial
 *   (beyond that NEP_ERR_NBR_OVERFLOW; there is no growth), a cell grid of at
 *   most 8192 cells.  Larger systems are rejected with NEP_ERR_INVALID_ARG or
 *   NEP_ERR_BOX before any GPU work.
 *   Scratch: one fixed device array of about 3.8 MB that the library
 *   declares at file scope; every GPU that loads the library holds it until
 *   the process exits.  No cudaMalloc, cudaFree or other allocating call is
 *   made.
 *   Set-up: the first call on a device (with that device current) looks up
 *   the array's device address once and caches it; make that first call
 *   before any stream capture.
 *   Device memory: xyz, types, forces and (when not NULL) site_energy must be
 *   device memory; a host pointer in any of them gives NEP_ERR_INVALID_ARG
 *   before any GPU work.
 *   Concurrency: all calls share the one array; calls whose GPU work overlaps
 *   (different streams, threads or processes' contexts on the same device
 *   within this process) race and give wrong results.  Each call clears what
 *   must start at zero, copies its energy and virial to the host and
 *   synchronises the stream before it returns.
 * Errors are reported through nep_last_error(NULL). */
int nep_compute_static(const nep_params* p, int64_t n_atoms, const double* xyz,
                       const double box[9], const int32_t* types, const int32_t pbc[3],
                       double* energy, double* forces, double* virial, double* site_energy,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEPZBL_H */
