/*
 * ftcj.h -- C ABI of the GB300 (sm_103a) long-range Fourier-transformed
 * Coulomb build: the integral-direct planewave density fitting of the
 * G != 0 Ewald term of the periodic Coulomb matrix of arXiv 2509.16460.
 *
 * Problem statement followed (paper Sec. 2.2-2.4):
 *   D^{0n}  = (1/Nk) sum_k exp(-i k.R_n) D^k                 (Eq. "FT for D")
 *   rho(G)  = sum_{mu nu L} D^{0[L]}_{mu nu} (mu0 nuL|G)      (LR step 1)
 *   V(-G)   = rho(-G) v(G),  v(G) = 4 pi exp(-G^2/4w^2)/(Omega G^2)
 *                                                             (LR step 2)
 *   J^{0L}_{mu nu} = sum_{G != 0} (mu0 nuL|G) V(-G)           (LR step 3,
 *                                                  Eq. "Ewald J", 2nd term)
 *   J^k     = sum_L exp(+i k.R_L) J^{0L}                      (Eq. "FT of J")
 *   E_J     = 1/2 sum_{G != 0} v(G) |rho(G)|^2
 * with (mu0 nuL|G) = int phi_mu(r) phi_nu(r - R_L) exp(-i G.r) dr
 * (Eq. "AFT for pair density"), G over the reciprocal lattice inside
 * |G| < Gcut, pairs of primitive shells screened by their overlap.
 *
 * Units: bohr, hartree.  Lattice rows are the lattice vectors a_i.  The
 * k-mesh is Gamma-centred, k_m = sum_i (m_i/N_i) b_i, flattened as
 * m = (m1*N2 + m2)*N3 + m3; BvK cells n use the same flattening.
 *
 * AO order: shell order; inside a Cartesian shell lx = l..0, ly = l-lx..0
 * (xx, xy, xz, yy, yz, zz); inside a spherical shell m = -l..l except p,
 * which is (x, y, z).  Every primitive is unit-normalised; the shell's
 * coefficients multiply normalised primitives.  Shells up to l = 2.
 *
 * Complex arrays are interleaved (re, im) doubles.
 *
 * Preconditions of the build: D^k Hermitian for every k and time-reversal
 * symmetric, D^{-k} = conj(D^k), so that D^{0n} and J^{0n} are real.  The
 * fold step keeps Re D^{0n}; ftcj_plan_info reports nothing about the
 * input, use ftcj_check_density to measure a violation.
 *
 * Errors: every call returns FTCJ_OK (0) or a negative FTCJ_E* code; no
 * exception or abort crosses this boundary.  ftcj_last_error() gives a
 * thread-local message for the last failing call on the calling thread.
 *
 * Ownership: the caller owns every input and output buffer.  The plan owns
 * all device scratch, allocated in ftcj_plan_create and freed in
 * ftcj_plan_destroy; the build calls allocate nothing.
 *
 * Threading: a plan is used by one host thread and one stream at a time.
 */
#ifndef FTCJ_H
#define FTCJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FTCJ_OK 0
#define FTCJ_EINVAL (-1)       /* bad argument or input */
#define FTCJ_ENOMEM (-2)       /* device or host allocation failed */
#define FTCJ_ECUDA (-3)        /* a CUDA runtime call failed */
#define FTCJ_ETIMEOUT (-4)     /* a bounded device wait gave up */
#define FTCJ_EUNSUPPORTED (-5) /* valid input outside what this build handles */

#define FTCJ_PREC_FP64 0       /* every step in FP64 */
#define FTCJ_PREC_SPLIT 1      /* walks (a4, a6) in double-float FP32 pairs; FP64 setup, sums and E_J */

#define FTCJ_LMAX 2            /* highest shell angular momentum */

typedef struct {
    double A[9]; /* row i = lattice vector a_i (bohr), row-major */
} ftcj_cell;

typedef struct {
    int centre;          /* index into ftcj_basis.xyz */
    int l;               /* 0..FTCJ_LMAX */
    int spherical;       /* 1: real solid harmonics, 0: Cartesian */
    int nprim;           /* >= 1 */
    const double* exps;  /* [nprim] > 0 */
    const double* coefs; /* [nprim], multiply unit-normalised primitives */
} ftcj_shell;

typedef struct {
    int ncentre;
    const double* xyz; /* [ncentre][3] Cartesian bohr */
    int nshell;
    const ftcj_shell* shells;
} ftcj_basis;

typedef struct {
    double omega;       /* Ewald range-separation parameter w > 0 (1/bohr) */
    double gcut;        /* sphere radius; <= 0: 2 w sqrt(ln(1/eps_g)) */
    double eps_g;       /* kernel floor exp(-Gcut^2/4w^2) when gcut <= 0 */
    double pair_thresh; /* keep primitive pairs with overlap bound > this */
    int precision;      /* FTCJ_PREC_FP64 or FTCJ_PREC_SPLIT */
    int max_dens;       /* densities per device batch (scratch is sized for it); <= 0: 1 */
    int chunk_points;   /* G points per walk chunk, 64..4096; <= 0: 4096 in the FP64 form; in the
                           split form the longest power of two (<= 4096) whose structure-factor
                           walk keeps three blocks per SM in shared memory (one kernel, >= 1024
                           points; else its classes 0-2 part, >= 512), else two blocks (>= 512),
                           else one */
    int rho_blocks;     /* persistent blocks of the structure-factor walk; <= 0: fill the GPU
                           (the split form then runs classes 3-4 and 0-2 as two launches where
                           shared memory holds the one-kernel walk below three blocks per SM);
                           > 0: that many blocks of the one-kernel walk */
    double pair_gcut_eps; /* > 0: per-pair G cutoffs (Sec. 2.5, Eq. "AFT screening obj"): each pair
                             record is evaluated only for |G| below the radius where its
                             screening estimate 8 pi eta G (4 pi/G^2) e^{-G^2/4w^2} |rho_ab(G)|
                             falls under this value (split and FP64 forms).
                             0: every pair over the whole sphere. */
    int shard_count;    /* > 1: a record-sharded plan for one of shard_count GPUs: it keeps only
                           share shard_index (0-based) of the screened pair records, a contiguous
                           range of their class-sorted order balanced by the walks' per-record cost
                           (ftcj_shard_bounds).  The shards' ftcj_rho and ftcj_jback outputs are
                           partial sums, to be summed across the shards (an all-reduce) before
                           ftcj_potential resp. ftcj_unfold_j; ftcj_jbuild, ftcj_jbuild_host and
                           ftcj_grad refuse a shard plan (EINVAL).  <= 1: the whole pair list. */
    int shard_index;
    int contraction;    /* FTCJ_CONTRACT_WALK (0): the G walks for the structure-factor pass;
                           FTCJ_CONTRACT_TC (1): the tensor-core separable contraction (Sec. 2.4,
                           orthorhombic fully separable case): rho(n) as a sliced bf16 tcgen05 matrix
                           product over (pair record, i, j), split form and orthorhombic cells only
                           (EUNSUPPORTED otherwise), whole sphere (pair_gcut_eps = 0); the
                           back-contraction (Alg. S1) takes the same form where the sphere's
                           (n_a, n_b) rows fit one exact accumulation, else the split walk
                           (ftcj_info.j_contraction says which) */
    int tc_wait_log2;   /* tensor-core kernels: each wait between their roles gives up after
                           2^tc_wait_log2 clock cycles (0: 2^32, about 2 s), raises the plan's device
                           error word (ftcj_plan_status) and lets the kernel drain and return; 1..40,
                           small values are for tests of that path */
    int classify;       /* 1: compact/diffuse classification of the pair densities (Sec. 2.6).  A pair
                           record whose two primitives both have exponents below alpha_cut is DD; the
                           DD records leave the planewave walks and take the GPW route (App. E): their
                           density is collocated on a uniform real-space grid of the cell, transformed
                           onto the G sphere, and their J' back-contracted on the same grid.  Integrals
                           between two compact pair densities keep the long-range kernel v(G), every
                           other one takes the full-range 4 pi / (Omega G^2), G = 0 removed.
                           ftcj_jbuild and ftcj_jbuild_host return that build; the step calls
                           (ftcj_rho, ftcj_potential, ftcj_jback), ftcj_grad, shard plans and batches
                           refuse a classified plan, and it takes no per-pair cutoffs (EUNSUPPORTED).
                           0: every pair record in the long-range walks. */
    double alpha_cut;   /* classify = 1: the exponent boundary; <= 0: w^2/2 (Eq. "cd cutoff") */
    int gpw_grid[3];    /* classify = 1: grid points along a_1, a_2, a_3; each <= 0: the smallest count
                           N_i with N_i |b_i| >= Gcut + sqrt(184 p_max) (every alias of a DD transform,
                           exponent p <= p_max, below e^{-46} on the sphere) and N_i > 2 max|n_i|;
                           an explicit count below 2 max|n_i| + 1 is refused (EINVAL) */
} ftcj_params;

#define FTCJ_CONTRACT_WALK 0
#define FTCJ_CONTRACT_TC 1

typedef struct {
    int nao;                  /* AOs per cell */
    int nk;                   /* k-points = BvK cells */
    int nshell;
    int ngroup;               /* distinct (centre, exponent) primitive groups */
    int64_t npairs;           /* pair records after the (a0,bL)<->(b0,a-L) reduction */
    int64_t npairs_ordered;   /* ordered screened primitive-shell pairs */
    int64_t ng_half;          /* G vectors in the half sphere (rho is stored there) */
    int64_t ng_full;          /* G != 0 in the full sphere = 2 ng_half */
    int64_t pair_g_units;     /* npairs_ordered * ng_full: the work unit count */
    int64_t pairs_by_class[5];/* pair records per L = l_a + l_b class */
    int nlines;               /* G lines along b_1 walked per pair */
    int nchunks;              /* G chunks (grid dimension of the walks) */
    double gcut;
    double volume;
    size_t device_bytes;      /* device memory held by the plan */
    int rho_blocks;           /* persistent blocks of the structure-factor walk */
    int n1_table;             /* split form, orthorhombic cell: entries of the per-record
                                 X(n1) table (0: the n1 walk runs the recurrence) */
    int64_t pair_g_units_screened; /* with pair_gcut_eps > 0: ordered pairs x G (full sphere)
                                      inside each record's own cutoff; else = pair_g_units */
    int64_t pair_g_units_walked;   /* record x G evaluations the walks perform (both passes
                                      count once), x4 for the (+-G, mirror) symmetries: the
                                      work actually done in the units of pair_g_units */
    int n_abs_max;            /* largest |n_i| of the sphere's G = sum_i n_i b_i (the split form
                                 needs <= 63) */
    int grad_split;           /* 1: ftcj_grad's back-contraction runs in double-float (split
                                 form with n_abs_max <= 27), 0: in FP64 */
    int rho_walk_launches;    /* kernel launches of one structure-factor walk pass: 2 where the
                                 split form runs it as two class parts, else 1 (0: nothing to walk) */
    int j_walk_launches;      /* the same for the back-contraction walk */
    int contraction;          /* FTCJ_CONTRACT_WALK or FTCJ_CONTRACT_TC (the plan's structure-factor pass) */
    int64_t tc_mma_flops;     /* tensor-core contraction: bf16 MMA flops (2 per multiply-add, every slice
                                 product and padding column included) of one structure-factor pass over
                                 max_dens densities; 0 for the walks */
    int j_contraction;        /* the back-contraction's form: FTCJ_CONTRACT_TC where a tensor-core plan's
                                 rows fit one exact accumulation (<= 672 rows of (n_a, n_b)), else
                                 FTCJ_CONTRACT_WALK */
    int64_t tc_j_mma_flops;   /* the same count for one tensor-core back-contraction; 0 for the walk */
    int tc_column_axis;       /* tensor-core form: the lattice axis of the columns (n_c), 0..2 */
    int tc_rows;              /* its rows (n_a, n_b) and row tiles of 128 */
    int tc_row_tiles;
    int tc_blocks_per_window; /* (i, j) blocks side by side in one structure-factor window */
    int tc_dens_per_launch;   /* densities per structure-factor launch */
    int64_t dd_pairs;         /* classified plan: DD pair records (GPW route); npairs, pairs_by_class and
                                 the pair*G counts above cover the compact records only */
    int64_t dd_pairs_ordered; /* the DD records' ordered primitive-shell pairs */
    double alpha_cut;         /* classified plan: the exponent boundary in use, else 0 */
    int gpw_grid[3];          /* the GPW grid (0 without DD records) */
    int gpw_separable;        /* 1: orthorhombic cell, per-axis factor tables (FP64); 2: the same with the grid
                                 contractions in double-float (split form); 0: per-point lattice images (FP64) */
    int gpw_launches;         /* kernel launches of the GPW route in one build over max_dens densities */
    int64_t dd_pairs_by_class[5]; /* DD records of class L = l_a + l_b (the GPW route's cost per grid point
                                     and density is 2 (L + 1) flops in each of collocation and integration) */
} ftcj_info;

typedef struct ftcj_plan ftcj_plan;

/* Plan for one cell, basis, k-mesh and parameter set.  Runs the pair
 * screening and sorting on the device (default stream, synchronised) and
 * allocates all scratch.  cell/basis/params are copied; the caller may free
 * them afterwards.  Errors: EINVAL (bad lattice, centres, exponents, omega,
 * k-mesh), EUNSUPPORTED (l > FTCJ_LMAX, unknown precision, a G line
 * longer than the walk chunk), ENOMEM, ECUDA. */
int ftcj_plan_create(const ftcj_cell* cell, const ftcj_basis* basis, const int kmesh[3],
                     const ftcj_params* params, ftcj_plan** out);

/* The record shares of a sharded build (host only, no device needed): records
 * sorted by class L (class_counts[L] of them, L = 0..4) are cut into
 * shard_count contiguous ranges of nearly equal walk cost, per record 38 L +
 * 100 FP32 operations per point in the split form, 4 L + 24 FP64 operations in
 * the FP64 form.  bounds[0..shard_count] (written): share s is records
 * [bounds[s], bounds[s+1]).  Errors: EINVAL. */
int ftcj_shard_bounds(const int64_t* class_counts, int precision, int shard_count, int64_t* bounds);

/* Sizes and counts of a plan (host struct, filled by the call). */
int ftcj_plan_info(const ftcj_plan* plan, ftcj_info* out);

/* Frees the plan and its device memory.  NULL is ignored. */
void ftcj_plan_destroy(ftcj_plan* plan);

/* Whole long-range build, steps a2..a8, on `stream` (a cudaStream_t; NULL =
 * legacy default stream).  All pointers are DEVICE memory owned by the
 * caller:
 *   Dk  complex [ndens][Nk][nao][nao]  (read)
 *   Jk  complex [ndens][Nk][nao][nao]  (written)
 *   EJ  double  [ndens]                (written, hartree per cell)
 * ndens >= 1; densities are processed in batches of params.max_dens.
 * Asynchronous: returns after enqueueing.  Errors: EINVAL, ECUDA. */
int ftcj_jbuild(ftcj_plan* plan, int ndens, const double* Dk, double* Jk, double* EJ, void* stream);

/* The same build on HOST buffers (same layouts), synchronising `stream`
 * before it returns.  A page-locked (cudaHostAlloc / cudaHostRegister) or
 * managed D^k or J^k is read or written by the k-mesh transform kernels
 * directly over the host link, so its transfer overlaps that kernel; a
 * pageable buffer is copied through plan-owned staging sized at plan creation
 * for max_dens densities.  ndens may exceed max_dens (batched). */
int ftcj_jbuild_host(ftcj_plan* plan, int ndens, const double* Dk_host, double* Jk_host, double* EJ_host,
                     void* stream);

/* ---- the individual steps (device pointers, asynchronous on stream) ---- */

/* a2: D^{0n} = Re (1/Nk) sum_k exp(-i k.R_n) D^k (Eq. "FT for D").
 * Dk complex [ndens][Nk][nao][nao] -> D0n double [ndens][Ncell][nao][nao],
 * ndens <= max_dens. */
int ftcj_fold_density(ftcj_plan* plan, int ndens, const double* Dk, double* D0n, void* stream);

/* a3 + a4: Hermite densities of every pair record (Alg. 2) and the
 * structure-factor pass over the half sphere (Alg. 1):
 * D0n double [ndens][Ncell][nao][nao] -> rho complex [ndens][ng_half] in
 * the order of ftcj_get_gvectors.  ndens <= max_dens. */
int ftcj_rho(ftcj_plan* plan, int ndens, const double* D0n, double* rho, void* stream);

/* a5: V and E_J from rho on the half sphere:
 * W(G) = 2 v(G) conj(rho(G)) complex [ndens][ng_half];
 * EJ[d] = sum_half v |rho|^2 (= 1/2 sum over the full sphere). */
int ftcj_potential(ftcj_plan* plan, int ndens, const double* rho, double* W, double* EJ, void* stream);

/* Allocation-free variant of the potential and energy step; needs no plan.
 * For callers that cannot call cudaMalloc: code running where another
 * allocator already owns the device memory (a framework's caching allocator
 * or a pre-reserved pool), and which therefore cannot create a plan, or code
 * that must not allocate inside its iteration loop.  For the same G list it
 * gives what ftcj_potential gives:
 *   W(G) = 2 v(G) conj(rho(G)),  EJ[d] = sum_G v(G) |rho_d(G)|^2,
 *   v(G) = 4 pi exp(-|G|^2/4w^2) / (Omega |G|^2),  G = n1 b_1 + n2 b_2 + n3 b_3.
 *   A     host double[9], lattice rows (bohr); omega > 0
 *   gvec  device int [ng][3] without (0,0,0) (v is not finite there)
 *   rho   device complex [ndens][ng];  W device complex [ndens][ng] (written)
 *   EJ    device double [ndens] (written)
 * Its only scratch, the per-block energy partial sums, is a fixed file-scope
 * device array of FTCJ_NOALLOC_MAX_PARTIALS doubles (128 KiB) that every GPU
 * loading the library keeps until the process exits.  No element of it has to
 * start at zero (a call reads only slots it wrote earlier in the same call);
 * it keeps the last call's contents; calls that overlap on the GPU share it
 * and race, so serialise them.  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.  The address is cached per device ordinal for
 * the life of the process, which assumes the device's primary context lives
 * that long: after cudaDeviceReset (or any re-creation of the primary
 * context) the cached address is stale, so do not call this entry point
 * again in that process.  All pointers must be on the current device, and
 * `stream` must belong to it.  Errors: EINVAL when ndens * ceil(ng/256) >
 * FTCJ_NOALLOC_MAX_PARTIALS (split the densities over several calls), for a
 * singular lattice, or omega <= 0.  The paper has no counterpart to this
 * entry point. */
#define FTCJ_NOALLOC_MAX_PARTIALS 16384
int ftcj_potential_noalloc(const double A[9], double omega, int ndens, int64_t ng, const int* gvec,
                           const double* rho, double* W, double* EJ, void* stream);

/* a6 + a7: back-contraction (Alg. S1) and transform to AOs (Alg. S2):
 * W complex [ndens][ng_half] -> J0n double [ndens][Ncell][nao][nao]
 * (J^{0L} folded into the BvK cells; overwritten).  ndens <= max_dens. */
int ftcj_jback(ftcj_plan* plan, int ndens, const double* W, double* J0n, void* stream);

/* a8: J^k = sum_n exp(+i k.R_n) J^{0n} (Eq. "FT of J"):
 * J0n double [ndens][Ncell][nao][nao] -> Jk complex [ndens][Nk][nao][nao].
 * ndens <= max_dens. */
int ftcj_unfold_j(ftcj_plan* plan, int ndens, const double* J0n, double* Jk, void* stream);

/* Nuclear gradient of the long-range energy with D^k held fixed (the
 * derivatives of the pair transforms with respect to their two centres,
 * from d/dA [(x-A)^i e^{-a(x-A)^2}] = 2a (x-A)^{i+1} e^{..} - i (x-A)^{i-1} e^{..}
 * applied to Eq. "FT of cart Gaussians" and the Gaussian product):
 *   grad[d][C][x] = dE_J[d]/dR_{C,x}  (device double [ndens][ncentre][3]),
 *   EJ[d]          (device double [ndens]).
 * The derivative of E_J with respect to D^k is J^k/Nk (ftcj_jbuild).
 * Runs a2..a5 and a back-contraction one degree higher than the build's,
 * in the plan's form (split: double-float on the FP32 pipe where every
 * |n_i| <= 27, so that FP32 holds the fifth powers exactly; else FP64),
 * followed by an FP64 assembly per centre.  With pair_gcut_eps > 0 the
 * double-float back-contraction walks the same points as the build's, so the
 * result is the derivative of the screened energy that ftcj_jbuild returns
 * (the FP64 one walks the whole sphere).
 * Asynchronous on `stream`. */
int ftcj_grad(ftcj_plan* plan, int ndens, const double* Dk, double* EJ, double* grad, void* stream);

/* Device error word of the plan's kernels that wait on one another inside a
 * block (the tensor-core contraction): bit 0 set when a bounded wait gave up
 * (the results of that build are invalid).  Synchronises `stream`, returns
 * the word in *flags and clears it.  A plan without such kernels reports 0. */
int ftcj_plan_status(ftcj_plan* plan, int* flags, void* stream);

/* Largest |Im D^{0n}| and largest |D^{0n}_{mu nu} - D^{0,-n}_{nu mu}| of
 * the input (host doubles out), i.e. how far D^k is from the precondition.
 * Synchronises `stream`.  ndens <= max_dens. */
int ftcj_check_density(ftcj_plan* plan, int ndens, const double* Dk, double* max_imag, double* max_asym,
                       void* stream);

/* ---- batches of independent cells ---- */

/* Several independent problems (each its own cell, basis, k-mesh and
 * parameters, e.g. an uneven set of cells or geometries) built together.
 * The cells' builds are spread over internal streams (largest estimated
 * work first, each stream taking the next cell when it is least loaded) and
 * joined back to the caller's stream, so small cells overlap on the GPU.
 * With FTCJ_BATCH_AUTOTUNE each cell's walk shape (chunk size, rho-walk
 * blocks) is chosen by ftcj_autotune before its plan is made. */
#define FTCJ_BATCH_AUTOTUNE 1
/* With FTCJ_BATCH_PERSISTENT the structure-factor walks, the potentials and
 * energies, and the back-contraction walks of every cell run as ONE
 * persistent launch over a shared work queue (Alg. 1 and Alg. S1 over many
 * cells): structure-factor items (cell, block of the cell's schedule, walk
 * chunk, density) first, largest first, then back-contraction items (cell,
 * tile, chunk, density) in the order the cells become ready.  The CTA that
 * finishes a cell's last structure-factor item sums its FP64 rows in fixed
 * order into rho, W and E_J; a back-contraction item waits (bounded, see
 * ftcj_batch_set_wait) for its cell's potential.  The k-mesh transforms and
 * Hermite maps run per cell on the streams before and after.  Every cell must
 * be split precision without per-pair cutoffs and with the walk contraction
 * (EUNSUPPORTED otherwise), all with or all without the orthorhombic X(n1)
 * table, and each call builds exactly params[c].max_dens densities of cell c
 * (EINVAL otherwise). */
#define FTCJ_BATCH_PERSISTENT 2
typedef struct ftcj_batch ftcj_batch;

/* cells/bases/params are arrays of ncell; kmeshes is [ncell][3]. */
int ftcj_batch_create(int ncell, const ftcj_cell* cells, const ftcj_basis* bases, const int* kmeshes,
                      const ftcj_params* params, int flags, ftcj_batch** out);

/* Per-cell sizes (as ftcj_plan_info). */
int ftcj_batch_info(const ftcj_batch* batch, int cell, ftcj_info* out);

/* Builds every cell: ndens[c] densities, device buffers Dk[c], Jk[c] (complex
 * [ndens][Nk][nao][nao]) and EJ[c] ([ndens]); pointer arrays on the host.
 * Asynchronous on `stream`. */
int ftcj_batch_jbuild(ftcj_batch* batch, const int* ndens, const double* const* Dk, double* const* Jk,
                      double* const* EJ, void* stream);

/* Captures one ftcj_batch_jbuild with these buffers into a CUDA graph held by
 * the batch (replacing any earlier one); nothing runs during the capture.
 * `stream` must not be capturing already and must not be the legacy default
 * stream. */
int ftcj_batch_capture(ftcj_batch* batch, const int* ndens, const double* const* Dk, double* const* Jk,
                       double* const* EJ, void* stream);

/* Launches the captured graph on `stream` (the buffers of the capture are
 * read and written again).  Errors: EINVAL if nothing was captured. */
int ftcj_batch_replay(ftcj_batch* batch, void* stream);

/* Persistent batches: a back-contraction item gives up waiting for its
 * cell's potential after 2^wait_log2 clock cycles (0: 2^32, about 2 s),
 * raises the batch's error word and skips its work.  0..40, else EINVAL. */
int ftcj_batch_set_wait(ftcj_batch* batch, int wait_log2);

/* The error word of the last persistent launch (bit 0: a wait gave up),
 * read on `stream` (synchronises it).  Returns FTCJ_ETIMEOUT when bit 0 is
 * set, FTCJ_OK otherwise (and for batches that are not persistent). */
int ftcj_batch_status(ftcj_batch* batch, int* flags, void* stream);

void ftcj_batch_destroy(ftcj_batch* batch);

/* Autotuner of the walk shape: builds the plan for every candidate
 * (chunk_points in {0 = the plan's default, 512, 1024, 2048, 4096} that hold
 * the longest G line, rho_blocks in {0 = the plan's own count, which fills
 * the GPU and may split the split-form walk by class, 2 x fill}; an explicit
 * value equal to the default is not tried twice), times ftcj_jbuild on a zero density
 * (the walks' cost does not depend on the values) with CUDA events, and
 * writes the fastest parameters to *out (and its time to *best_ms, may be
 * NULL).  Allocates and frees its own buffers; synchronises the device. */
int ftcj_autotune(const ftcj_cell* cell, const ftcj_basis* basis, const int kmesh[3], const ftcj_params* in,
                  ftcj_params* out, double* best_ms);

/* ---- measurement ---- */

/* Phases of one build batch, in launch order. */
#define FTCJ_PHASE_FOLD 0      /* a2: k -> BvK transform stages */
#define FTCJ_PHASE_HERMITE 1   /* a3: Hermite densities */
#define FTCJ_PHASE_RHO 2       /* a4: structure-factor walk */
#define FTCJ_PHASE_POTENTIAL 3 /* a5: row reduction, W and E_J */
#define FTCJ_PHASE_JWALK 4     /* a6: back-contraction walk */
#define FTCJ_PHASE_JAO 5       /* a7: transform to AOs (and the J^{0n} clear) */
#define FTCJ_PHASE_UNFOLD 6    /* a8: BvK -> k transform stages */
#define FTCJ_PHASE_GPW_RHO 7   /* classified plans, inside FTCJ_PHASE_RHO: the DD records' collocation on the
                                  grid and its transform onto the sphere (0 otherwise) */
#define FTCJ_PHASE_GPW_J 8     /* classified plans, inside FTCJ_PHASE_JWALK: the adjoint transform and the DD
                                  records' integration on the grid (0 otherwise) */
#define FTCJ_NPHASE 9
/* Phases 0..6 partition the build; 7 and 8 are parts of phases 2 and 4. */

/* Turn per-phase CUDA-event timing of ftcj_jbuild / ftcj_jbuild_host on
 * (max_batches > 0: events for that many batches are created now) or off
 * (0: events released).  Events are recorded on the build's stream. */
int ftcj_profile_enable(ftcj_plan* plan, int max_batches);

/* Sums of the per-phase device times (ms) over the batches recorded since
 * the last read, the number of batches, and the number of kernels the
 * library launched in them; waits for the recorded events and resets. */
int ftcj_profile_read(ftcj_plan* plan, double ms[FTCJ_NPHASE], int* batches, int64_t* launches);

/* Kernel launches of one build batch of nd densities (no launch happens). */
int ftcj_launches_per_batch(const ftcj_plan* plan, int nd, int64_t* launches);

/* Measured fused multiply-add throughput of this GPU in flop/s (2 per FMA):
 * precision 0 = FP64, 1 = FP32.  Runs a short register-resident FMA loop on
 * every SM and synchronises `stream`. */
int ftcj_probe_fma_peak(int precision, double* flops_per_s, void* stream);

/* ---- plan exports (host buffers, filled by the call) ---- */

/* n triples [ng_half][3] of the half sphere, in rho's storage order. */
int ftcj_get_gvectors(const ftcj_plan* plan, int* n_out);

/* Pair records [npairs][6]: group a, group b, L1, L2, L3, weight (1 for a
 * self pair, 2 when the record also stands for its mirror (b0, a-L)). */
int ftcj_get_pairs(const ftcj_plan* plan, int* out);

/* Primitive groups: centre[ngroup], exponent[ngroup], and the member list
 * [nmember][3] = (group, shell, primitive index); returns nmember through
 * *nmember (pass members = NULL to query). */
int ftcj_get_groups(const ftcj_plan* plan, int* centre, double* exponent, int* members, int* nmember);

const char* ftcj_strerror(int code);
const char* ftcj_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FTCJ_H */
