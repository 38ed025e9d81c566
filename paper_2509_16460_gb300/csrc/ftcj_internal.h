// Internal declarations of the GB300 long-range Coulomb library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ftcj.h"

namespace ftcj {

constexpr int kLmax = FTCJ_LMAX;           // highest shell l
constexpr int kLpair = 2 * kLmax;          // highest pair class L = l_a + l_b
constexpr int kNclass = kLpair + 1;        // classes 0..4
constexpr int kNcartMax = (kLmax + 1) * (kLmax + 2) / 2;
constexpr int kMaxTerms = (kLpair + 1) * (kLpair + 2) * (kLpair + 3) / 6;  // 35
constexpr int kTile = 128;                 // pair records per walker block
constexpr int kBatch = 32;                 // points per rho reduction batch
constexpr int kChunkMax = 4096;            // G points per walk chunk
constexpr int kRedPoints = 4;  // G points per block of the rho row reduction
constexpr int kSortTile = 1024;            // candidates per sort tile
// events of one profiled batch: the 8 bounds of phases 0..6, then the start
// and end of each of the two GPW phases
constexpr int kProfEvents = 12;
// The split walks form n^i and n2^j n3^k (i, j + k <= degree) as exact FP32
// integers: |n| <= 63 keeps degree 4 below 2^24, |n| <= 27 degree 5 (the
// gradient's sums).
constexpr int kSplitNmax = 63;
constexpr int kSplitGradNmax = 27;

__host__ __device__ constexpr int nterms(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int nmono(int lam) { return (lam + 1) * (lam + 2) / 2; }
__host__ __device__ constexpr int lam_offset(int lam) { return lam * (lam + 1) * (lam + 2) / 6; }
// position of the monomial (a, b, lam-a-b) of total degree lam, order a = lam..0, b = lam-a..0
__host__ __device__ inline int mono_index(int lam, int a, int b) {
    int idx = 0;
    for (int x = lam; x > a; --x) idx += lam - x + 1;
    return idx + (lam - a - b);
}

// A primitive group: one (centre, exponent) shared by one or more shells.
struct GroupDev {
    double x, y, z, alpha;
    int lmax, mem0, mem1, centre;
};

// One shell that uses a group's primitive.  coef already holds the contraction
// coefficient times the radial normalisation (2a/pi)^{3/4} (4a)^{l/2}.
struct MemberDev {
    int l, sph, ao, pad;
    double coef;
};

// A screened pair record (a in the home cell, b in cell L).
struct PairDev {
    int ga, gb;
    int L[3];
    int cell, mcell;  // BvK index of [L] and [-L]
    int weight;       // 1 self pair, 2 stands for its mirror too
    int cls;          // la_max + lb_max
    int pad;
    double P[3];
    double p;
    double K;         // exp(-mu |A-B-R_L|^2) (pi/p)^{3/2}
};

// Per-pair constants of the G walk (recurrence multipliers).
struct PairWalk {
    double c;             // 1/(4p)
    double f1, f2, f3;    // fractional coordinates of P, reduced to [-1/2, 1/2)
    double q1, q2, q3;    // exp(-2c M_ii)
    double x12, y12, x13, y13, x23, y23;  // exp(-/+ 2c M_ij)
    double e1r, e1i, e2r, e2i, e3r, e3i;  // exp(-2 pi i f_j)
    double pad;
};

// One G line along b_1 at fixed (n2, n3) in the walk, with the transition
// from the previous line of the same chunk.
enum : int { OP_FIRST = 0, OP_N2F = 1, OP_NEGSTART = 2, OP_N2B = 3, OP_N3 = 4 };
struct WLine {
    int n2, n3, lo, hi, op, pt;  // pt: index of the line's first stored point
    float qa, qb, qc;            // |G|^2 = qa n1^2 + 2 qb n1 + qc along the line
};
struct WChunk {
    int l0, l1, p0, p1;  // lines [l0,l1), points [p0,p1)
};

struct Tile {
    int cls, first, count;  // pairs [first, first+count) of one class
    float gcut2;            // squared G radius the tile walks (per-pair cutoffs), else +inf
};

// Per-class layout of the Hermite-term arrays (SoA within each class).
struct MapLayout {
    long long start[kNclass + 1];
    long long base[kNclass];
    long long total;
};

// Flattened thread ranges of a per-record kernel: class c owns threads
// [tstart[c], tstart[c+1]), slots[c] threads per record from record rstart[c].
struct MapThreads {
    long long tstart[kNclass + 1];
    long long rstart[kNclass];
    int slots[kNclass];
};

// Record-major blocks of one class (the split form's map kernels): class c
// owns blocks [bstart[c], bstart[c+1]), each holding `per` whole records of
// `width` threads and `stage` shared values per record.
struct RecBlocks {
    long long rstart[kNclass];
    long long rcount[kNclass];
    int bstart[kNclass + 1];
    int per[kNclass];
    int width[kNclass];
    int stage[kNclass];
};

// Where the split form's Hermite-term map writes D'_t: with pos == nullptr the
// per-class SoA layout in record order (MapLayout); else the tensor-core
// layout [dens][class c][term t][position], the position of a record within
// its class given by pos (the contraction's K order), the class's stride
// rounded up to 16 entries so that every 16 consecutive positions of a term
// are one aligned 128-byte row.
struct TermDest {
    const int* pos;
    long long base[kNclass];
    long long stride[kNclass];
    long long total;
};

// Per-cell constants, passed to kernels by value (so plans of different cells
// can be alive and used together).
struct CellConst {
    double A[9];     // rows a_i
    double Bt[9];    // rows b_i / (2 pi)
    double M6[6];    // metric b_i.b_j: M11, M22, M33, M12, M13, M23
    double bn[3];    // |b_i|
    double vpar[2];  // 4 pi / Omega, 1 / (4 w^2)
    int km[3];
    int pad;
};

struct Gpw;

}  // namespace ftcj

struct ftcj_plan {
    // geometry and parameters
    double A[9], B[9], M[9];
    double vol, omega, gcut;
    int km[3], nk;
    ftcj_params params;
    int max_dens;
    // basis
    int nao, nshell, ngroup, nmember, ncentre;
    std::vector<ftcj::GroupDev> groups;
    std::vector<ftcj::MemberDev> members;
    std::vector<int> member_shell, member_prim, member_group;
    // walk
    std::vector<ftcj::WLine> lines;
    std::vector<ftcj::WChunk> chunks;
    std::vector<int> gvec;  // [ng_half][3]
    int64_t ng_half;
    int chunk_max;        // G points per walk chunk (a plan parameter)
    int max_chunk_pts;
    int n1_min, n1_max;
    int n_abs_max;  // largest |n_i| of the sphere's G = sum_i n_i b_i
    // pairs
    int64_t npairs, npairs_ordered;
    int shard_count = 1, shard_index = 0;  // record-sharded plan: share shard_index of shard_count
    int64_t class_start[ftcj::kNclass + 1];
    int64_t term_base[ftcj::kNclass];  // SoA offset of each class in a per-density term array
    int64_t total_terms;
    int64_t term_base_g[ftcj::kNclass];  // gradient: terms of degree class + 1
    int64_t total_terms_g;
    std::vector<ftcj::Tile> tiles;  // ordered by decreasing class
    int npb;                         // rho pass: blocks per (chunk, density)
    int num_sms;
    // device buffers
    ftcj::GroupDev* d_groups = nullptr;
    ftcj::MemberDev* d_members = nullptr;
    ftcj::PairDev* d_pairs = nullptr;
    ftcj::PairWalk* d_walk = nullptr;
    ftcj::WLine* d_lines = nullptr;
    ftcj::WChunk* d_chunks = nullptr;
    ftcj::Tile* d_tiles = nullptr;
    int* d_sched = nullptr;
    std::vector<int> rho_sched;  // rho pass: npb+1 offsets, then tile ids grouped by block
    float* d_rec_gcut = nullptr;     // per-record G cutoff (pair_gcut_eps > 0)
    int ntiles_hi = 0;               // leading tiles of classes 3-4 (split J walk launches them apart)
    int rho_hi_tiles = 0, npb_hi = 0;  // the same for the split rho walk, and the blocks of its first launch
    cudaStream_t aux = nullptr;      // second stream of the split J walk (fork/join by events)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t units_screened = 0, units_walked = 0;
    std::vector<int64_t> tile_npts;  // half-sphere points inside each tile's radius (cutoffs on)
    int* d_gvec = nullptr;
    double* d_vg = nullptr;          // v(G) on the half sphere
    double* d_tw = nullptr;          // twiddles, [3][16][16] complex
    double* d_Tmat = nullptr;        // relative-coordinate transforms, per lambda
    double* d_D0n = nullptr;         // [max_dens][nk][nao][nao]
    double* d_J0n = nullptr;
    double* d_cbuf0 = nullptr;       // complex [max_dens][nk][nao][nao]
    double* d_cbuf1 = nullptr;
    double* d_Dp = nullptr;          // [max_dens][total_terms]
    double* d_Jp = nullptr;          // [max_dens][nchunks][total_terms]
    double* d_Jg = nullptr;          // [max_dens][nchunks][total_terms_g] (gradient sums)
    double* d_maps = nullptr;        // per-record maps AO block -> D'_ijk, see hmap.cu
    long long* d_map_off = nullptr;  // [npairs + 1]
    long long map_doubles = 0;
    ftcj::MapThreads mt_terms, mt_outs;
    ftcj::RecBlocks rb_terms, rb_outs;  // a3 / a7 blocks of the double-float maps
    bool maps_df = false;               // maps stored as double-float (split form)
    size_t rb_terms_smem = 0, rb_outs_smem = 0;
    double* d_rho_part = nullptr;    // complex [max_dens][npb][ng_half]
    double* d_rho = nullptr;         // complex [max_dens][ng_half]
    double* d_W = nullptr;           // complex [max_dens][ng_half]
    double* d_Epart = nullptr;       // [max_dens][nEblocks]
    double* d_Dk_stage = nullptr;    // host-variant staging, complex [max_dens][nk][nao][nao]
    double* d_Jk_stage = nullptr;
    double* d_EJ_stage = nullptr;
    double* d_check = nullptr;       // [2]
    void* d_split_init = nullptr;    // split form: walk state at each chunk start, [nchunks][npairs]
    void* d_split_const = nullptr;   // split form: recurrence multipliers, [npairs]
    // tensor-core separable contraction of the structure-factor pass (tc.cu)
    bool tc = false;
    int tc_axis[3] = {0, 1, 2};  // row axes a, b and the column axis c
    int tc_ncols = 0, tc_nd = 0, tc_npad = 0;  // n_c = 0..ncols-1; densities per launch; MMA N
    int tc_colw = 0, tc_G = 0;                 // real columns per (i, j) block; blocks per window
    int tc_rows = 0, tc_mtiles = 0, tc_nna = 0, tc_nnb = 0, tc_tabw = 0;
    int64_t tc_nkappa = 0;
    int tc_nwin = 0, tc_wpg = 0, tc_ngroups = 0;  // K windows, windows per group, groups (partial rows)
    int tc_tslots = 0;                            // stage-table slots in shared memory
    int64_t tc_mma_flops = 0;                     // bf16 MMA flops of one pass over max_dens densities
    void* d_tc_rows = nullptr;   // int2 [rows]
    int* d_tc_map = nullptr;     // [rows][ncols]
    int* d_tc_kappa = nullptr;   // [nwin * 512] record ids of each window
    int* d_tc_wpairs = nullptr;  // (i | j << 3) of the windows' blocks
    void* d_tc_winfo = nullptr;  // int4 [nwin]: class, blocks, first block
    void* d_tc_tab = nullptr;    // float4 [npairs][tabw]
    float* d_tc_cl = nullptr;    // [npairs]
    int* d_tc_err = nullptr;     // device error word of the bounded waits
    int* d_tc_pos = nullptr;     // [npairs]: position of each record in its class's K order
    int* d_tc_ebw = nullptr;     // [nwin][128]: the windows' column scales, per build
    float* d_tc_clw = nullptr;   // [nwin]: the windows' smallest widths
    long long tc_dp_base[ftcj::kNclass] = {}, tc_dp_stride[ftcj::kNclass] = {}, tc_dp_total = 0;
    // tensor-core form of the back-contraction (tc.cu); false: the split walk runs it
    bool tc_j = false;
    int tc_jnd = 0, tc_jgw = 0, tc_jG = 0, tc_jnpad = 0;  // densities per launch, columns per density, blocks per item, MMA N
    int tc_jnstage = 0, tc_jnitems = 0;                     // 8-row stages, work items
    int tc_jparts = 0, tc_jspp = 0;                         // row parts (one exact accumulation each), stages per part
    int64_t tc_j_mma_flops = 0;                             // bf16 MMA flops of one pass over max_dens densities
    void* d_tc_jitems = nullptr;  // int4 [items]: class, blocks, first block, first record
    int* d_tc_jpairs = nullptr;   // (i | j << 3) of the items' blocks
    void* d_tc_vs = nullptr;      // bf16 sliced V_ij stage tiles
    int* d_tc_ev = nullptr;       // their column scales
    int rho_rows = 0;            // partial rows the rho reduction sums (walk blocks or tensor-core groups)
    // density classification (Sec. 2.6): the records a plan keeps (0 all, 1 compact, 2 DD)
    int rec_filter = 0;
    double alpha_cut = 0.0;
    ftcj_plan* dd = nullptr;   // the DD records (GPW route): a plan of their own over the same basis
    ftcj::Gpw* gpw = nullptr;  // GPW grid, transforms and buffers (gpw.cu)
    int jp_fixed = 0;          // > 0: partial J' arrays the J -> AO map sums, whatever the walk
    int precision = FTCJ_PREC_FP64;
    bool ortho = false;  // reciprocal metric diagonal (orthorhombic cell)
    ftcj::CellConst cc;
    int nEblocks = 0;
    size_t device_bytes = 0;
    // per-phase event timing (ftcj_profile_enable)
    std::vector<cudaEvent_t> prof_events;  // [max_batches][kProfEvents]
    int prof_max = 0, prof_used = 0;
    int64_t prof_launches = 0;
};

namespace ftcj {

// error reporting (thread-local message)
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define FTCJ_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ::ftcj::cuda_fail(e_, #call); \
    } while (0)

// Lets `func` use up to the device's opt-in shared memory per block (the
// attribute is per kernel, shared by every plan, so it is never lowered) and
// fails with EUNSUPPORTED if `need` bytes exceed that maximum.
int allow_dynamic_smem(const void* func, size_t need);

// --- setup (screen.cu) ---
int screen_and_sort(ftcj_plan* P);  // fills pairs, walk constants, tiles

// --- fold / unfold (fold.cu) ---
int launch_fold(ftcj_plan* P, int ndens, const double* Dk, double* D0n, cudaStream_t s);
int launch_fold_build(ftcj_plan* P, int ndens, const double* Dk, double* D0n, cudaStream_t s);  // Hermitian D^k
int launch_unfold(ftcj_plan* P, int ndens, const double* J0n, double* Jk, cudaStream_t s);
int launch_check_density(ftcj_plan* P, int ndens, const double* Dk, double* out2, cudaStream_t s);
int launch_twiddles(ftcj_plan* P);
int setup_fold(ftcj_plan* P);
int fused_fold_supported(const ftcj_plan* P);

// --- Hermite densities and J back-transform (hermite.cu) ---
int upload_hermite_tables(ftcj_plan* P);
int launch_grad_assemble(ftcj_plan* P, int ndens, const double* D0n, double* grad, cudaStream_t s);
void host_hermite_tables(const ftcj_plan* P, std::vector<double>& U, std::vector<int>& cart, std::vector<int>& Toff);

// --- per-record maps of the Hermite-density contraction (hmap.cu) ---
int build_maps(ftcj_plan* P);
int launch_hermite_map(ftcj_plan* P, int ndens, const double* D0n, cudaStream_t s);
int launch_jtransform_map(ftcj_plan* P, int ndens, double* J0n, cudaStream_t s, bool zero = true);

// --- G walks (walk.cu) ---
int upload_walk_tables(ftcj_plan* P);
int launch_vg(ftcj_plan* P);
int launch_rho_walk(ftcj_plan* P, int ndens, cudaStream_t s);
int launch_rho_reduce(ftcj_plan* P, int ndens, double* rho_out, double* W_out, double* EJ_out,
                      const double* rho_in, cudaStream_t s);
int launch_j_walk(ftcj_plan* P, int ndens, const double* W, cudaStream_t s);
int launch_j_walk_grad(ftcj_plan* P, int ndens, const double* W, cudaStream_t s);
int rho_walk_blocks_per_sm(ftcj_plan* P, int* out);

// --- split-precision walks (walk_split.cu) ---
int setup_split(ftcj_plan* P);
int split_xtab_entries(const ftcj_plan* P);  // 0 when the split walks run the n1 recurrence
size_t split_rho_smem(const ftcj_plan* P, int part);  // shared memory of one split structure-factor block (part: 0 all classes, 1 classes 0-2)
int launch_pair_gcut(ftcj_plan* P);      // per-record cutoffs from the (double) maps, in build_maps
int apply_pair_cutoffs(ftcj_plan* P);
int keep_record_share(ftcj_plan* P);
void shard_bounds(const int64_t* class_counts, int precision, int shard_count, int64_t* bounds);    // sort records by cutoff within each class, radius per tile
int rho_walk_split_blocks_per_sm(ftcj_plan* P, int part, int* out);  // part: 0 all, 1 classes 0-2, 2 classes 3-4
int launch_rho_walk_split(ftcj_plan* P, int ndens, cudaStream_t s);
int launch_j_walk_split(ftcj_plan* P, int ndens, const double* W, cudaStream_t s);
int launch_j_walk_grad_split(ftcj_plan* P, int ndens, const double* W, cudaStream_t s);
bool split_grad_walk_exact(const ftcj_plan* P);

// --- tensor-core separable contraction (tc.cu) ---
int setup_tc(ftcj_plan* P);
int launch_tc_rho(ftcj_plan* P, int ndens, cudaStream_t s);
int tc_rho_launches(const ftcj_plan* P, int nd);
int launch_tc_j(ftcj_plan* P, int ndens, const double* W, cudaStream_t s);
// one persistent launch of the walks of a batch of cells (walk_split.cu)
struct BatchWalks;
int batch_walks_create(const std::vector<ftcj_plan*>& plans, BatchWalks** out);
int batch_walks_launch(BatchWalks* bw, const std::vector<ftcj_plan*>& plans, long long spin, cudaStream_t s);
int batch_walks_error(BatchWalks* bw, int* word, cudaStream_t s);
int batch_walks_launches(const BatchWalks* bw);
void batch_walks_destroy(BatchWalks* bw);
int tc_j_launches(const ftcj_plan* P, int nd);
// partial back-contraction sums the J -> AO map adds: one per walk chunk, or per row part of the tensor-core form
inline int jp_chunks(const ftcj_plan* P) {
    return P->jp_fixed > 0 ? P->jp_fixed : (P->tc_j ? P->tc_jparts : (int)P->chunks.size());
}

// --- GPW route of the DD pair densities (gpw.cu) ---
int setup_gpw(ftcj_plan* P);  // after the compact plan is built: P->dd, the grid and its buffers
void free_gpw(ftcj_plan* P);
int launch_gpw_rho(ftcj_plan* P, int ndens, cudaStream_t s);  // rho_D(G) from P->dd's Hermite terms
int launch_gpw_potential(ftcj_plan* P, int ndens, double* EJ, cudaStream_t s);  // W_C into P->d_W, W_D, E_J
int launch_gpw_j(ftcj_plan* P, int ndens, cudaStream_t s);  // J' of the DD records into P->dd->d_Jp
int gpw_launches(const ftcj_plan* P, int ndens);
int gpw_grid_dim(const ftcj_plan* P, int axis);
int gpw_separable(const ftcj_plan* P);

// --- measurement (profile.cu) ---
void release_profiling(ftcj_plan* P);
int64_t launches_per_batch(const ftcj_plan* P);
int split_j_launches(const ftcj_plan* P);  // kernel launches of one split J walk (1 or 2)

}  // namespace ftcj
