// Tensor-core form of the structure-factor pass (Alg. 1) for orthorhombic
// cells.
//
// In an orthorhombic cell the pair prefactor factorises over the three axes
// (Sec. 2.4, the orthorhombic fully separable case; App. D):
//   exp(-|G|^2/4p) exp(-i G.P) = X(n_a) Y(n_b) Z(n_c),
//   X(n) = exp(-c M_aa n^2) exp(-2 pi i f_a n),   c = 1/(4p),
// f_a the fractional coordinate of the pair centre.  With a pair record's
// Hermite densities D'_{ijk} (the walks' convention: the record adds
// X Y Z sum_ijk D'_ijk (-i n_a)^i (-i n_b)^j (-i n_c)^k to rho(n)),
//   rho(n_a, n_b, n_c) = sum_{(i,j)} P_ij(n_a, n_b) sum_r A[(n_a, n_b), r] B_ij[r, n_c]
//   A = X_r(n_a) Y_r(n_b)                              (geometry only)
//   B_ij = Z_r(n_c) sum_k D'_{r,ijk} (-i n_c)^k         (per density)
//   P_ij = (-i n_a)^i (-i n_b)^j                        (exact small integers)
// For the records of one class L, all (i, j) with i + j <= L share A, so the
// column blocks B_ij (up to G of them side by side) form one complex matrix
// product over K = records: rows are the (n_a, n_b) of the sphere's
// projection, columns (i, j) x n_c >= 0 x densities (the stored half sphere
// maps to n_c >= 0, through -n and a conjugate where n_c < 0).  The powers
// P_ij are applied to each block's sums when tensor memory is drained, so
// that A carries only the Gaussian and the phase: a row's entries over a
// window of records sorted by their width differ little in size, which is
// what keeps the slicing below at full relative precision.
//
// Precision.  bf16 products summed in FP32 carry 8 bits; the target is FP64-
// class.  The operands are therefore split after Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012): every row
// of A and every column of B, over a window of 512 records, gets a
// power-of-two scale 2^e bounding its entries, and each entry is cut into six
// slices m_s 2^{e-6-7s} with integers |m_s| <= 64.  Slice s of A times slice t
// of B is a tcgen05.mma of kind::f16 (bf16 operands, FP32 accumulator in
// tensor memory); products with s + t <= 5 are formed (21 per k-step), the
// others fall below 2^-40 of the window's scale.  Products of the same level
// s + t land in one accumulator: levels 0, 1, 2 are exact integer sums
// (|m| <= 64, at most 3 products per level and 1024 real K terms per window
// keep every partial sum below 2^24), levels 3..5 share a fourth, rounded
// accumulator.  At each window's end the accumulators are scaled by
// 2^{eA+eB}, multiplied by P_ij and added in double-float (FP32 pairs,
// df.cuh) to sums kept in tensor memory, which are written as FP64 partial
// rows and summed across window groups in fixed order by the row reduction.
//
// Kernel shape (one CTA per SM: 512 tensor-memory columns and ~200 KB of
// shared memory), thirteen warps: warps 0-10 form the operand slices of a
// 16-record stage into one of two shared-memory buffers (plain 16-byte stores
// in the no-swizzle K-major core-matrix layout the MMA descriptors name);
// lane 0 of warp 11 issues the MMAs; warp 12 stages each stage's record
// factor tables with bulk copies (cp.async.bulk, completion counted in bytes
// on an mbarrier) and their Hermite terms into a ring of shared-memory slots
// ahead of use.  Warps 0-11 also compute the window scales and drain tensor
// memory.  Stages are handed over with mbarriers (arrivals; tcgen05.commit
// for the MMA side).  Every wait is bounded: past ~2 s of clock a waiting
// thread raises the CTA's abort flag and the plan's device error word, every
// thread leaves its loops, the copies and MMAs in flight are waited for
// (again bounded) and tensor memory is freed before the CTA exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <set>
#include <vector>

#include "df.cuh"
#include "ftcj_internal.h"

namespace ftcj {
namespace {

constexpr int kTcM = 128;                      // rows per tile (MMA M)
constexpr int kTcStageK = 16;                  // records per stage: two MMA k-steps of 16 real (re, im)
constexpr int kTcWin = 512;                    // records per exact-accumulation window (1024 real K)
constexpr int kTcStagesPerWin = kTcWin / kTcStageK;
constexpr int kTcNmma = 256;                   // MMA N at most
constexpr int kTcS = 6;                        // slices per operand
constexpr int kTcAcc = 4;                      // accumulators: levels 0, 1, 2 exact, levels 3..5 rounded
constexpr int kTcTmemCols = 512;
constexpr int kTcGmax = 15;                    // (i, j) blocks per window at most (class 4 has 15)
constexpr int kTcEbMax = 128;                  // column scales per window at most
constexpr int kTcNbuf = 2;                     // stage buffers
constexpr int kTcTabSlotsMax = 4;              // stage tables in flight
constexpr int kTcAsliceBytes = kTcM * 2 * kTcStageK * 2;  // 128 rows x 32 real K x bf16
constexpr long long kTcSpinCycles = 1LL << 32;            // ~2 s of SM clock per wait

struct TcArgs {
    const int2* rows;    // (n_a, n_b) per row
    const int* map;      // [rows][ncols]: half-sphere index, ~index where the stored point is -n, INT_MIN none
    const int* wrec;     // [nwin][kTcWin]: record ids of each window, -1 for padding
    const int4* winfo;   // [nwin]: class L, number of (i,j) blocks, first block index into wpairs,
                         // position of the window's first record in its class's K order
    const int* wpairs;   // (i | j << 3) of each block
    const float4* tab;   // per record [tabw]: X(0..), Y(0..), Z(0..) as complex double-float
    const float* cl;     // per record c log2(e)
    const float2* Dp;    // Hermite densities (double-float) in the K order: [dens][class][term][position]
    long long dp_total;
    long long dp_base[kNclass];
    long long dp_stride[kNclass];
    double2* out;        // partial rows [dens][ngroups][ng_half]
    long long ng_half;
    int* err;            // device error word (bit 0: a bounded wait gave up)
    float Maa, Mbb, Mcc;
    int ax, bx, cx;      // lattice axes of the row indices (a, b) and of the column index (c)
    int tabw, offY, offZ;
    int ncols;           // complex columns per density and block: n_c = 0 .. ncols-1
    int nd, d0;          // densities of this launch, first density
    int colw;            // real columns per block: 2 nd ncols
    int G;               // blocks per window at most
    int npad;            // MMA N: G colw rounded up to 16
    int accw;            // real columns of the double-float sums: colw rounded up to 8
    int nwin, win_per_group, ngroups;
    int nrows;
    long long spin;      // clock cycles a wait between roles may take before it gives up
    int* ebw;            // [nwin][kTcEbMax]: column scales of each window (k_tc_rho_bounds)
    float* clw;          // [nwin]: smallest c log2(e) of each window's records
};

// ---- PTX wrappers -----------------------------------------------------------

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of b to complete; false when it gave up (after
// ~2 s of clock, or because another thread of the CTA already did).
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, long long spin) {
    const long long t0 = clock64();
    while (!mbar_test(b, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > spin) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// A bounded barrier of the eight operand warps (an mbarrier counting one
// arrival per warp): unlike bar.sync it cannot hang when a thread has left
// after a failed wait.  The outcome is the same for every lane of a warp.
__device__ bool prod_sync(uint64_t* b, uint32_t& ph, volatile int* abort_flag, int lane, long long spin) {
    __syncwarp();
    if (lane == 0) mbar_arrive(b);
    const bool ok = mbar_wait(b, ph, abort_flag, spin);
    ph ^= 1u;
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, no swizzle, core matrices of 8
// rows x 16 B; K-adjacent core matrices 128 B apart (leading byte offset),
// 8-row groups 512 B apart (stride byte offset: 32 real K per stage row)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
                 : "memory");
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- operand slices ---------------------------------------------------------

// 2^k for an exponent in the normal FP32 range (k clamped to it)
__device__ __forceinline__ float pow2f(int k) {
    k = max(-126, min(127, k));
    return __int_as_float((k + 127) << 23);
}

// Slices of x = hi + lo (|x| < 2^e, sc = 2^(6-e)): o[s] = m_s 2^(-7s) with
// integers |m_s| <= 64 (<= 72 for s = 3, which takes the low part's
// rounding), so that x = 2^(e-6) sum_s o[s] up to 2^(e-41).  Each slice rounds
// the remainder to a multiple of 2^(-7s) by adding and subtracting 1.5 x
// 2^(23-7s) (round to nearest even, no fast-math reassociation); slices 0-2
// peel the high part exactly, the low part joins at slice 3 with one rounding
// below 2^(e-45).
__device__ __forceinline__ void slice6(float hi, float lo, float sc, float (&o)[kTcS]) {
    float h = hi * sc;
    const float l = lo * sc;
    o[0] = (h + 0x1.8p23f) - 0x1.8p23f;
    h -= o[0];
    o[1] = (h + 0x1.8p16f) - 0x1.8p16f;
    h -= o[1];
    o[2] = (h + 0x1.8p9f) - 0x1.8p9f;
    h = (h - o[2]) + l;
    o[3] = (h + 0x1.8p2f) - 0x1.8p2f;
    h -= o[3];
    o[4] = (h + 0x1.8p-5f) - 0x1.8p-5f;
    h -= o[4];
    o[5] = (h + 0x1.8p-12f) - 0x1.8p-12f;
}

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // exact: every slice has <= 8 significant bits
    return *reinterpret_cast<uint32_t*>(&v);
}

// element offset of (row, k) in a stage tile [rows][32 real K] of core matrices
__device__ __forceinline__ int tile_off(int row, int k) {
    return (((row >> 3) * 4 + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// (-i)^p z
__device__ __forceinline__ cdf rot_mi(cdf z, int p) {
    switch (p & 3) {
        case 0: return z;
        case 1: return cdf{z.im, df_neg(z.re)};
        case 2: return cdf{df_neg(z.re), df_neg(z.im)};
        default: return cdf{df_neg(z.im), z.re};
    }
}

__device__ __forceinline__ int exp_bound(float log2_bound) {
    // smallest e with 2^e > the bound, from a log2 estimate good to ~1e-4
    if (!(log2_bound > -100.f)) return -100;
    return (int)floorf(log2_bound + 1e-3f) + 1;
}

struct TcRow {
    int na, nb;
    float Q;  // M_aa na^2 + M_bb nb^2
};

struct TcSmem {
    int rec[kTcWin];
    int pairs[kTcGmax];
    int tidx[kTcGmax][5];  // index of D'_{ijk} for block (i, j) and k = 0..4 (-1 past the class's degree)
    int eA[kTcM];
    int eB[kTcEbMax];
    TcRow rowi[kTcM];
    int winL, wnpair, wpos, clmin_bits;
    uint64_t full[kTcNbuf], empty[kTcNbuf], accf, acce, done, psync;
    uint64_t tfull[kTcTabSlotsMax], tempty[kTcTabSlotsMax];
    uint32_t tmem;
    int abort_flag;
};

// One table slot of a stage: the 16 records' factor tables (copied whole by
// the bulk-copy engine, tabw float4 each), then the Hermite terms D'_{ijk} of
// the 16 records as rows [block][density][k = 0..4][record] (one 128-byte
// bulk copy per row; rows past the block's degree are not written or read).
__host__ __device__ inline size_t tab_slot_bytes(int tabw, int G, int nd) {
    const size_t b = (size_t)kTcStageK * tabw * 16 + (size_t)G * nd * 5 * kTcStageK * 8;
    return (b + 127) / 128 * 128;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t tx) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(saddr(b)),
                 "r"(tx)
                 : "memory");
}

// index of D'_{p1 p2 p3} (powers of n_1, n_2, n_3) for powers (i, j, k) of (n_a, n_b, n_c)
__device__ __forceinline__ int term_of(const TcArgs& g, int i, int j, int k) {
    const int p1 = g.ax == 0 ? i : (g.bx == 0 ? j : k);
    const int p2 = g.ax == 1 ? i : (g.bx == 1 ? j : k);
    const int lam = i + j + k;
    return lam_offset(lam) + mono_index(lam, p1, p2);
}

// A: the four records of group gg (stage-local 4 gg .. 4 gg + 3) for one row,
// X_r(n_a) Y_r(n_b) sliced, as six 16-byte stores (one core-matrix row per slice)
__device__ __forceinline__ void form_a(const TcArgs& g, const TcSmem& sm, const float4* tabs, int q, int row,
                                       int gg, float scA, unsigned char* as) {
    const TcRow ri = sm.rowi[row];
    const bool rvalid = ri.na != INT_MIN;
    const float sa = ri.na < 0 ? -1.f : 1.f, sb = ri.nb < 0 ? -1.f : 1.f;  // X(-n) = conj X(n)
    const int ia = abs(ri.na), ib = g.offY + abs(ri.nb);
    float sl[kTcS][8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int kq = gg * 4 + u;
        cdf a{{0.f, 0.f}, {0.f, 0.f}};
        if (rvalid && sm.rec[q * kTcStageK + kq] >= 0) {
            const float4 xv = tabs[kq * g.tabw + ia], yv = tabs[kq * g.tabw + ib];
            a = cdf_mul(cdf{{xv.x, xv.y}, {sa * xv.z, sa * xv.w}}, cdf{{yv.x, yv.y}, {sb * yv.z, sb * yv.w}});
        }
        float sr[kTcS], si[kTcS];
        slice6(a.re.hi, a.re.lo, scA, sr);
        slice6(a.im.hi, a.im.lo, scA, si);
#pragma unroll
        for (int s = 0; s < kTcS; ++s) {
            sl[s][2 * u] = sr[s];
            sl[s][2 * u + 1] = si[s];
        }
    }
    const int off = tile_off(row, gg * 8);
#pragma unroll
    for (int s = 0; s < kTcS; ++s) {
        uint4 v;
        v.x = pack_bf2(sl[s][0], sl[s][1]);
        v.y = pack_bf2(sl[s][2], sl[s][3]);
        v.z = pack_bf2(sl[s][4], sl[s][5]);
        v.w = pack_bf2(sl[s][6], sl[s][7]);
        *reinterpret_cast<uint4*>(as + (size_t)s * kTcAsliceBytes + (size_t)off * 2) = v;
    }
}

// B: four records (stage-local 4 kg .. 4 kg + 3) of one (block gb, output pair
// p = n_c nd + d), sliced, in the real form rows (record, re) -> [Re B | Im B],
// (record, im) -> [-Im B | Re B]: columns gb colw + 2p and + 1, one 16-byte
// core-matrix row per slice and column.  Blocks past the window's count are zero.
__device__ __forceinline__ void form_b(const TcArgs& g, const TcSmem& sm, const float4* tabs, const float2* dps,
                                       int q, int kg, int gb, int p, unsigned char* bs, int bslice) {
    const int nc = p / g.nd, d = p - nc * g.nd;
    float s0[kTcS][8], s1[kTcS][8];  // column 2p: (Re, -Im) per record; column 2p + 1: (Im, Re)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int kq = kg * 4 + u;
        cdf bv{{0.f, 0.f}, {0.f, 0.f}};
        if (gb < sm.wnpair && sm.rec[q * kTcStageK + kq] >= 0) {
            const float4 zv = tabs[kq * g.tabw + g.offZ + nc];
            const float2* dv = dps + (gb * g.nd + d) * 5 * kTcStageK + kq;
            const int pr = sm.pairs[gb], nk = sm.winL - (pr & 7) - (pr >> 3);  // k = 0 .. L - i - j
            df re{0.f, 0.f}, im{0.f, 0.f};
            float pw = 1.f;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) {
                if (kk > nk) break;
                const float2 v = dv[kk * kTcStageK];
                const df term = df_mulf(df{v.x, v.y}, pw);  // D'_k n_c^k, exact power
                switch (kk & 3) {                           // (-i)^k
                    case 0: re = df_add(re, term); break;
                    case 1: im = df_sub(im, term); break;
                    case 2: re = df_sub(re, term); break;
                    default: im = df_add(im, term); break;
                }
                pw *= (float)nc;
            }
            bv = cdf_mul(cdf{{zv.x, zv.y}, {zv.z, zv.w}}, cdf{re, im});
        }
        const float scB = pow2f(6 - sm.eB[gb * g.ncols * g.nd + p]);
        float sr[kTcS], si[kTcS];
        slice6(bv.re.hi, bv.re.lo, scB, sr);
        slice6(bv.im.hi, bv.im.lo, scB, si);
#pragma unroll
        for (int s = 0; s < kTcS; ++s) {
            s0[s][2 * u] = sr[s];
            s0[s][2 * u + 1] = -si[s];
            s1[s][2 * u] = si[s];
            s1[s][2 * u + 1] = sr[s];
        }
    }
    const int c0 = gb * g.colw + 2 * p;
    const int o0 = tile_off(c0, kg * 8), o1 = tile_off(c0 + 1, kg * 8);
#pragma unroll
    for (int s = 0; s < kTcS; ++s) {
        uint4 v;
        v.x = pack_bf2(s0[s][0], s0[s][1]);
        v.y = pack_bf2(s0[s][2], s0[s][3]);
        v.z = pack_bf2(s0[s][4], s0[s][5]);
        v.w = pack_bf2(s0[s][6], s0[s][7]);
        *reinterpret_cast<uint4*>(bs + (size_t)s * bslice + (size_t)o0 * 2) = v;
        v.x = pack_bf2(s1[s][0], s1[s][1]);
        v.y = pack_bf2(s1[s][2], s1[s][3]);
        v.z = pack_bf2(s1[s][4], s1[s][5]);
        v.w = pack_bf2(s1[s][6], s1[s][7]);
        *reinterpret_cast<uint4*>(bs + (size_t)s * bslice + (size_t)o1 * 2) = v;
    }
}

constexpr int kTcProdWarps = 14;
constexpr int kTcProdThreads = kTcProdWarps * 32;
constexpr int kTcMmaWarp = 14;
constexpr int kTcLoadWarp = 15;
constexpr int kTcWarps = 16;
constexpr int kTcEpiWarps = 12;
constexpr int kTcEpiThreads = kTcEpiWarps * 32;
constexpr int kTcThreadsAll = kTcWarps * 32;
constexpr int kTcTasksMax = 3;        // operand tasks per thread and stage: (512 + 4 G npo) / 448 <= 3
constexpr int kTcTaskA = 1 << 20;     // task flag: an A task (row | group << 7), else a B task

// Per window (one block each), once per build and density group: the
// window's smallest width c (every row of A gets the scale exp(-c_min Q))
// and the column scales of B, |B_ij| <= exp(-c Mcc n^2) sum_k |D'_ijk| n^k,
// maximised over the window's records, per (block, n_c, density).
__global__ void __launch_bounds__(256) k_tc_rho_bounds(TcArgs g) {
    __shared__ int eB[kTcEbMax];
    __shared__ int tidx[kTcGmax][5];
    __shared__ int clmin_bits;
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int4 wi = __ldg(g.winfo + w);
    const int L = wi.x, npair = wi.y, npo = g.nd * g.ncols;
    for (int i = tid; i < kTcEbMax; i += blockDim.x) eB[i] = -100;
    if (tid == 0) {
        for (int b = 0; b < npair; ++b) {
            const int pr = __ldg(g.wpairs + wi.z + b), i = pr & 7, j = pr >> 3;
            for (int kk = 0; kk < 5; ++kk) tidx[b][kk] = kk <= L - i - j ? term_of(g, i, j, kk) : -1;
        }
        clmin_bits = __float_as_int(INFINITY);
    }
    __syncthreads();
    const long long cnt = g.dp_stride[L];
    const float2* dpL = g.Dp + g.dp_base[L];
    float cmin = INFINITY;
    for (int k = tid; k < kTcWin; k += blockDim.x) {  // warp-uniform trip count (512 / 256)
        const int r = __ldg(g.wrec + (size_t)w * kTcWin + k);
        const float cr = r >= 0 ? __ldg(g.cl + r) : 0.f;
        if (r >= 0) cmin = fminf(cmin, cr);
        const long long loc = wi.w + k;
        for (int gb = 0; gb < npair; ++gb) {
            for (int d = 0; d < g.nd; ++d) {
                float cm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                if (r >= 0) {
                    const float2* dp = dpL + (long long)(g.d0 + d) * g.dp_total + loc;
#pragma unroll
                    for (int kk = 0; kk < 5; ++kk) {
                        const int t = tidx[gb][kk];
                        if (t >= 0) cm[kk] = fabsf(__ldg(dp + (long long)t * cnt).x) * 1.0001f;
                    }
                }
                for (int nc = 0; nc < g.ncols; ++nc) {
                    const float x = (float)nc;
                    const float sv = cm[0] + x * (cm[1] + x * (cm[2] + x * (cm[3] + x * cm[4])));
                    int eb = r >= 0 && sv > 0.f ? exp_bound(log2f(sv) - cr * g.Mcc * x * x) : -100;
                    eb = __reduce_max_sync(0xffffffffu, eb);  // warp maximum, one shared atomic per warp
                    if (lane == 0) atomicMax(&eB[gb * npo + nc * g.nd + d], eb);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
    if (lane == 0 && cmin < INFINITY) atomicMin(&clmin_bits, __float_as_int(cmin));
    __syncthreads();
    for (int i = tid; i < kTcEbMax; i += blockDim.x) g.ebw[(size_t)w * kTcEbMax + i] = eB[i];
    if (tid == 0) g.clw[w] = __int_as_float(clmin_bits);
}

__global__ void __launch_bounds__(kTcThreadsAll, 1) k_tc_rho(TcArgs g, int ntslots) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* abuf = tsm;                                                    // [nbuf][S][8192]
    unsigned char* bbuf = abuf + (size_t)kTcNbuf * kTcS * kTcAsliceBytes;          // [nbuf][S][npad*64]
    const int bslice = g.npad * 64;
    unsigned char* tring = bbuf + (size_t)kTcNbuf * kTcS * bslice;                 // [ntslots][slot]
    const size_t tslot = tab_slot_bytes(g.tabw, g.G, g.nd);
    TcSmem& sm = *reinterpret_cast<TcSmem*>(tring + (size_t)ntslots * tslot);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kg = blockIdx.x, mt = blockIdx.y;
    const int w0 = kg * g.win_per_group, w1 = min(g.nwin, w0 + g.win_per_group);
    volatile int* abort_flag = &sm.abort_flag;
    const bool mma_warp = warp == kTcMmaWarp, load_warp = warp == kTcLoadWarp;
    const bool epi = warp < kTcEpiWarps;  // drains tensor memory: four lane quadrants x three column thirds

    if (tid == 0) {
        for (int b = 0; b < kTcNbuf; ++b) {
            mbar_init(&sm.full[b], kTcProdWarps);
            mbar_init(&sm.empty[b], 1);
        }
        for (int b = 0; b < ntslots; ++b) {
            mbar_init(&sm.tfull[b], 1);
            mbar_init(&sm.tempty[b], kTcProdWarps);
        }
        mbar_init(&sm.accf, 1);
        mbar_init(&sm.acce, kTcEpiWarps);
        mbar_init(&sm.done, 1);
        mbar_init(&sm.psync, kTcWarps);
        sm.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < kTcM) {
        const int m = mt * kTcM + tid;
        const int2 rw = m < g.nrows ? __ldg(g.rows + m) : make_int2(INT_MIN, 0);
        TcRow ri;
        ri.na = rw.x;
        ri.nb = rw.y;
        ri.Q = rw.x != INT_MIN ? g.Maa * (float)rw.x * (float)rw.x + g.Mbb * (float)rw.y * (float)rw.y : 0.f;
        sm.rowi[tid] = ri;
    }
    // zero both stage buffers once: padding columns of B are never written
    for (int i = tid; i < kTcNbuf * kTcS * bslice / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(bbuf)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&sm.tmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    // epilogue roles (warps 0-11): TMEM lanes 32 (w & 3) .. + 31, 8-column chunks c8 = w / 4 (mod 3)
    const int equad = warp & 3, ewarp3 = warp >> 2, erow = 32 * equad + lane;
    const uint32_t tlane = (uint32_t)(32 * equad) << 16;
    const int npo = g.nd * g.ncols;  // complex outputs per block
    const int nchunk = g.colw / 8;   // 8-column chunks of a block (4 complex outputs each)
    const uint32_t acc_hi = (uint32_t)(4 * g.npad), acc_lo = acc_hi + (uint32_t)g.colw;
    if (epi) {
        for (int c8 = ewarp3; c8 < nchunk; c8 += 3) {
            const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            tc_st8(tmem + tlane + acc_hi + (uint32_t)(8 * c8), z);
            tc_st8(tmem + tlane + acc_lo + (uint32_t)(8 * c8), z);
        }
        tc_wait_st();
    }
    // The operand tasks of a stage, the same for every stage: B tasks (four
    // records of one (block, output pair)) then A tasks (four records of one
    // row), dealt to the operand threads in snake order (0..P-1, P-1..0, ...),
    // so that the heavier B tasks and the A tasks spread evenly.
    int tk[kTcTasksMax], ntask = 0;
    {
        const int nbt = (kTcStageK / 4) * g.G * npo, ntot = nbt + kTcM * 4;
#pragma unroll
        for (int e = 0; e < kTcTasksMax; ++e) {
            const int k = e * kTcProdThreads + ((e & 1) ? kTcProdThreads - 1 - tid : tid);
            tk[e] = 0;
            if (!mma_warp && !load_warp && k < ntot) {
                if (k < nbt) {
                    const int p = k % npo, t2 = k / npo, gb = t2 % g.G, kgq = t2 / g.G;
                    tk[e] = kgq | (gb << 2) | (p << 6);
                } else {
                    tk[e] = (k - nbt) | kTcTaskA;
                }
                ntask = e + 1;
            }
        }
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(g.npad >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    long long gs = 0;  // stages so far (every role counts the same)
    uint32_t ph = 0;
    bool ok = true;
    for (int w = w0; w < w1 && ok; ++w) {
        // ---- window records, blocks and scales ----
        for (int i = tid; i < kTcWin; i += kTcThreadsAll) sm.rec[i] = __ldg(g.wrec + (size_t)w * kTcWin + i);
        for (int i = tid; i < kTcEbMax; i += kTcThreadsAll) sm.eB[i] = __ldg(g.ebw + (size_t)w * kTcEbMax + i);
        if (tid == 0) {
            const int4 wi = __ldg(g.winfo + w);
            sm.winL = wi.x;
            sm.wnpair = wi.y;
            sm.wpos = wi.w;
            for (int b = 0; b < wi.y; ++b) {
                const int pr = __ldg(g.wpairs + wi.z + b), i = pr & 7, j = pr >> 3;
                sm.pairs[b] = pr;
                for (int kk = 0; kk < 5; ++kk) sm.tidx[b][kk] = kk <= wi.x - i - j ? term_of(g, i, j, kk) : -1;
            }
            sm.clmin_bits = __float_as_int(__ldg(g.clw + w));
        }
        if (!(ok = prod_sync(&sm.psync, ph, abort_flag, lane, g.spin))) break;
        const int L = sm.winL, npair = sm.wnpair;
        const float clmin = __int_as_float(sm.clmin_bits);
        // ---- stages ----
        if (load_warp) {
            // rows of D' a stage needs: (block, density, k <= L - i - j)
            int nrow = 0;
            for (int gb = 0; gb < npair; ++gb) nrow += g.nd * (L - (sm.pairs[gb] & 7) - (sm.pairs[gb] >> 3) + 1);
            const float2* dpL = g.Dp + g.dp_base[L];
            for (int q = 0; q < kTcStagesPerWin; ++q, ++gs) {
                const int ts = (int)(gs % ntslots);
                const long long use = gs / ntslots;
                if (use > 0) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&sm.tempty[ts], (uint32_t)((use - 1) & 1), abort_flag, g.spin));
                    if (!ok) break;
                }
                unsigned char* slotp = tring + (size_t)ts * tslot;
                float2* dps = reinterpret_cast<float2*>(slotp + (size_t)kTcStageK * g.tabw * 16);
                // A stage holds records from its first entry on, or none (the padding at a
                // window's end): its D' rows are copied only when it holds some, and then
                // stay inside the class's 16-padded stride.
                const int srow = sm.rec[q * kTcStageK] >= 0 ? nrow : 0;
                if (lane == 0) {
                    uint32_t nv = 0;
                    for (int u = 0; u < kTcStageK; ++u) nv += sm.rec[q * kTcStageK + u] >= 0 ? 1u : 0u;
                    mbar_arrive_tx(&sm.tfull[ts], nv * (uint32_t)g.tabw * 16u + (uint32_t)srow * kTcStageK * 8u);
                }
                __syncwarp();
                // lanes 0-15: the records' factor tables; the rest: 128-byte rows of D'
                for (int idx = lane; idx < kTcStageK + srow; idx += 32) {
                    if (idx < kTcStageK) {
                        const int r = sm.rec[q * kTcStageK + idx];
                        if (r >= 0)
                            bulk_copy(slotp + (size_t)idx * g.tabw * 16, g.tab + (size_t)r * g.tabw,
                                      (uint32_t)g.tabw * 16u, &sm.tfull[ts]);
                    } else {
                        int row = idx - kTcStageK, gb = 0;
                        for (;;) {  // row -> (block, density, k)
                            const int nkb = L - (sm.pairs[gb] & 7) - (sm.pairs[gb] >> 3) + 1;
                            if (row < g.nd * nkb) break;
                            row -= g.nd * nkb;
                            ++gb;
                        }
                        const int pr = sm.pairs[gb], nkb = L - (pr & 7) - (pr >> 3) + 1;
                        const int d = row / nkb, kk = row - d * nkb;
                        const long long src = (long long)(g.d0 + d) * g.dp_total +
                                              (long long)sm.tidx[gb][kk] * g.dp_stride[L] + sm.wpos + q * kTcStageK;
                        bulk_copy(dps + ((gb * g.nd + d) * 5 + kk) * kTcStageK, dpL + src, kTcStageK * 8u,
                                  &sm.tfull[ts]);
                    }
                }
                __syncwarp();
            }
        } else if (!mma_warp) {
            for (int q = 0; q < kTcStagesPerWin; ++q, ++gs) {
                const int slot = (int)(gs & 1), ts = (int)(gs % ntslots);
                ok = __all_sync(0xffffffffu, mbar_wait(&sm.tfull[ts], (uint32_t)((gs / ntslots) & 1), abort_flag, g.spin));
                if (!ok) break;
                if (gs >= kTcNbuf) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&sm.empty[slot], (uint32_t)(((gs >> 1) - 1) & 1), abort_flag, g.spin));
                    if (!ok) break;
                }
                const unsigned char* slotp = tring + (size_t)ts * tslot;
                const float4* tabs = reinterpret_cast<const float4*>(slotp);
                const float2* dps = reinterpret_cast<const float2*>(slotp + (size_t)kTcStageK * g.tabw * 16);
                unsigned char* as = abuf + (size_t)slot * kTcS * kTcAsliceBytes;
                unsigned char* bs = bbuf + (size_t)slot * kTcS * bslice;
#pragma unroll
                for (int e = 0; e < kTcTasksMax; ++e) {
                    if (e < ntask) {
                        const int k = tk[e];
                        if (k & kTcTaskA) {
                            const int row = k & (kTcM - 1), gg = (k >> 7) & 3;
                            form_a(g, sm, tabs, q, row, gg, pow2f(6 - exp_bound(-clmin * sm.rowi[row].Q)), as);
                        } else {
                            form_b(g, sm, tabs, dps, q, k & 3, (k >> 2) & 15, k >> 6, bs, bslice);
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&sm.full[slot]);
                    mbar_arrive(&sm.tempty[ts]);
                }
            }
        } else {
            if (lane == 0) {
                const uint32_t a0 = saddr(abuf), b0 = saddr(bbuf);
                bool first[kTcAcc] = {true, true, true, true};
                bool mok = true;
                for (int q = 0; q < kTcStagesPerWin; ++q, ++gs) {
                    const int slot = (int)(gs & 1);
                    if (!(mok = mbar_wait(&sm.full[slot], (uint32_t)((gs >> 1) & 1), abort_flag, g.spin))) break;
                    tc_fence_after();
                    const uint32_t as = a0 + slot * kTcS * kTcAsliceBytes, bs = b0 + slot * kTcS * bslice;
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int s = 0; s < kTcS; ++s)
#pragma unroll
                            for (int t = 0; s + t < kTcS; ++t) {
                                const int lv = min(s + t, kTcAcc - 1);
                                tc_mma(tmem + (uint32_t)(lv * g.npad), sdesc(as + s * kTcAsliceBytes + h * 256),
                                       sdesc(bs + t * bslice + h * 256), idesc, first[lv] ? 0u : 1u);
                                first[lv] = false;
                            }
                    tc_commit(&sm.empty[slot]);
                }
                if (mok) tc_commit(&sm.accf);
                ok = mok;
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            gs = __shfl_sync(0xffffffffu, gs, 0);
        }
        if (!ok) break;
        // ---- drain: each block's level sums, scaled and times P_ij, into the double-float sums (warps 0-11) ----
        if (epi) {
            ok = __all_sync(0xffffffffu, mbar_wait(&sm.accf, (uint32_t)((w - w0) & 1), abort_flag, g.spin));
            if (!ok) break;
            tc_fence_after();
            const TcRow ri = sm.rowi[erow];
            const int eAe = exp_bound(-clmin * ri.Q);
            for (int c8 = ewarp3; c8 < nchunk; c8 += 3) {
                float H[8], Lo[8];
                tc_ld8(tmem + tlane + acc_hi + (uint32_t)(8 * c8), H);
                tc_ld8(tmem + tlane + acc_lo + (uint32_t)(8 * c8), Lo);
                for (int gb = 0; gb < npair; ++gb) {
                    const int i = sm.pairs[gb] & 7, j = sm.pairs[gb] >> 3;
                    float pij = 1.f;  // n_a^i n_b^j, exact
                    for (int k = 0; k < i; ++k) pij *= (float)ri.na;
                    for (int k = 0; k < j; ++k) pij *= (float)ri.nb;
                    float T[kTcAcc][8];
#pragma unroll
                    for (int lv = 0; lv < kTcAcc; ++lv)
                        tc_ld8(tmem + tlane + (uint32_t)(lv * g.npad + gb * g.colw + 8 * c8), T[lv]);
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const int p = 4 * c8 + u / 2;
                        if (p < npo) {
                            cdf v;
                            v.re = df_add(df_add(two_sum(T[0][u], T[1][u]), df{T[2][u], 0.f}), df{T[3][u], 0.f});
                            v.im = df_add(df_add(two_sum(T[0][u + 1], T[1][u + 1]), df{T[2][u + 1], 0.f}),
                                          df{T[3][u + 1], 0.f});
                            const float sc = pow2f(eAe + sm.eB[gb * npo + p] - 12);  // exact power of two
                            v = cdf{df_mulf(df{v.re.hi * sc, v.re.lo * sc}, pij),
                                    df_mulf(df{v.im.hi * sc, v.im.lo * sc}, pij)};
                            v = rot_mi(v, i + j);
                            const df re = df_add(df{H[u], Lo[u]}, v.re), im = df_add(df{H[u + 1], Lo[u + 1]}, v.im);
                            H[u] = re.hi;
                            Lo[u] = re.lo;
                            H[u + 1] = im.hi;
                            Lo[u + 1] = im.lo;
                        }
                    }
                }
                tc_st8(tmem + tlane + acc_hi + (uint32_t)(8 * c8), H);
                tc_st8(tmem + tlane + acc_lo + (uint32_t)(8 * c8), Lo);
            }
            tc_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acce);
        }
        // the MMAs of the next window wait for every draining warp
        if (mma_warp && w + 1 < w1) {
            ok = __all_sync(0xffffffffu, mbar_wait(&sm.acce, (uint32_t)((w - w0) & 1), abort_flag, g.spin));
            tc_fence_after();
        }
        if (!(ok = prod_sync(&sm.psync, ph, abort_flag, lane, g.spin) && ok)) break;  // window tables reused next window
    }
    // ---- partial rows ----
    if (ok && !*abort_flag && epi) {
        tc_fence_after();
        const int mo = mt * kTcM + erow;
        for (int c8 = ewarp3; c8 < nchunk; c8 += 3) {
            float H[8], Lo[8];
            tc_ld8(tmem + tlane + acc_hi + (uint32_t)(8 * c8), H);
            tc_ld8(tmem + tlane + acc_lo + (uint32_t)(8 * c8), Lo);
            if (mo < g.nrows) {
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const int p = 4 * c8 + u / 2;
                    if (p < npo) {
                        const int nc = p / g.nd, d = p - nc * g.nd;
                        int idx = __ldg(g.map + (size_t)mo * g.ncols + nc);
                        if (idx != INT_MIN) {
                            const bool cj = idx < 0;
                            if (cj) idx = ~idx;
                            const double re = (double)H[u] + (double)Lo[u];
                            const double im = (double)H[u + 1] + (double)Lo[u + 1];
                            g.out[((long long)(g.d0 + d) * g.ngroups + kg) * g.ng_half + idx] =
                                make_double2(re, cj ? -im : im);
                        }
                    }
                }
            }
        }
    }
    if (load_warp && lane == 0) {
        // bulk copies still in flight (after a failed wait) land before the CTA exits
        for (int b = 0; b < ntslots && b < gs; ++b) {
            const long long last = gs - 1 - ((gs - 1 - b) % ntslots);  // last stage that used slot b
            const long long t0 = clock64();
            while (!mbar_test(&sm.tfull[b], (uint32_t)((last / ntslots) & 1)) && clock64() - t0 < kTcSpinCycles) {
            }
        }
    }
    if (mma_warp) {
        // everything issued completes before tensor memory is freed
        if (lane == 0) {
            tc_commit(&sm.done);
            const long long t0 = clock64();
            while (!mbar_test(&sm.done, 0u) && clock64() - t0 < kTcSpinCycles) {
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(g.err, 1);
    if (mma_warp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

// per-record factor tables X(0..na), Y(0..nb), Z(0..nc) in FP64, kept as double-float
__global__ void k_tc_tables(const PairWalk* __restrict__ walk, long long npairs, int ax, int bx, int cx, int nna,
                            int nnb, int nnc, double Maa, double Mbb, double Mcc, float4* __restrict__ tab,
                            float* __restrict__ cl) {
    const int tabw = nna + nnb + nnc;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npairs * tabw) return;
    const long long r = t / tabw;
    const int e = (int)(t - r * tabw);
    const PairWalk w = walk[r];
    const double f[3] = {w.f1, w.f2, w.f3};
    double M, fr;
    int n;
    if (e < nna) {
        n = e;
        M = Maa;
        fr = f[ax];
    } else if (e < nna + nnb) {
        n = e - nna;
        M = Mbb;
        fr = f[bx];
    } else {
        n = e - nna - nnb;
        M = Mcc;
        fr = f[cx];
    }
    const double gval = exp(-w.c * M * (double)n * (double)n);
    double th = fr * (double)n;
    th -= rint(th);
    double s, c;
    sincospi(2.0 * th, &s, &c);
    const df re = df_from_double(gval * c), im = df_from_double(-gval * s);
    tab[t] = make_float4(re.hi, re.lo, im.hi, im.lo);
    if (e == 0) cl[r] = (float)(w.c * 1.4426950408889634);
}

// shared memory of one CTA with `nts` table slots (at least 120 KB, so that a
// second CTA never shares an SM: each one takes all 512 tensor-memory
// columns, and a second would wait in tcgen05.alloc)
size_t tc_smem_bytes(int npad, int tabw, int G, int nd, int nts) {
    const size_t need = (size_t)kTcNbuf * kTcS * kTcAsliceBytes + (size_t)kTcNbuf * kTcS * npad * 64 +
                        (size_t)nts * tab_slot_bytes(tabw, G, nd) + sizeof(TcSmem) + 64;
    return std::max<size_t>(need, 120 * 1024);
}

template <class T>
int tc_upload(ftcj_plan* P, T** ptr, const std::vector<T>& v) {
    const size_t n = std::max<size_t>(v.size(), 1);
    cudaError_t e = cudaMalloc((void**)ptr, sizeof(T) * n);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(FTCJ_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    P->device_bytes += sizeof(T) * n;
    if (!v.empty()) FTCJ_CUDA(cudaMemcpy(*ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return FTCJ_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// column layout for nd densities and ncols values of n_c: real columns per
// block (a multiple of 8) and the largest block count G whose level
// accumulators (4 x G x colw, rounded to 16) and double-float sums (2 colw)
// fit the 512 tensor-memory columns; G = 0 when not even one block fits
void tc_columns(int nd, int ncols, int* colw, int* G, int* npad) {
    *colw = round_up(2 * nd * ncols, 8);
    *G = 0;
    *npad = 0;
    for (int gg = kTcGmax; gg >= 1; --gg) {
        const int np = round_up(gg * *colw, 16);
        if (np <= kTcNmma && 4 * np + 2 * *colw <= kTcTmemCols && gg * nd * ncols <= kTcEbMax) {
            *G = gg;
            *npad = np;
            return;
        }
    }
}


// ---- the back-contraction (Alg. S1) in the same separable form -------------
//
// The walks' back-contraction sums, over the stored half sphere,
//   J'_{r,ijk} = Re sum_n (-i)^{i+j+k} n_a^i n_b^j n_c^k X_r(n_a) Y_r(n_b) Z_r(n_c) W(n).
// On the grid of rows m = (n_a, n_b) and columns n_c >= 0 (a stored point -n
// enters as conj W, since the conjugate of the summand at -n is the summand
// at n with conj W) this is
//   J'_{r,ijk} = Re (-i)^k sum_{n_c} n_c^k Z_r(n_c) U_ij[r, n_c],
//   U_ij[r, n_c] = sum_m A^T[r, m] V_ij[m, n_c],
//   A^T[r, m] = X_r(n_a) Y_r(n_b),  V_ij = (-i)^{i+j} n_a^i n_b^j W(m, n_c),
// a complex matrix product with M = 128 records of one class, K = the rows
// (real and imaginary parts), N = (i, j) blocks x densities x n_c.  V_ij does
// not depend on the record: it is sliced once per build (k_tc_vbound,
// k_tc_vslice) into stage tiles in global memory that bulk copies bring into
// shared memory, and only A^T is formed in the kernel, from the 128 records'
// factor tables staged once per work item.  Every entry of A^T has modulus
// <= 1 (scale 2^1 for all of them); each column of V_ij gets its own scale
// over all rows, so that entries far out in the sphere (where W has decayed)
// sit many bits below their column's scale.  Seven slices (products with
// s + t <= 6, 28 per k-step) keep the truncation below 2^-45 of the scales.
// The rows are cut into parts of at most 512 (1024 real K terms), each a
// work item of its own: within a part, levels 0-3 are exact (the level-3 sums
// stay below 1024 x 14720 < 2^24 in units of 2^-21: |A| <= 1 bounds the
// leading slice of A by 32) and only levels 4-6 share the rounded fifth
// accumulator.  The tensor core's FP32 accumulation does not round to
// nearest, so the rounded accumulator's error grows with the number of MMAs
// that add into it and with its size; keeping level 3 out of it keeps that
// error ~2^-7 of the four-accumulator scheme's.  The level sums go straight
// to the epilogue, which forms the part's J' for k <= L - i - j in
// double-float and writes it as one of the partial FP64 sums the J -> AO map
// adds.

constexpr int kTcJStageM = 8;        // rows per stage: one MMA k-step of 16 real K
constexpr int kTcJS = 7;             // slices per operand
constexpr int kTcJProducts = kTcJS * (kTcJS + 1) / 2;  // slice products formed: s + t <= 6
constexpr int kTcJPartStages = 64;   // stages per row part at most: 512 rows, one exact accumulation
constexpr int kTcJPartRows = kTcJPartStages * kTcJStageM;
constexpr int kTcJAcc = 5;           // accumulators: levels 0-3 exact, levels 4-6 rounded
constexpr int kTcJNmax = 96;         // MMA N at most: five level accumulators in the 512 columns
constexpr int kTcJAsliceBytes = kTcM * 2 * kTcJStageM * 2;  // 128 records x 16 real K x bf16
constexpr int kTcJTasks = kTcM * kTcJStageM;                  // (record, row) entries of a stage
constexpr int kTcPairsAll = 15;      // (i, j) with i + j <= 4

__host__ __device__ constexpr int pair_index(int i, int j) { return i * 5 - i * (i - 1) / 2 + j; }

__device__ __forceinline__ void pair_of_index(int pr, int& i, int& j) {
    i = 0;
    while (pr > 4 - i) {
        pr -= 5 - i;
        ++i;
    }
    j = pr;
}

// Seven slices of x = hi + lo (|x| < 2^e, sc = 2^(6-e)): o[s] = m_s 2^(-7s),
// integers |m_s| <= 64, x = 2^(e-6) sum_s o[s] up to 2^(e-51).  As in the
// six-slice split, but the low part joins at slice 3 through an error-free
// sum, so that none of its bits above 2^-45 (in units of o[0]) is lost.
__device__ __forceinline__ void slice7(float hi, float lo, float sc, float (&o)[kTcJS]) {
    float h = hi * sc;
    const float l = lo * sc;
    o[0] = (h + 0x1.8p23f) - 0x1.8p23f;
    h -= o[0];
    o[1] = (h + 0x1.8p16f) - 0x1.8p16f;
    h -= o[1];
    o[2] = (h + 0x1.8p9f) - 0x1.8p9f;
    h -= o[2];
    const df j = two_sum(h, l);  // h + l = j.hi + j.lo exactly
    o[3] = (j.hi + 0x1.8p2f) - 0x1.8p2f;
    h = (j.hi - o[3]) + j.lo;
    o[4] = (h + 0x1.8p-5f) - 0x1.8p-5f;
    h -= o[4];
    o[5] = (h + 0x1.8p-12f) - 0x1.8p-12f;
    h -= o[5];
    o[6] = (h + 0x1.8p-19f) - 0x1.8p-19f;
}

// element offset of (row, k) in a stage tile [rows][16 real K] of core matrices
__device__ __forceinline__ int tile_off16(int row, int k) {
    return (((row >> 3) * 2 + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// K-major, no swizzle: K-adjacent core matrices 128 B apart, 8-row groups 256 B apart
__device__ __forceinline__ uint64_t sdesc16(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           (1ull << 46);
}

struct TcJArgs {
    const int2* rows;       // (n_a, n_b) per row (the structure-factor pass's rows)
    const int* map;         // [rows][ncols]: half-sphere index, ~index where the stored point is -n, INT_MIN none
    const double2* W;       // potential W(G) on the half sphere, [dens][ng_half]
    const int4* items;      // work items: class L | row part << 8, blocks, first block index into ipairs, first record
    const int* ipairs;      // (i | j << 3) of each block
    const float4* tab;      // per record [tabw]: X(0..), Y(0..), Z(0..) as complex double-float
    __nv_bfloat16* vs;      // sliced V_ij: [15 (i, j)][stage][slice][colw x 16 real K] stage tiles
    int* ev;                // column scales of V_ij: [15][nd][ncols]
    double* Jp;             // partial back-contraction sums [dens][part][term] in the split form's class layout
    long long ng_half;
    long long jp_total;     // doubles per density of Jp
    long long cls_start[kNclass + 1];
    long long term_base[kNclass];
    int* err;               // device error word (bit 0: a bounded wait gave up)
    int ax, bx, cx;
    int tabw, offY, offZ;
    int ncols, nd, d0;
    int gw;                 // real columns per density: 2 ncols rounded up to 8
    int colw;               // real columns per block: nd gw
    int npad;               // MMA N of a full item: blocks x colw rounded up to 16 (<= 128)
    int nrows, nstage, nitems;
    int nparts, spp;        // row parts, stages per part
    long long spin;         // clock cycles a wait between roles may take before it gives up
};

// column scales: the exponent bound of max over the rows of |n_a^i n_b^j W(m, n_c)|
__global__ void __launch_bounds__(256) k_tc_vbound(TcJArgs g) {
    const int col = blockIdx.x;  // ((i, j) nd + d) ncols + n_c
    const int nc = col % g.ncols, d = (col / g.ncols) % g.nd, pr = col / (g.ncols * g.nd);
    int i, j;
    pair_of_index(pr, i, j);
    float mx = 0.f;
    for (int m = threadIdx.x; m < g.nrows; m += blockDim.x) {
        const int2 rw = __ldg(g.rows + m);
        const int idx = __ldg(g.map + (size_t)m * g.ncols + nc);
        if (idx == INT_MIN) continue;
        const double2 w = __ldg(g.W + (long long)(g.d0 + d) * g.ng_half + (idx < 0 ? ~idx : idx));
        float p = 1.f;
        for (int k = 0; k < i; ++k) p *= (float)abs(rw.x);
        for (int k = 0; k < j; ++k) p *= (float)abs(rw.y);
        mx = fmaxf(mx, p * (float)fmax(fabs(w.x), fabs(w.y)));
    }
    __shared__ float red[256];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    // |Re V|, |Im V| <= mx up to the FP32 rounding of the bound
    if (threadIdx.x == 0) g.ev[col] = red[0] > 0.f ? exp_bound(log2f(red[0] * 1.0001f)) : -100;
}

// V_ij sliced into stage tiles: tile (i, j), stage q, slice s holds column
// d gw + 2 n_c + part and K = (row, re/im) in the real form rows
// (m, re) -> [Re V | Im V], (m, im) -> [-Im V | Re V]; columns past 2 ncols
// stay zero from the allocation.
__global__ void __launch_bounds__(256) k_tc_vslice(TcJArgs g) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_pair = (long long)g.nstage * kTcJStageM * g.nd * g.ncols;
    if (t >= kTcPairsAll * per_pair) return;
    const int pr = (int)(t / per_pair);
    long long rem = t - pr * per_pair;
    const int nc = (int)(rem % g.ncols);
    rem /= g.ncols;
    const int d = (int)(rem % g.nd);
    rem /= g.nd;
    const int ml = (int)(rem % kTcJStageM), q = (int)(rem / kTcJStageM);
    const int m = q * kTcJStageM + ml;
    int i, j;
    pair_of_index(pr, i, j);
    cdf v{{0.f, 0.f}, {0.f, 0.f}};
    if (m < g.nrows) {
        const int2 rw = __ldg(g.rows + m);
        const int idx = __ldg(g.map + (size_t)m * g.ncols + nc);
        if (idx != INT_MIN) {
            const double2 w = __ldg(g.W + (long long)(g.d0 + d) * g.ng_half + (idx < 0 ? ~idx : idx));
            float p = 1.f;  // n_a^i n_b^j, exact
            for (int k = 0; k < i; ++k) p *= (float)rw.x;
            for (int k = 0; k < j; ++k) p *= (float)rw.y;
            const cdf wv{split_double(w.x), split_double(idx < 0 ? -w.y : w.y)};
            v = rot_mi(cdf{df_mulf(wv.re, p), df_mulf(wv.im, p)}, i + j);
        }
    }
    const float sc = pow2f(6 - g.ev[(pr * g.nd + d) * g.ncols + nc]);
    float sr[kTcJS], si[kTcJS];
    slice7(v.re.hi, v.re.lo, sc, sr);
    slice7(v.im.hi, v.im.lo, sc, si);
    const int c0 = d * g.gw + 2 * nc;
    __nv_bfloat16* base = g.vs + ((size_t)pr * g.nstage + q) * kTcJS * (size_t)g.colw * 16;
    const int o0 = tile_off16(c0, 2 * ml), o1 = tile_off16(c0 + 1, 2 * ml);
#pragma unroll
    for (int s = 0; s < kTcJS; ++s) {
        __nv_bfloat16* bs = base + (size_t)s * g.colw * 16;
        *reinterpret_cast<uint32_t*>(bs + o0) = pack_bf2(sr[s], -si[s]);
        *reinterpret_cast<uint32_t*>(bs + o1) = pack_bf2(si[s], sr[s]);
    }
}

struct TcJSmem {
    int rec[kTcM];
    int pairs[kTcGmax];
    int tidx[kTcGmax][5];  // index of J'_{ijk} for block (i, j) and k = 0..4 (-1 past the class's degree)
    int2 rowi[kTcJPartRows];  // the part's rows
    int iL, inb, ipart;
    uint64_t full[kTcNbuf], empty[kTcNbuf], bfull[kTcNbuf], tfull, accf, acce, done, psync;
    uint32_t tmem;
    int abort_flag;
};

// index of J'_{p1 p2 p3} (powers of n_1, n_2, n_3) for powers (i, j, k) of (n_a, n_b, n_c)
__device__ __forceinline__ int term_of_j(const TcJArgs& g, int i, int j, int k) {
    const int p1 = g.ax == 0 ? i : (g.bx == 0 ? j : k);
    const int p2 = g.ax == 1 ? i : (g.bx == 1 ? j : k);
    const int lam = i + j + k;
    return lam_offset(lam) + mono_index(lam, p1, p2);
}

// A^T entry (record r, stage row ml): X_r(n_a) Y_r(n_b) sliced, one 4-byte
// store (re, im) per slice; a warp's 32 entries (8 records x 4 rows) fill
// eight core-matrix rows, 128 contiguous bytes
__device__ __forceinline__ void form_aj(const TcJArgs& g, const TcJSmem& sm, const float4* tabs, int q, int k,
                                        unsigned char* as) {
    const int ml = (k & 3) | (((k >> 5) & 1) << 2);
    const int r = ((k >> 2) & 7) | ((k >> 6) << 3);
    const int m = q * kTcJStageM + ml;  // q: stage of the part
    cdf a{{0.f, 0.f}, {0.f, 0.f}};
    if (sm.rowi[m].x != INT_MIN && sm.rec[r] >= 0) {
        const int2 rw = sm.rowi[m];
        const float4 xv = tabs[r * g.tabw + abs(rw.x)], yv = tabs[r * g.tabw + g.offY + abs(rw.y)];
        const float sa = rw.x < 0 ? -1.f : 1.f, sb = rw.y < 0 ? -1.f : 1.f;  // X(-n) = conj X(n)
        a = cdf_mul(cdf{{xv.x, xv.y}, {sa * xv.z, sa * xv.w}}, cdf{{yv.x, yv.y}, {sb * yv.z, sb * yv.w}});
    }
    float sr[kTcJS], si[kTcJS];
    slice7(a.re.hi, a.re.lo, 0x1p5f, sr);  // |A| <= 1 < 2^1
    slice7(a.im.hi, a.im.lo, 0x1p5f, si);
    const int off = tile_off16(r, 2 * ml);
#pragma unroll
    for (int s = 0; s < kTcJS; ++s)
        *reinterpret_cast<uint32_t*>(as + (size_t)s * kTcJAsliceBytes + (size_t)off * 2) = pack_bf2(sr[s], si[s]);
}

// Persistent over the work items (class, group of (i, j) blocks, 128
// records, row part), with the structure-factor kernel's roles: warps 0-13
// form the A^T slices of each 8-row stage, lane 0 of warp 14 issues the MMAs, warp 15
// brings the item's factor tables (once per item) and the V_ij stage tiles
// in with bulk copies; warps 0-11 then form J' from tensor memory (lane
// quadrant w & 3, (block, density) groups w / 4 mod 3).  Waits are bounded
// as in the structure-factor kernel.
__global__ void __launch_bounds__(kTcThreadsAll, 1) k_tc_j(TcJArgs g) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int bslice = g.npad * 32;
    unsigned char* abuf = tsm;                                                     // [nbuf][S][4096]
    unsigned char* bbuf = abuf + (size_t)kTcNbuf * kTcJS * kTcJAsliceBytes;          // [nbuf][S][npad x 32]
    float4* tabs = reinterpret_cast<float4*>(bbuf + (size_t)kTcNbuf * kTcJS * bslice);  // [128][tabw]
    TcJSmem& sm = *reinterpret_cast<TcJSmem*>(tabs + (size_t)kTcM * g.tabw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_flag = &sm.abort_flag;
    const bool mma_warp = warp == kTcMmaWarp, load_warp = warp == kTcLoadWarp, epi = warp < kTcEpiWarps;
    if (tid == 0) {
        for (int b = 0; b < kTcNbuf; ++b) {
            mbar_init(&sm.full[b], kTcProdWarps);
            mbar_init(&sm.empty[b], 1);
            mbar_init(&sm.bfull[b], 1);
        }
        mbar_init(&sm.tfull, 1);
        mbar_init(&sm.accf, 1);
        mbar_init(&sm.acce, kTcEpiWarps);
        mbar_init(&sm.done, 1);
        mbar_init(&sm.psync, kTcWarps);
        sm.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // columns of B past an item's blocks are never read into an output: clear them once
    for (int i = tid; i < kTcNbuf * kTcJS * bslice / 16; i += kTcThreadsAll)
        reinterpret_cast<uint4*>(bbuf)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&sm.tmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const int equad = warp & 3, ethird = warp >> 2, erow = 32 * equad + lane;
    const uint32_t tlane = (uint32_t)(32 * equad) << 16;
    long long gs = 0;  // stages so far (every role counts the same)
    int nit = 0;       // items finished
    int ntab = 0;      // table loads issued (load warp)
    uint32_t ph = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
        // ---- the item: class, blocks, records ----
        const int4 in = __ldg(g.items + it);
        const int iL = in.x & 255, part = in.x >> 8;
        if (tid == 0) {
            sm.iL = iL;
            sm.inb = in.y;
            sm.ipart = part;
            for (int b = 0; b < in.y; ++b) {
                const int pr = __ldg(g.ipairs + in.z + b), i = pr & 7, j = pr >> 3;
                sm.pairs[b] = pr;
                for (int kk = 0; kk < 5; ++kk) sm.tidx[b][kk] = kk <= iL - i - j ? term_of_j(g, i, j, kk) : -1;
            }
        }
        if (tid < kTcM) sm.rec[tid] = (long long)in.w + tid < g.cls_start[iL + 1] ? in.w + tid : -1;
        for (int m = tid; m < kTcJPartRows; m += kTcThreadsAll) {
            const int mg = part * g.spp * kTcJStageM + m;
            sm.rowi[m] = m < g.spp * kTcJStageM && mg < g.nrows ? __ldg(g.rows + mg) : make_int2(INT_MIN, 0);
        }
        if (!(ok = prod_sync(&sm.psync, ph, abort_flag, lane, g.spin))) break;
        const int L = sm.iL, nb = sm.inb, q0 = sm.ipart * g.spp, nst = min(g.spp, g.nstage - q0);
        if (load_warp) {
            // the records' factor tables, then every stage's V_ij tiles
            if (lane == 0) {
                uint32_t nv = 0;
                for (int r = 0; r < kTcM; ++r) nv += sm.rec[r] >= 0 ? 1u : 0u;
                mbar_arrive_tx(&sm.tfull, nv * (uint32_t)g.tabw * 16u);
            }
            __syncwarp();
            for (int r = lane; r < kTcM; r += 32)
                if (sm.rec[r] >= 0)
                    bulk_copy(tabs + (size_t)r * g.tabw, g.tab + (size_t)sm.rec[r] * g.tabw, (uint32_t)g.tabw * 16u,
                              &sm.tfull);
            ++ntab;
            const uint32_t blk = (uint32_t)g.colw * 32u;  // bytes of one block's slice of a stage
            for (int q = 0; q < nst; ++q, ++gs) {
                const int slot = (int)(gs & 1);
                if (gs >= kTcNbuf) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&sm.empty[slot], (uint32_t)(((gs >> 1) - 1) & 1), abort_flag, g.spin));
                    if (!ok) break;
                }
                unsigned char* bs = bbuf + (size_t)slot * kTcJS * bslice;
                if (lane == 0) mbar_arrive_tx(&sm.bfull[slot], (uint32_t)(nb * kTcJS) * blk);
                __syncwarp();
                for (int c = lane; c < nb * kTcJS; c += 32) {
                    const int gb = c / kTcJS, s = c - gb * kTcJS;
                    const int pr = sm.pairs[gb];
                    const size_t src =
                        (((size_t)pair_index(pr & 7, pr >> 3) * g.nstage + q0 + q) * kTcJS + s) * g.colw * 16;
                    bulk_copy(bs + (size_t)s * bslice + (size_t)gb * blk, g.vs + src, blk, &sm.bfull[slot]);
                }
                __syncwarp();
            }
        } else if (!mma_warp) {
            ok = __all_sync(0xffffffffu, mbar_wait(&sm.tfull, (uint32_t)(nit & 1), abort_flag, g.spin));
            if (ok) {
                for (int q = 0; q < nst; ++q, ++gs) {
                    const int slot = (int)(gs & 1);
                    if (gs >= kTcNbuf) {
                        ok = __all_sync(0xffffffffu,
                                        mbar_wait(&sm.empty[slot], (uint32_t)(((gs >> 1) - 1) & 1), abort_flag, g.spin));
                        if (!ok) break;
                    }
                    unsigned char* as = abuf + (size_t)slot * kTcJS * kTcJAsliceBytes;
                    for (int k = tid; k < kTcJTasks; k += kTcProdThreads) form_aj(g, sm, tabs, q, k, as);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.full[slot]);
                }
            }
        } else {
            if (lane == 0) {
                const uint32_t a0 = saddr(abuf), b0 = saddr(bbuf);
                const int nw = min(g.npad, (nb * g.colw + 15) / 16 * 16);
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nw >> 3) << 17) |
                                       ((uint32_t)(kTcM >> 4) << 24);
                bool first[kTcJAcc] = {true, true, true, true, true};
                bool mok = true;
                if (nit > 0) mok = mbar_wait(&sm.acce, (uint32_t)((nit - 1) & 1), abort_flag, g.spin);  // tensor memory drained
                tc_fence_after();
                for (int q = 0; q < nst && mok; ++q, ++gs) {
                    const int slot = (int)(gs & 1);
                    if (!(mok = mbar_wait(&sm.full[slot], (uint32_t)((gs >> 1) & 1), abort_flag, g.spin))) break;
                    if (!(mok = mbar_wait(&sm.bfull[slot], (uint32_t)((gs >> 1) & 1), abort_flag, g.spin))) break;
                    tc_fence_after();
                    const uint32_t as = a0 + slot * kTcJS * kTcJAsliceBytes, bs = b0 + slot * kTcJS * bslice;
#pragma unroll
                    for (int s = 0; s < kTcJS; ++s)
#pragma unroll
                        for (int t = 0; s + t < kTcJS; ++t) {
                            const int lv = min(s + t, kTcJAcc - 1);
                            tc_mma(tmem + (uint32_t)(lv * g.npad), sdesc16(as + s * kTcJAsliceBytes),
                                   sdesc16(bs + t * bslice), idesc, first[lv] ? 0u : 1u);
                            first[lv] = false;
                        }
                    tc_commit(&sm.empty[slot]);
                }
                if (mok) tc_commit(&sm.accf);
                ok = mok;
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            gs = __shfl_sync(0xffffffffu, gs, 0);
        }
        if (!ok) break;
        // ---- J'_{r,ijk} = Re (-i)^k sum_{n_c} n_c^k Z_r(n_c) U_ij[r, n_c] (warps 0-11) ----
        if (epi) {
            ok = __all_sync(0xffffffffu, mbar_wait(&sm.accf, (uint32_t)(nit & 1), abort_flag, g.spin));
            if (!ok) break;
            tc_fence_after();
            const int r = sm.rec[erow];
            const long long cnt = g.cls_start[L + 1] - g.cls_start[L];
            for (int grp = ethird; grp < nb * g.nd; grp += 3) {
                const int gb = grp / g.nd, d = grp - gb * g.nd;
                const int pr = sm.pairs[gb], i = pr & 7, j = pr >> 3, nk = L - i - j;
                const int* evp = g.ev + (pair_index(i, j) * g.nd + d) * g.ncols;
                cdf J[5];
#pragma unroll
                for (int kk = 0; kk < 5; ++kk) J[kk] = cdf{{0.f, 0.f}, {0.f, 0.f}};
                for (int c8 = 0; c8 < g.gw / 8; ++c8) {
                    float T[kTcJAcc][8];
#pragma unroll
                    for (int lv = 0; lv < kTcJAcc; ++lv)
                        tc_ld8(tmem + tlane + (uint32_t)(lv * g.npad + gb * g.colw + d * g.gw + 8 * c8), T[lv]);
                    if (r < 0) continue;
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const int nc = 4 * c8 + u / 2;
                        if (nc < g.ncols) {
                            cdf v;
                            v.re = df_add(df_add(df_add(two_sum(T[0][u], T[1][u]), df{T[2][u], 0.f}), df{T[3][u], 0.f}),
                                          df{T[4][u], 0.f});
                            v.im = df_add(df_add(df_add(two_sum(T[0][u + 1], T[1][u + 1]), df{T[2][u + 1], 0.f}),
                                                 df{T[3][u + 1], 0.f}),
                                          df{T[4][u + 1], 0.f});
                            const float sc = pow2f(1 + __ldg(evp + nc) - 12);  // exact power of two
                            v = cdf{df{v.re.hi * sc, v.re.lo * sc}, df{v.im.hi * sc, v.im.lo * sc}};
                            const float4 zv = tabs[erow * g.tabw + g.offZ + nc];
                            const cdf zu = cdf_mul(cdf{{zv.x, zv.y}, {zv.z, zv.w}}, v);
                            float pw = 1.f;  // n_c^k, exact
#pragma unroll
                            for (int kk = 0; kk < 5; ++kk) {
                                if (kk <= nk) J[kk] = cdf{df_add(J[kk].re, df_mulf(zu.re, pw)), df_add(J[kk].im, df_mulf(zu.im, pw))};
                                pw *= (float)nc;
                            }
                        }
                    }
                }
                if (r >= 0) {
                    double* jp = g.Jp + ((long long)(g.d0 + d) * g.nparts + sm.ipart) * g.jp_total + g.term_base[L] +
                                 (r - g.cls_start[L]);
#pragma unroll
                    for (int kk = 0; kk < 5; ++kk)
                        if (kk <= nk) {
                            const df re = rot_mi(J[kk], kk).re;
                            jp[(long long)sm.tidx[gb][kk] * cnt] = (double)re.hi + (double)re.lo;
                        }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acce);
        }
        ++nit;
        // the tables, records and blocks are rewritten by the next item
        if (!(ok = prod_sync(&sm.psync, ph, abort_flag, lane, g.spin) && ok)) break;
    }
    if (load_warp && lane == 0) {
        // bulk copies still in flight (after a failed wait) land before the CTA exits
        for (int b = 0; b < kTcNbuf && b < gs; ++b) {
            const long long last = gs - 1 - ((gs - 1 - b) % kTcNbuf);
            const long long t0 = clock64();
            while (!mbar_test(&sm.bfull[b], (uint32_t)((last >> 1) & 1)) && clock64() - t0 < kTcSpinCycles) {
            }
        }
        if (ntab > 0) {
            const long long t0 = clock64();
            while (!mbar_test(&sm.tfull, (uint32_t)((ntab - 1) & 1)) && clock64() - t0 < kTcSpinCycles) {
            }
        }
    }
    if (mma_warp) {
        // everything issued completes before tensor memory is freed
        if (lane == 0) {
            tc_commit(&sm.done);
            const long long t0 = clock64();
            while (!mbar_test(&sm.done, 0u) && clock64() - t0 < kTcSpinCycles) {
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(g.err, 1);
    if (mma_warp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

size_t tc_j_smem_bytes(int npad, int tabw) {
    const size_t need = (size_t)kTcNbuf * kTcJS * kTcJAsliceBytes + (size_t)kTcNbuf * kTcJS * npad * 32 +
                        (size_t)kTcM * tabw * 16 + sizeof(TcJSmem) + 64;
    return std::max<size_t>(need, 120 * 1024);
}

}  // namespace

int tc_supported(const ftcj_plan* P) { return P->ortho ? 1 : 0; }

// clock-cycle budget of one wait between the kernels' roles
long long tc_spin(const ftcj_plan* P) {
    return P->params.tc_wait_log2 > 0 ? (1LL << P->params.tc_wait_log2) : kTcSpinCycles;
}

int setup_tc_j(ftcj_plan* P);

// Plan-time set-up of the tensor-core form: the column axis, the rows and
// their half-sphere map, the factor tables, the windows (class, block group,
// 512 records sorted by width) and the partial-row count.
int setup_tc(ftcj_plan* P) {
    if (!P->ortho) return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction needs an orthorhombic cell");
    if (P->precision != FTCJ_PREC_SPLIT)
        return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction is part of the split-precision form");
    if (P->d_rec_gcut) return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction walks the whole sphere");
    if (P->npairs >= (1 << 24)) return fail(FTCJ_EUNSUPPORTED, "more than 2^24 pair records");
    const int64_t ngh = P->ng_half;
    int64_t recs_by_class[kNclass];
    for (int L = 0; L < kNclass; ++L) recs_by_class[L] = P->class_start[L + 1] - P->class_start[L];
    // the column axis: operand work ~ row tiles x (record passes x 128 rows + B entries), per density group
    struct AxisPlan {
        std::vector<std::pair<int, int>> rows;
        int ncols = 0, nd = 0, colw = 0, G = 0, npad = 0;
    } best;
    int best_c = -1;
    double best_cost = 1e300;
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        AxisPlan ap;
        std::set<std::pair<int, int>> rs;
        int ncmax = 0;
        for (int64_t q = 0; q < ngh; ++q) {
            int n[3] = {P->gvec[3 * q], P->gvec[3 * q + 1], P->gvec[3 * q + 2]};
            if (n[c] < 0)
                for (int x = 0; x < 3; ++x) n[x] = -n[x];
            rs.insert({n[a], n[b]});
            ncmax = std::max(ncmax, n[c]);
        }
        ap.ncols = ncmax + 1;
        for (ap.nd = P->max_dens; ap.nd >= 1; --ap.nd) {
            tc_columns(ap.nd, ap.ncols, &ap.colw, &ap.G, &ap.npad);
            if (ap.G > 0) break;
        }
        if (ap.nd < 1 || ap.G < 1) continue;
        ap.rows.assign(rs.begin(), rs.end());
        const double mt = (double)((ap.rows.size() + kTcM - 1) / kTcM);
        const double launches = (double)((P->max_dens + ap.nd - 1) / ap.nd);
        double work = 0.0;
        for (int L = 0; L < kNclass; ++L) {
            const int nb = (L + 1) * (L + 2) / 2;
            const double passes = (double)((nb + ap.G - 1) / ap.G);
            work += (double)recs_by_class[L] * (passes * kTcM + 1.5 * nb * ap.nd * ap.ncols);
        }
        const double cost = launches * mt * work;
        if (cost < best_cost) {
            best_cost = cost;
            best_c = c;
            best = ap;
        }
    }
    if (best_c < 0) return fail(FTCJ_EUNSUPPORTED, "the sphere is too long on every axis for the tensor-core tile");
    const int c = best_c, a = (c + 1) % 3, b = (c + 2) % 3;
    P->tc_axis[0] = a;
    P->tc_axis[1] = b;
    P->tc_axis[2] = c;
    P->tc_ncols = best.ncols;
    P->tc_nd = best.nd;
    P->tc_colw = best.colw;
    P->tc_G = best.G;
    P->tc_npad = best.npad;
    P->tc_rows = (int)best.rows.size();
    P->tc_mtiles = (P->tc_rows + kTcM - 1) / kTcM;
    // half-sphere map: row (n_a, n_b), column n_c >= 0
    std::vector<int> map((size_t)P->tc_rows * P->tc_ncols, INT_MIN);
    {
        std::vector<std::pair<int, int>>& rows = best.rows;
        for (int64_t q = 0; q < ngh; ++q) {
            int n[3] = {P->gvec[3 * q], P->gvec[3 * q + 1], P->gvec[3 * q + 2]};
            bool cj = false;
            if (n[c] < 0) {
                for (int x = 0; x < 3; ++x) n[x] = -n[x];
                cj = true;
            }
            const auto it = std::lower_bound(rows.begin(), rows.end(), std::make_pair(n[a], n[b]));
            const size_t rix = (size_t)(it - rows.begin());
            map[rix * P->tc_ncols + n[c]] = cj ? ~(int)q : (int)q;
        }
    }
    std::vector<int2> rowv(best.rows.size());
    int nam = 0, nbm = 0;
    for (size_t i = 0; i < best.rows.size(); ++i) {
        rowv[i] = make_int2(best.rows[i].first, best.rows[i].second);
        nam = std::max(nam, std::abs(best.rows[i].first));
        nbm = std::max(nbm, std::abs(best.rows[i].second));
    }
    P->tc_nna = nam + 1;
    P->tc_nnb = nbm + 1;
    // factor tables first: the windows below sort records by their width
    const int tabw = P->tc_nna + P->tc_nnb + P->tc_ncols;
    P->tc_tabw = tabw;
    const size_t ntab = (size_t)std::max<int64_t>(P->npairs, 1) * tabw;
    FTCJ_CUDA(cudaMalloc(&P->d_tc_tab, sizeof(float4) * ntab));
    P->device_bytes += sizeof(float4) * ntab;
    FTCJ_CUDA(cudaMalloc(&P->d_tc_cl, sizeof(float) * std::max<int64_t>(P->npairs, 1)));
    P->device_bytes += sizeof(float) * std::max<int64_t>(P->npairs, 1);
    FTCJ_CUDA(cudaMalloc(&P->d_tc_err, sizeof(int)));
    FTCJ_CUDA(cudaMemset(P->d_tc_err, 0, sizeof(int)));
    std::vector<float> clh((size_t)std::max<int64_t>(P->npairs, 1), 0.f);
    if (P->npairs > 0) {
        const long long n = P->npairs * (long long)tabw;
        k_tc_tables<<<(unsigned)((n + 255) / 256), 256>>>(P->d_walk, P->npairs, a, b, c, P->tc_nna, P->tc_nnb,
                                                        P->tc_ncols, P->M[4 * a], P->M[4 * b], P->M[4 * c],
                                                        reinterpret_cast<float4*>(P->d_tc_tab), P->d_tc_cl);
        FTCJ_CUDA(cudaGetLastError());
        FTCJ_CUDA(cudaMemcpy(clh.data(), P->d_tc_cl, sizeof(float) * P->npairs, cudaMemcpyDeviceToHost));
    }
    // windows: for each class L, its (i, j) blocks in groups of G, and the
    // class's records sorted by width c = 1/4p in blocks of 512 (the K order of
    // the matrix product; records of similar width have entries of similar size)
    std::vector<int> wrec, wpairs;
    std::vector<int4> winfo;
    std::vector<int> pos((size_t)std::max<int64_t>(P->npairs, 1), 0);
    // Hermite terms in the K order: [dens][class][term][position], each class's stride a multiple of 16
    P->tc_dp_total = 0;
    for (int L = 0; L < kNclass; ++L) {
        P->tc_dp_base[L] = P->tc_dp_total;
        P->tc_dp_stride[L] = (recs_by_class[L] + kTcStageK - 1) / kTcStageK * kTcStageK;
        P->tc_dp_total += (long long)nterms(L) * P->tc_dp_stride[L];
    }
    for (int L = 0; L < kNclass; ++L) {
        std::vector<int> recs;
        for (int64_t r = P->class_start[L]; r < P->class_start[L + 1]; ++r) recs.push_back((int)r);
        if (recs.empty()) continue;
        std::stable_sort(recs.begin(), recs.end(), [&](int x, int y) { return clh[x] < clh[y]; });
        for (size_t k = 0; k < recs.size(); ++k) pos[recs[k]] = (int)k;
        std::vector<int> blocks;
        for (int i = 0; i <= L; ++i)
            for (int j = 0; i + j <= L; ++j) blocks.push_back(i | (j << 3));
        for (size_t g0 = 0; g0 < blocks.size(); g0 += P->tc_G) {
            const int nb = (int)std::min<size_t>(P->tc_G, blocks.size() - g0);
            const int first = (int)wpairs.size();
            wpairs.insert(wpairs.end(), blocks.begin() + g0, blocks.begin() + g0 + nb);
            for (size_t r0 = 0; r0 < recs.size(); r0 += kTcWin) {
                winfo.push_back(make_int4(L, nb, first, (int)r0));
                for (int k = 0; k < kTcWin; ++k) wrec.push_back(r0 + k < recs.size() ? recs[r0 + k] : -1);
            }
        }
    }
    if (winfo.empty()) {  // no records: one empty window keeps the launch shape valid
        winfo.push_back(make_int4(0, 0, 0, 0));
        wrec.assign(kTcWin, -1);
    }
    P->tc_nwin = (int)winfo.size();
    // MMA work of one pass: per window and row tile, 32 stages x 2 k-steps x 21 slice products of
    // M = 128 rows, N = the window's columns, K = 16, for every density group
    P->tc_mma_flops = 0;
    for (int d0 = 0; d0 < P->max_dens; d0 += P->tc_nd) {
        const int ndg = std::min(P->tc_nd, P->max_dens - d0);
        const int colw = round_up(2 * ndg * P->tc_ncols, 8), np = round_up(P->tc_G * colw, 16);
        for (const int4& wi : winfo) {
            const long long nw = std::min(np, round_up(std::max(1, wi.y) * colw, 16));
            P->tc_mma_flops += (long long)P->tc_mtiles * kTcStagesPerWin * 2 * 21 * 2LL * kTcM * nw * 16;
        }
    }
    // window groups: one CTA per SM over all (group, row tile) pairs, so the
    // grid is a single wave of equal CTAs (a partial second wave would double the pass)
    const int want = std::max(1, std::min(P->tc_nwin, P->num_sms / std::max(1, P->tc_mtiles)));
    P->tc_wpg = std::max(1, (P->tc_nwin + want - 1) / want);
    P->tc_ngroups = (P->tc_nwin + P->tc_wpg - 1) / P->tc_wpg;
    // table slots in flight: as many as shared memory holds, 2 to 4
    int dev = 0, optin = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    P->tc_tslots = 0;
    for (int nts = kTcTabSlotsMax; nts >= 2 && !P->tc_tslots; --nts)
        if (tc_smem_bytes(P->tc_npad, tabw, P->tc_G, P->tc_nd, nts) <= (size_t)optin) P->tc_tslots = nts;
    if (!P->tc_tslots)
        return fail(FTCJ_EUNSUPPORTED, "the G sphere is too long for the tensor-core kernel's shared-memory tables");
    int rc;
    int2* rows_dev = nullptr;
    if ((rc = tc_upload(P, &rows_dev, rowv))) return rc;
    P->d_tc_rows = rows_dev;
    if ((rc = tc_upload(P, &P->d_tc_map, map))) return rc;
    if ((rc = tc_upload(P, &P->d_tc_kappa, wrec))) return rc;
    if ((rc = tc_upload(P, &P->d_tc_wpairs, wpairs))) return rc;
    if ((rc = tc_upload(P, &P->d_tc_pos, pos))) return rc;
    int4* winfo_dev = nullptr;
    if ((rc = tc_upload(P, &winfo_dev, winfo))) return rc;
    P->d_tc_winfo = winfo_dev;
    if ((rc = tc_upload(P, &P->d_tc_ebw, std::vector<int>((size_t)P->tc_nwin * kTcEbMax, -100)))) return rc;
    if ((rc = tc_upload(P, &P->d_tc_clw, std::vector<float>((size_t)P->tc_nwin, 0.f)))) return rc;
    if ((rc = allow_dynamic_smem((const void*)k_tc_rho, tc_smem_bytes(P->tc_npad, tabw, P->tc_G, P->tc_nd, P->tc_tslots))))
        return rc;
    return setup_tc_j(P);
}

int launch_tc_rho(ftcj_plan* P, int ndens, cudaStream_t s) {
    if (P->ng_half == 0 || P->npairs == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_rho_part, 0, sizeof(double2) * (size_t)ndens * P->tc_ngroups * P->ng_half, s));
        return FTCJ_OK;
    }
    TcArgs g;
    g.rows = reinterpret_cast<const int2*>(P->d_tc_rows);
    g.map = P->d_tc_map;
    g.wrec = P->d_tc_kappa;
    g.winfo = reinterpret_cast<const int4*>(P->d_tc_winfo);
    g.wpairs = P->d_tc_wpairs;
    g.tab = reinterpret_cast<const float4*>(P->d_tc_tab);
    g.cl = P->d_tc_cl;
    g.Dp = reinterpret_cast<const float2*>(P->d_Dp);
    g.dp_total = P->tc_dp_total;
    for (int cc = 0; cc < kNclass; ++cc) {
        g.dp_base[cc] = P->tc_dp_base[cc];
        g.dp_stride[cc] = P->tc_dp_stride[cc];
    }
    g.out = reinterpret_cast<double2*>(P->d_rho_part);
    g.ng_half = P->ng_half;
    g.err = P->d_tc_err;
    g.Maa = (float)P->M[4 * P->tc_axis[0]];
    g.Mbb = (float)P->M[4 * P->tc_axis[1]];
    g.Mcc = (float)P->M[4 * P->tc_axis[2]];
    g.ax = P->tc_axis[0];
    g.bx = P->tc_axis[1];
    g.cx = P->tc_axis[2];
    g.tabw = P->tc_tabw;
    g.offY = P->tc_nna;
    g.offZ = P->tc_nna + P->tc_nnb;
    g.ncols = P->tc_ncols;
    g.G = P->tc_G;
    g.nwin = P->tc_nwin;
    g.win_per_group = P->tc_wpg;
    g.ngroups = P->tc_ngroups;
    g.nrows = P->tc_rows;
    g.spin = tc_spin(P);
    g.ebw = P->d_tc_ebw;
    g.clw = P->d_tc_clw;
    const size_t smem = tc_smem_bytes(P->tc_npad, P->tc_tabw, P->tc_G, P->tc_nd, P->tc_tslots);
    for (int d0 = 0; d0 < ndens; d0 += P->tc_nd) {
        g.d0 = d0;
        g.nd = std::min(P->tc_nd, ndens - d0);
        int colw, Gx, npad;
        tc_columns(g.nd, g.ncols, &colw, &Gx, &npad);
        // the plan's block count G is kept; a smaller last density group only narrows each block
        g.colw = colw;
        g.npad = round_up(P->tc_G * colw, 16);
        k_tc_rho_bounds<<<(unsigned)P->tc_nwin, 256, 0, s>>>(g);
        FTCJ_CUDA(cudaGetLastError());
        k_tc_rho<<<dim3((unsigned)P->tc_ngroups, (unsigned)P->tc_mtiles), kTcThreadsAll, smem, s>>>(g, P->tc_tslots);
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}

int tc_rho_launches(const ftcj_plan* P, int nd) { return 2 * ((nd + P->tc_nd - 1) / P->tc_nd); }

// Plan-time set-up of the tensor-core back-contraction: densities per
// launch, (i, j) blocks per work item, the items and the V_ij tile buffer.
// tc_j stays false, and the split walk runs the back-contraction, where the
// rows exceed one exact accumulation, one density's columns exceed the MMA
// width, or the factor tables exceed shared memory.
int setup_tc_j(ftcj_plan* P) {
    P->tc_j = false;
    const int gw = round_up(2 * P->tc_ncols, 8);
    int64_t tiles[kNclass];
    for (int L = 0; L < kNclass; ++L) tiles[L] = (P->class_start[L + 1] - P->class_start[L] + kTcM - 1) / kTcM;
    // densities per launch: the fewest A^T formations (items x launches)
    int nd_best = 0, G_best = 0;
    double cost_best = 1e300;
    for (int nd = 1; nd <= P->max_dens; ++nd) {
        const int colw = nd * gw;
        if (colw > kTcJNmax) break;
        const int G = std::min(kTcGmax, kTcJNmax / colw);
        double items = 0.0;
        for (int L = 0; L < kNclass; ++L) {
            const int nb = (L + 1) * (L + 2) / 2;
            items += (double)tiles[L] * ((nb + G - 1) / G);
        }
        const double cost = (double)((P->max_dens + nd - 1) / nd) * items;
        if (cost <= cost_best) {
            cost_best = cost;
            nd_best = nd;
            G_best = G;
        }
    }
    if (!nd_best) return FTCJ_OK;
    const int npad = round_up(G_best * nd_best * gw, 16);
    int dev = 0, optin = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (tc_j_smem_bytes(npad, P->tc_tabw) > (size_t)optin) return FTCJ_OK;
    // row parts of at most 64 stages, as even as the stage count allows
    const int nstage = (P->tc_rows + kTcJStageM - 1) / kTcJStageM;
    const int spp = (nstage + (nstage + kTcJPartStages - 1) / kTcJPartStages - 1) /
                    ((nstage + kTcJPartStages - 1) / kTcJPartStages);
    const int nparts = (nstage + spp - 1) / spp;  // every part holds at least one stage
    // work items, the costliest classes first: (class, block group, 128 records, row part)
    std::vector<int4> items;
    std::vector<int> ipairs;
    for (int L = kNclass - 1; L >= 0; --L) {
        if (!tiles[L]) continue;
        std::vector<int> blocks;
        for (int i = 0; i <= L; ++i)
            for (int j = 0; i + j <= L; ++j) blocks.push_back(i | (j << 3));
        for (size_t g0 = 0; g0 < blocks.size(); g0 += G_best) {
            const int nb = (int)std::min<size_t>(G_best, blocks.size() - g0);
            const int first = (int)ipairs.size();
            ipairs.insert(ipairs.end(), blocks.begin() + g0, blocks.begin() + g0 + nb);
            for (int64_t t = 0; t < tiles[L]; ++t)
                for (int h = 0; h < nparts; ++h)
                    items.push_back(make_int4(L | (h << 8), nb, first, (int)(P->class_start[L] + t * kTcM)));
        }
    }
    P->tc_jnd = nd_best;
    P->tc_jgw = gw;
    P->tc_jG = G_best;
    P->tc_jnpad = npad;
    P->tc_jnstage = nstage;
    P->tc_jparts = nparts;
    P->tc_jspp = spp;
    P->tc_jnitems = (int)items.size();
    // MMA work of one back-contraction over max_dens densities: per item and stage 21 slice
    // products of M = 128 records, N = the item's columns, K = 16
    P->tc_j_mma_flops = 0;
    for (int d0 = 0; d0 < P->max_dens; d0 += nd_best) {
        const int colw = std::min(nd_best, P->max_dens - d0) * gw, np = round_up(G_best * colw, 16);
        for (const int4& it : items) {
            const int part = it.x >> 8, nst = std::min(spp, nstage - part * spp);
            P->tc_j_mma_flops +=
                (long long)nst * kTcJProducts * 2LL * kTcM * std::min(np, round_up(it.y * colw, 16)) * 16;
        }
    }
    int rc;
    int4* items_dev = nullptr;
    if ((rc = tc_upload(P, &items_dev, items))) return rc;
    P->d_tc_jitems = items_dev;
    if ((rc = tc_upload(P, &P->d_tc_jpairs, ipairs))) return rc;
    const size_t nvs = (size_t)kTcPairsAll * P->tc_jnstage * kTcJS * (size_t)nd_best * gw * 16;
    FTCJ_CUDA(cudaMalloc(&P->d_tc_vs, sizeof(__nv_bfloat16) * nvs));
    P->device_bytes += sizeof(__nv_bfloat16) * nvs;
    FTCJ_CUDA(cudaMemset(P->d_tc_vs, 0, sizeof(__nv_bfloat16) * nvs));
    const size_t nev = (size_t)kTcPairsAll * nd_best * P->tc_ncols;
    FTCJ_CUDA(cudaMalloc(&P->d_tc_ev, sizeof(int) * nev));
    P->device_bytes += sizeof(int) * nev;
    if ((rc = allow_dynamic_smem((const void*)k_tc_j, tc_j_smem_bytes(npad, P->tc_tabw)))) return rc;
    P->tc_j = true;
    return FTCJ_OK;
}

int launch_tc_j(ftcj_plan* P, int ndens, const double* W, cudaStream_t s) {
    if (P->ng_half == 0 || P->npairs == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_Jp, 0, sizeof(double) * (size_t)ndens * P->tc_jparts * P->total_terms, s));
        return FTCJ_OK;
    }
    TcJArgs g;
    g.rows = reinterpret_cast<const int2*>(P->d_tc_rows);
    g.map = P->d_tc_map;
    g.W = reinterpret_cast<const double2*>(W);
    g.items = reinterpret_cast<const int4*>(P->d_tc_jitems);
    g.ipairs = P->d_tc_jpairs;
    g.tab = reinterpret_cast<const float4*>(P->d_tc_tab);
    g.vs = reinterpret_cast<__nv_bfloat16*>(P->d_tc_vs);
    g.ev = P->d_tc_ev;
    g.Jp = P->d_Jp;
    g.ng_half = P->ng_half;
    g.jp_total = P->total_terms;
    for (int c = 0; c <= kNclass; ++c) g.cls_start[c] = P->class_start[c];
    for (int c = 0; c < kNclass; ++c) g.term_base[c] = P->term_base[c];
    g.err = P->d_tc_err;
    g.ax = P->tc_axis[0];
    g.bx = P->tc_axis[1];
    g.cx = P->tc_axis[2];
    g.tabw = P->tc_tabw;
    g.offY = P->tc_nna;
    g.offZ = P->tc_nna + P->tc_nnb;
    g.ncols = P->tc_ncols;
    g.gw = P->tc_jgw;
    g.nrows = P->tc_rows;
    g.nstage = P->tc_jnstage;
    g.nitems = P->tc_jnitems;
    g.nparts = P->tc_jparts;
    g.spin = tc_spin(P);
    g.spp = P->tc_jspp;
    const size_t smem = tc_j_smem_bytes(P->tc_jnpad, P->tc_tabw);
    const int grid = std::max(1, std::min(P->num_sms, P->tc_jnitems));
    for (int d0 = 0; d0 < ndens; d0 += P->tc_jnd) {
        g.d0 = d0;
        g.nd = std::min(P->tc_jnd, ndens - d0);
        // the plan's block count is kept; a smaller last density group only narrows each block
        g.colw = g.nd * g.gw;
        g.npad = round_up(P->tc_jG * g.colw, 16);
        k_tc_vbound<<<(unsigned)(kTcPairsAll * g.nd * g.ncols), 256, 0, s>>>(g);
        FTCJ_CUDA(cudaGetLastError());
        const long long nv = (long long)kTcPairsAll * g.nstage * kTcJStageM * g.nd * g.ncols;
        k_tc_vslice<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(g);
        FTCJ_CUDA(cudaGetLastError());
        k_tc_j<<<(unsigned)grid, kTcThreadsAll, smem, s>>>(g);
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}

int tc_j_launches(const ftcj_plan* P, int nd) { return 3 * ((nd + P->tc_jnd - 1) / P->tc_jnd); }

}  // namespace ftcj
