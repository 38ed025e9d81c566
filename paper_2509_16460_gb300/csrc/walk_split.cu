// Split-precision form of the structure-factor pass (Alg. 1) and of the
// back-contraction (Alg. S1).
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so here every per-point and
// per-line operation runs on the FP32 pipe in double-float arithmetic (a value
// is hi + lo, two FP32 numbers, ~48 significant bits; df.cuh).  FP64 is kept for
// what needs it once per pair and chunk: the range reduction of the phase
// argument n.f, exp(-|G|^2/4p) and the phase at the first line of each walk
// chunk (k_split_setup, once per plan), the per-G sums of the block rows, and
// E_J (k_rho_reduce, shared with the FP64 form).
//
// The walk is the FP64 form's (walk.cu) with the Gaussian and the phase
// advanced together: along a line gp(n1) = exp(-|G|^2/4p) exp(-2 pi i n.f) is
// multiplied by the complex ratio R(n1) = r(n1) exp(-2 pi i f1), and R by the
// real q1 = exp(-2c M11); lines and planes likewise carry complex ratios.
#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "ftcj_internal.h"

namespace ftcj {
namespace {

constexpr int kSBatch = 8;  // points per reduction batch of the split rho walk (4 lanes per point)


struct Layout {
    long long start[kNclass + 1];
    long long base[kNclass];
    long long total;
};

// walk state at a line, all complex: plane centre (0,0,n3) and line centre (0,n2,n3)
struct SState {
    cdf gpC, Tc, RF0c, RB0c, rF0c, rB0c;  // plane: value, n3-step ratio, n2-step ratios at n2=0, n1-ratios at n2=0
    cdf gpL, Sd, RfL, RbL;                // line: value, n2-step ratio (current direction), n1-ratios
};

__device__ __forceinline__ cdf to_cdf(double re, double im) { return cdf{df_from_double(re), df_from_double(im)}; }

__device__ __forceinline__ void cexp_phase(double th, double& re, double& im) {
    th -= rint(th);
    double s, c;
    sincospi(2.0 * th, &s, &c);
    re = c;
    im = -s;
}

// closed-form state at line (n2, n3) in FP64, stored as double-float
__device__ void split_state(const PairWalk& w, const double* M6, int n2, int n3, SState& s) {
    const double c = w.c;
    const double M11 = M6[0], M22 = M6[1], M33 = M6[2], M12 = M6[3], M13 = M6[4], M23 = M6[5];
    const double a2 = (double)n2, a3 = (double)n3;
    double p3r, p3i, p23r, p23i;
    cexp_phase(a3 * w.f3, p3r, p3i);
    cexp_phase(a2 * w.f2 + a3 * w.f3, p23r, p23i);
    double g;
    g = exp(-c * M33 * a3 * a3);
    s.gpC = to_cdf(g * p3r, g * p3i);
    g = exp(-c * M33 * (2.0 * a3 + 1.0));
    s.Tc = to_cdf(g * w.e3r, g * w.e3i);
    g = exp(-c * (M22 + 2.0 * M23 * a3));
    s.RF0c = to_cdf(g * w.e2r, g * w.e2i);
    g = exp(-c * (M22 - 2.0 * M23 * a3));
    s.RB0c = to_cdf(g * w.e2r, -g * w.e2i);
    g = exp(-c * (M11 + 2.0 * M13 * a3));
    s.rF0c = to_cdf(g * w.e1r, g * w.e1i);
    g = exp(-c * (M11 - 2.0 * M13 * a3));
    s.rB0c = to_cdf(g * w.e1r, -g * w.e1i);
    g = exp(-c * (M22 * a2 * a2 + 2.0 * M23 * a2 * a3 + M33 * a3 * a3));
    s.gpL = to_cdf(g * p23r, g * p23i);
    if (n2 >= 0) {
        g = exp(-c * (M22 * (2.0 * a2 + 1.0) + 2.0 * M23 * a3));
        s.Sd = to_cdf(g * w.e2r, g * w.e2i);
    } else {
        g = exp(-c * (M22 * (1.0 - 2.0 * a2) - 2.0 * M23 * a3));
        s.Sd = to_cdf(g * w.e2r, -g * w.e2i);
    }
    const double beta = M12 * a2 + M13 * a3;
    g = exp(-c * (M11 + 2.0 * beta));
    s.RfL = to_cdf(g * w.e1r, g * w.e1i);
    g = exp(-c * (M11 - 2.0 * beta));
    s.RbL = to_cdf(g * w.e1r, -g * w.e1i);
}

// per-pair real multipliers of the recurrences, double-float
struct SConst {
    df q1, q2, q3, x12, y12, x13, y13, x23, y23;
};

// Once per plan: chunk-start states and the multipliers of every pair record.
__global__ void k_split_setup(const PairWalk* __restrict__ walk, long long npairs, const WLine* __restrict__ lines,
                              const WChunk* __restrict__ chunks, int nchunks, SState* __restrict__ init,
                              SConst* __restrict__ cst, CellConst cc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (i >= npairs) return;
    const PairWalk w = walk[i];
    const WLine ln = lines[chunks[ch].l0];
    SState s;
    split_state(w, cc.M6, ln.n2, ln.n3, s);
    init[(long long)ch * npairs + i] = s;
    if (ch == 0) {
        SConst k;
        k.q1 = df_from_double(w.q1);
        k.q2 = df_from_double(w.q2);
        k.q3 = df_from_double(w.q3);
        k.x12 = df_from_double(w.x12);
        k.y12 = df_from_double(w.y12);
        k.x13 = df_from_double(w.x13);
        k.y13 = df_from_double(w.y13);
        k.x23 = df_from_double(w.x23);
        k.y23 = df_from_double(w.y23);
        cst[i] = k;
    }
}

__device__ __forceinline__ SConst idle_const() {
    SConst k;
    const df one{1.f, 0.f};
    k.q1 = k.q2 = k.q3 = k.x12 = k.y12 = k.x13 = k.y13 = k.x23 = k.y23 = one;
    return k;
}

__device__ __forceinline__ SState idle_state() {
    SState s;
    const cdf z{{0.f, 0.f}, {0.f, 0.f}};
    s.gpC = s.Tc = s.RF0c = s.RB0c = s.rF0c = s.rB0c = z;
    s.gpL = s.Sd = s.RfL = s.RbL = z;
    return s;
}

// One transition of the walk program.  With ORTHO (the per-record X(n1)
// table serves every line) the n1 ratios RfL, RbL, rF0c, rB0c are not used
// and not advanced.  Line steps inside a plane use the deferred-renormalisation
// products (at most one plane's lines deep); plane steps keep the plane values
// renormalised, and every plane restarts the line values from them.
template <bool ORTHO>
__device__ __forceinline__ void split_step(const SConst& k, int op, SState& s, const SState* init_p, bool valid) {
    switch (op) {
        case OP_FIRST:
            s = valid ? *init_p : idle_state();
            break;
        case OP_N2F:
            s.gpL = cdf_mul_u(s.gpL, s.Sd);
            s.Sd = cdf_scale_u(s.Sd, k.q2);
            if (!ORTHO) {
                s.RfL = cdf_scale_u(s.RfL, k.x12);
                s.RbL = cdf_scale_u(s.RbL, k.y12);
            }
            break;
        case OP_NEGSTART:
            s.gpL = cdf_mul_u(s.gpC, s.RB0c);
            s.Sd = cdf_scale_u(s.RB0c, k.q2);
            if (!ORTHO) {
                s.RfL = cdf_scale_u(s.rF0c, k.y12);
                s.RbL = cdf_scale_u(s.rB0c, k.x12);
            }
            break;
        case OP_N2B:
            s.gpL = cdf_mul_u(s.gpL, s.Sd);
            s.Sd = cdf_scale_u(s.Sd, k.q2);
            if (!ORTHO) {
                s.RfL = cdf_scale_u(s.RfL, k.y12);
                s.RbL = cdf_scale_u(s.RbL, k.x12);
            }
            break;
        default:  // OP_N3
            s.gpC = cdf_mul(s.gpC, s.Tc);
            s.Tc = cdf_scale(s.Tc, k.q3);
            s.RF0c = cdf_scale(s.RF0c, k.x23);
            s.RB0c = cdf_scale(s.RB0c, k.y23);
            if (!ORTHO) {
                s.rF0c = cdf_scale(s.rF0c, k.x13);
                s.rB0c = cdf_scale(s.rB0c, k.y13);
            }
            s.gpL = s.gpC;
            s.Sd = s.RF0c;
            s.RfL = s.rF0c;
            s.RbL = s.rB0c;
            break;
    }
}

template <int L>
__device__ __forceinline__ void powers23f(int n2, int n3, float pq[L + 1][L + 1]) {
    float p2[L + 1], p3[L + 1];
    p2[0] = 1.f;
    p3[0] = 1.f;
#pragma unroll
    for (int j = 1; j <= L; ++j) {
        p2[j] = p2[j - 1] * (float)n2;  // exact: |n|^4 < 2^24
        p3[j] = p3[j - 1] * (float)n3;
    }
#pragma unroll
    for (int j = 0; j <= L; ++j)
#pragma unroll
        for (int k = 0; k + j <= L; ++k) pq[j][k] = p2[j] * p3[k];
}

// ---- rho -----------------------------------------------------------------

__device__ __forceinline__ cdf unpack(float4 v) { return cdf{{v.x, v.y}, {v.z, v.w}}; }

// sum_i c_i x^i for an integer-valued x (|x|^L exact in FP32): the terms are
// independent products added in a pairwise tree, which gives the warp more
// independent instructions than Horner's serial chain at the same count
template <int L>
__device__ __forceinline__ cdf poly_at(const cdf* c, float x) {
    float p[L + 1];
    p[0] = 1.f;
#pragma unroll
    for (int i = 1; i <= L; ++i) p[i] = p[i - 1] * x;
    cdf t[L + 1];
    t[0] = c[0];
#pragma unroll
    for (int i = 1; i <= L; ++i) t[i] = cdf{df_mulf_u(c[i].re, p[i]), df_mulf_u(c[i].im, p[i])};
#pragma unroll
    for (int w = 1; w <= L; w *= 2)
#pragma unroll
        for (int i = 0; i + w <= L; i += 2 * w) t[i] = cdf_add_u(t[i], t[i + w]);
    return t[0];
}

// Sums the batch's contributions over the block's 128 records: in warp w the
// four lanes j, j+8, j+16, j+24 each add a quarter of point j's column of the
// warp's 32 records, two shuffles join the quarters, and the four warp sums
// are added into the row.  Not inlined: one copy serves every call site of
// the five record classes, which keeps the walk inside the instruction cache.
__device__ __noinline__ void split_flush(float4* buf, float4* red, float4* row, const int* pidx, int rbase,
                                        int nvalid) {
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, wv = tid >> 5;
    const int j = lane & (kSBatch - 1), quarter = lane / kSBatch;
    cdf s{{0.f, 0.f}, {0.f, 0.f}};
    if (j < nvalid) {
        const float4* b = buf + j * (kTile + 1) + wv * 32 + quarter * 8;
        cdf t[4];
#pragma unroll
        for (int k = 0; k < 8; k += 2) t[k / 2] = cdf_add_u(unpack(b[k]), unpack(b[k + 1]));
        s = cdf_add_u(cdf_add_u(t[0], t[1]), cdf_add_u(t[2], t[3]));  // pairwise: depth 3, not 8
    }
#pragma unroll
    for (int off = 16; off >= kSBatch; off >>= 1) {
        cdf o;
        o.re.hi = __shfl_down_sync(0xffffffffu, s.re.hi, off);
        o.re.lo = __shfl_down_sync(0xffffffffu, s.re.lo, off);
        o.im.hi = __shfl_down_sync(0xffffffffu, s.im.hi, off);
        o.im.lo = __shfl_down_sync(0xffffffffu, s.im.lo, off);
        s = cdf_add_u(s, o);
    }
    if (quarter == 0 && j < nvalid) red[wv * 32 + j] = make_float4(s.re.hi, s.re.lo, s.im.hi, s.im.lo);
    __syncthreads();
    if (tid < nvalid) {
        const int pr = pidx ? pidx[tid] : rbase + tid;  // point indices given, or consecutive points
        cdf r = unpack(row[pr]);
#pragma unroll
        for (int q = 0; q < kTile / 32; ++q) r = cdf_add_u(r, unpack(red[q * 32 + tid]));
        r = cdf_norm(r);
        row[pr] = make_float4(r.re.hi, r.re.lo, r.im.hi, r.im.lo);
    }
}

// Builds the record's table X(n1) = exp(-c M11 n1^2) exp(-2 pi i f1 n1) for
// n1 in [0, nx) with the line-independent ratios of an orthorhombic cell (the
// first line's RfL and q1).  There the backward ratio is the conjugate of the
// forward one, so X(-n1) = conj X(n1) and the half table serves both ends.
__device__ __forceinline__ void build_xtab(const SState& s0, const df q1, int nx, float4* Xs, int tid) {
    cdf x{{1.f, 0.f}, {0.f, 0.f}};
    cdf R = s0.RfL;
    for (int n = 0; n < nx; ++n) {
        Xs[n * kTile + tid] = make_float4(x.re.hi, x.re.lo, x.im.hi, x.im.lo);
        x = cdf_mul(x, R);
        R = cdf_scale(R, q1);
    }
}

// X(m) from the half table: conj X(-m) for m < 0 (dir 1 walks m < 0)
__device__ __forceinline__ cdf xtab_at(const float4* Xs, int m, int dir, int tid) {
    const float4 v = Xs[(dir == 0 ? m : -m) * kTile + tid];
    const float sg = dir == 0 ? 1.f : -1.f;
    return cdf{{v.x, v.y}, {sg * v.z, sg * v.w}};
}

// The tile's part of a line under its G radius (per-pair cutoffs): the n1
// with qa n1^2 + 2 qb n1 + qc < R2, intersected with [lo, hi].  FP32: points
// within rounding of the radius may fall either side, where the screening
// estimate is already at its threshold.
__device__ __forceinline__ void tile_line_range(const WLine& ln, float R2, int& lo, int& hi) {
    const float disc = ln.qb * ln.qb - ln.qa * (ln.qc - R2);
    if (!(disc >= 0.f)) {
        lo = 1;
        hi = 0;
        return;
    }
    const float x0 = -ln.qb / ln.qa, h = sqrtf(disc) / ln.qa;
    lo = max(lo, (int)ceilf(x0 - h));
    hi = min(hi, (int)floorf(x0 + h));
}

// Skipping state of a radius-limited tile in an orthorhombic cell, where the
// smallest |G| of a line grows with |n2| inside a plane and the smallest |G|
// of a plane grows with n3: once a line lies wholly outside the radius, so do
// the rest of its direction in that plane (and, for a plane's centre line,
// every later plane), and the walk jumps to the next transition that starts
// from the plane values (OP_NEGSTART, OP_N3, or a chunk's OP_FIRST).
enum { kWalkOn = 0, kSkipPos = 1, kSkipNeg = 2, kSkipRest = 3 };

__device__ __forceinline__ bool line_outside(const WLine& ln, float R2) {
    return !(ln.qb * ln.qb - ln.qa * (ln.qc - R2) >= 0.f);
}

// true: skip this line without advancing the walk state
__device__ __forceinline__ bool skip_line(int& mode, int op) {
    if (mode == kSkipPos && op != OP_NEGSTART && op != OP_N3 && op != OP_FIRST) return true;
    if (mode == kSkipNeg && op != OP_N3 && op != OP_FIRST) return true;
    mode = kWalkOn;
    return false;
}

__device__ __forceinline__ int skip_mode_after(const WLine& ln) {
    return ln.n2 == 0 ? kSkipRest : (ln.n2 > 0 ? kSkipPos : kSkipNeg);
}

// Index within the chunk of the first point visited in direction dir of line
// ln (stored order: n1 = max(lo,0) .. hi, then min(hi,-1) .. lo; the tile
// visits first = max(tile lo, 0) resp. min(tile hi, -1)); the following
// points of the direction have the next indices.
__device__ __forceinline__ int first_index(const WLine& ln, int p0, int dir, int first) {
    const int f = max(ln.lo, 0);
    if (dir == 0) return ln.pt - p0 + (first - f);
    const int n0 = ln.hi >= f ? ln.hi - f + 1 : 0;
    return ln.pt - p0 + n0 + (min(ln.hi, -1) - first);
}

template <int L, bool ORTHO, bool CUT>
__device__ void rho_tile_split(const Tile& tl, const Layout& lay, const float2* __restrict__ Dp_d,
                               const SConst* __restrict__ cst, const SState* __restrict__ init_c,
                               const WLine* __restrict__ lines, const WChunk ch, float4* buf, float4* red,
                               float4* row, float2* Dsm, float4* Xs, int nx, int* spt) {
    constexpr int NT = nterms(L);
    const int tid = threadIdx.x;
    const bool valid = tid < tl.count;
    const long long pi = (long long)tl.first + tid;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long loc = pi - lay.start[L];
    // the record's coefficients live in a thread-private shared-memory slice
    // (read once per line), keeping registers for the per-point recurrences
#pragma unroll
    for (int t = 0; t < NT; ++t)
        Dsm[t * kTile + tid] = valid ? Dp_d[lay.base[L] + (long long)t * cnt + loc] : make_float2(0.f, 0.f);
    const SConst k = valid ? cst[pi] : idle_const();
    const SState* init_p = init_c + (valid ? pi : 0);
    if (ORTHO) build_xtab(valid ? *init_p : idle_state(), k.q1, nx, Xs, tid);
    SState s;
    int slot = 0, par = 0, rbase = 0, mode = kWalkOn;
    for (int li = ch.l0; li < ch.l1; ++li) {
        const WLine ln = lines[li];
        if (ORTHO && CUT) {
            if (mode == kSkipRest) break;
            if (skip_line(mode, ln.op)) continue;
        }
        split_step<ORTHO>(k, ln.op, s, init_p, valid);
        int lo = ln.lo, hi = ln.hi;
        if (CUT) {
            if (ORTHO && line_outside(ln, tl.gcut2)) {
                mode = skip_mode_after(ln);
                continue;
            }
            tile_line_range(ln, tl.gcut2, lo, hi);
        }
        if (lo > hi) continue;
        cdf c[L + 1];
        {
            float pq[L + 1][L + 1];
            powers23f<L>(ln.n2, ln.n3, pq);
#pragma unroll
            for (int i = 0; i <= L; ++i) c[i] = cdf{{0.f, 0.f}, {0.f, 0.f}};
            int t = 0;
#pragma unroll
            for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                for (int i = lam; i >= 0; --i)
#pragma unroll
                    for (int j = lam - i; j >= 0; --j) {
                        const int kk = lam - i - j;
                        const float2 dv = Dsm[t * kTile + tid];
                        const df v = df_mulf_u(df{dv.x, dv.y}, pq[j][kk]);
                        switch (lam & 3) {
                            case 0: c[i].re = df_add_u(c[i].re, v); break;
                            case 1: c[i].im = df_add_u(c[i].im, df_neg(v)); break;
                            case 2: c[i].re = df_add_u(c[i].re, df_neg(v)); break;
                            default: c[i].im = df_add_u(c[i].im, v); break;
                        }
                        ++t;
                    }
        }
        if (ORTHO) {
            // the line value gp(0) goes into the coefficients; X(n1) carries the rest
#pragma unroll
            for (int i = 0; i <= L; ++i) c[i] = cdf_mul_u(s.gpL, c[i]);
        }
        // not unrolled: the walk's instruction footprint (five classes) stays in the instruction cache
#pragma unroll 1
        for (int dir = 0; dir < 2; ++dir) {
            int m0, m1, step;
            cdf gp, R;
            if (dir == 0) {
                if (hi < 0) continue;
                m0 = 0;
                m1 = hi;
                step = 1;
                if (!ORTHO) {
                    gp = s.gpL;
                    R = s.RfL;
                }
            } else {
                if (lo > -1) continue;
                m0 = -1;
                m1 = lo;
                step = -1;
                if (!ORTHO) {
                    gp = cdf_mul_u(s.gpL, s.RbL);
                    R = cdf_scale_u(s.RbL, k.q1);
                }
            }
            if (ORTHO) {
                // no recurrence to carry: visit exactly the line's points of this direction
                m0 = dir == 0 ? max(lo, 0) : min(hi, -1);
                if ((m1 - m0) * step < 0) continue;
            }
            int q = CUT ? first_index(ln, ch.p0, dir, dir == 0 ? max(lo, 0) : min(hi, -1)) : 0;
            float x = (float)m0;
            const float xstep = (float)step;
            for (int m = m0;; m += step, x += xstep) {
                if (ORTHO || (m >= lo && m <= hi)) {
                    const cdf a = poly_at<L>(c, x);
                    cdf xv;
                    if (ORTHO) xv = xtab_at(Xs, m, dir, tid);
                    const cdf z = ORTHO ? cdf_mul_u(xv, a) : cdf_mul_u(gp, a);
                    buf[slot * (kTile + 1) + tid] = make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
                    if (CUT) {
                        if (tid == 0) spt[par * kSBatch + slot] = q;
                        ++q;
                    }
                    if (++slot == kSBatch) {
                        split_flush(buf, red, row, CUT ? spt + par * kSBatch : nullptr, rbase, kSBatch);
                        par ^= 1;  // the next batch's indices go to the other half
                        rbase += kSBatch;
                        slot = 0;
                    }
                }
                if (m == m1) break;
                if (!ORTHO) {
                    gp = cdf_mul_u(gp, R);
                    R = cdf_scale_u(R, k.q1);
                }
            }
        }
    }
    if (slot > 0) split_flush(buf, red, row, CUT ? spt + par * kSBatch : nullptr, rbase, slot);
    __syncthreads();
}

// The structure-factor walk, persistent over the plan's tile schedule.  PART
// 0: tiles of every class; PART 1: classes 0-2 (a 10-term D' slice, sized for
// four blocks per SM); PART 2: classes 3-4.  Where shared memory holds the
// one-kernel walk below three blocks per SM, parts 2 and 1 run as two launches
// in turn, blocks [0, npb_hi) and [npb_hi, npb) of the schedule and the rows.
template <bool ORTHO, bool CUT, int PART>
__global__ void __launch_bounds__(kTile, PART == 1 ? 4 : 3) k_rho_walk_split(
    const Tile* __restrict__ tiles, int b0, Layout lay, const float2* __restrict__ Dp, const SConst* __restrict__ cst,
    const SState* __restrict__ init, long long npairs, const WLine* __restrict__ lines,
    const WChunk* __restrict__ chunks, int npb, double2* __restrict__ rho_part, long long ng_half,
    const int* __restrict__ sched, int nx) {
    extern __shared__ float4 ssm[];
    __shared__ int spt[2 * kSBatch];  // point indices of the current and the previous batch
    const int b = b0 + blockIdx.x, cidx = blockIdx.y, d = blockIdx.z;
    const WChunk ch = chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    float4* buf = ssm;
    float4* red = buf + kSBatch * (kTile + 1);
    float2* Dsm = reinterpret_cast<float2*>(red + kTile);
    float4* Xs = reinterpret_cast<float4*>(Dsm + nterms(PART == 1 ? 2 : 4) * kTile);
    float4* row = Xs + (ORTHO ? nx * kTile : 0);
    for (int i = threadIdx.x; i < npts; i += blockDim.x) row[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const float2* Dp_d = Dp + (long long)d * lay.total;
    const SState* init_c = init + (long long)cidx * npairs;
    // this block's tiles: sched[b] .. sched[b+1] index the list after the npb+1 offsets
    for (int j = sched[b]; j < sched[b + 1]; ++j) {
        const Tile tl = tiles[sched[npb + 1 + j]];
#define FTCJ_RHO_TILE(Lc) \
    rho_tile_split<Lc, ORTHO, CUT>(tl, lay, Dp_d, cst, init_c, lines, ch, buf, red, row, Dsm, Xs, nx, spt)
        if (PART == 1) {
            if (tl.cls == 0) FTCJ_RHO_TILE(0);
            else if (tl.cls == 1) FTCJ_RHO_TILE(1);
            else FTCJ_RHO_TILE(2);
        } else if (PART == 2) {
            if (tl.cls == 3) FTCJ_RHO_TILE(3);
            else FTCJ_RHO_TILE(4);
        } else {
            switch (tl.cls) {
                case 0: FTCJ_RHO_TILE(0); break;
                case 1: FTCJ_RHO_TILE(1); break;
                case 2: FTCJ_RHO_TILE(2); break;
                case 3: FTCJ_RHO_TILE(3); break;
                default: FTCJ_RHO_TILE(4); break;
            }
        }
#undef FTCJ_RHO_TILE
    }
    __syncthreads();
    double2* out = rho_part + ((long long)d * npb + b) * ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const float4 v = row[i];
        out[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

// ---- J -------------------------------------------------------------------

// L: degree of the sums (the record's class, or one more for the nuclear
// gradient's sums); C: the record's class, which places its terms in `lay`.
template <int L, bool ORTHO, bool CUT, int C = L>
__device__ void j_tile_split(const Tile& tl, const Layout& lay, const SConst* __restrict__ cst,
                             const SState* __restrict__ init_c, const WLine* __restrict__ lines, const WChunk ch,
                             const float4* __restrict__ wsm,
                             double* __restrict__ Jp_dc, float2* Jsm, float4* Xs, int nx) {
    constexpr int NT = nterms(L);
    const int tid = threadIdx.x;
    const bool valid = tid < tl.count;
    const long long pi = (long long)tl.first + tid;
    const long long cnt = lay.start[C + 1] - lay.start[C];
    const long long loc = pi - lay.start[C];
    const SConst k = valid ? cst[pi] : idle_const();
    const SState* init_p = init_c + (valid ? pi : 0);
    // the record's J' accumulators live in a thread-private shared-memory slice
    // (updated once per line)
#pragma unroll
    for (int t = 0; t < NT; ++t) Jsm[t * kTile + tid] = make_float2(0.f, 0.f);
    if (ORTHO) build_xtab(valid ? *init_p : idle_state(), k.q1, nx, Xs, tid);
    SState s;
    int mode = kWalkOn;
    for (int li = ch.l0; li < ch.l1; ++li) {
        const WLine ln = lines[li];
        if (ORTHO && CUT) {
            if (mode == kSkipRest) break;
            if (skip_line(mode, ln.op)) continue;
        }
        split_step<ORTHO>(k, ln.op, s, init_p, valid);
        int lo = ln.lo, hi = ln.hi;
        if (CUT) {
            if (ORTHO && line_outside(ln, tl.gcut2)) {
                mode = skip_mode_after(ln);
                continue;
            }
            tile_line_range(ln, tl.gcut2, lo, hi);
        }
        if (lo > hi) continue;
        cdf A[L + 1];
#pragma unroll
        for (int i = 0; i <= L; ++i) A[i] = cdf{{0.f, 0.f}, {0.f, 0.f}};
        int qs = ln.pt - ch.p0;  // without cutoffs the line's points are visited in stored order
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            int m0, m1, step;
            cdf gp, R;
            if (dir == 0) {
                if (hi < 0) continue;
                m0 = 0;
                m1 = hi;
                step = 1;
                if (!ORTHO) {
                    gp = s.gpL;
                    R = s.RfL;
                }
            } else {
                if (lo > -1) continue;
                m0 = -1;
                m1 = lo;
                step = -1;
                if (!ORTHO) {
                    gp = cdf_mul_u(s.gpL, s.RbL);
                    R = cdf_scale_u(s.RbL, k.q1);
                }
            }
            if (ORTHO) {
                // no recurrence to carry: visit exactly the line's points of this direction
                m0 = dir == 0 ? max(lo, 0) : min(hi, -1);
                if ((m1 - m0) * step < 0) continue;
            }
            int q = CUT ? first_index(ln, ch.p0, dir, dir == 0 ? max(lo, 0) : min(hi, -1)) : qs;
            float x = (float)m0;
            const float xstep = (float)step;
            for (int m = m0;; m += step, x += xstep) {
                if (ORTHO || (m >= lo && m <= hi)) {
                    const cdf w = unpack(wsm[q++]);
                    cdf xv;
                    if (ORTHO) xv = xtab_at(Xs, m, dir, tid);
                    const cdf t = ORTHO ? cdf_mul_u(xv, w) : cdf_mul_u(gp, w);
                    A[0] = cdf_add_u(A[0], t);
                    float p = 1.f;
#pragma unroll
                    for (int i = 1; i <= L; ++i) {
                        p *= x;  // n1^i, exact (|n1|^L < 2^24)
                        A[i] = cdf{df_add_u(A[i].re, df_mulf_u(t.re, p)), df_add_u(A[i].im, df_mulf_u(t.im, p))};
                    }
                }
                if (m == m1) break;
                if (!ORTHO) {
                    gp = cdf_mul_u(gp, R);
                    R = cdf_scale_u(R, k.q1);
                }
            }
            qs = q;
        }
        if (ORTHO) {
#pragma unroll
            for (int i = 0; i <= L; ++i) A[i] = cdf_mul_u(s.gpL, A[i]);
        }
        float pq[L + 1][L + 1];
        powers23f<L>(ln.n2, ln.n3, pq);
        int t = 0;
#pragma unroll
        for (int lam = 0; lam <= L; ++lam)
#pragma unroll
            for (int i = lam; i >= 0; --i)
#pragma unroll
                for (int j = lam - i; j >= 0; --j) {
                    const int kk = lam - i - j;
                    df a;
                    switch (lam & 3) {
                        case 0: a = A[i].re; break;
                        case 1: a = A[i].im; break;
                        case 2: a = df_neg(A[i].re); break;
                        default: a = df_neg(A[i].im); break;
                    }
                    const float2 jv = Jsm[t * kTile + tid];
                    const df r = df_add(df{jv.x, jv.y}, df_mulf_u(a, pq[j][kk]));
                    Jsm[t * kTile + tid] = make_float2(r.hi, r.lo);
                    ++t;
                }
    }
    if (valid) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const float2 jv = Jsm[t * kTile + tid];
            Jp_dc[lay.base[C] + (long long)t * cnt + loc] = (double)jv.x + (double)jv.y;
        }
    }
}

// The back-contraction walk.  PART 0: tiles of every class; PART 1: classes
// 0-2 only (a 10-term J' slice, sized for four blocks per SM); PART 2: classes
// 3-4.  Parts 1 and 2 run as two launches side by side where the shared
// memory of the one-kernel walk (a long chunk's W beside a 35-term J' slice)
// would hold it below three blocks per SM.  E = 1: the sums of degree L + 1
// that the nuclear gradient contracts (one more power of G from d/dR_A), into
// the gradient's term layout; the slices grow to 20 resp. 56 terms, and the
// degree-5 part takes the registers of two blocks per SM.
template <bool ORTHO, bool CUT, int PART, int E>
__global__ void __launch_bounds__(kTile, PART == 1 ? 4 : (E ? 2 : 3)) k_j_walk_split(
    const Tile* __restrict__ tiles, int tile0, Layout lay, const SConst* __restrict__ cst,
    const SState* __restrict__ init, long long npairs, const WLine* __restrict__ lines,
    const WChunk* __restrict__ chunks, int nchunks, const double2* __restrict__ W, long long ng_half, int nx,
    int max_chunk_pts, double* __restrict__ Jp) {
    extern __shared__ float4 ssm[];
    const int tix = tile0 + blockIdx.x, cidx = blockIdx.y, d = blockIdx.z;
    const WChunk ch = chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    float4* wsm = ssm;
    float2* Jsm = reinterpret_cast<float2*>(ssm + max_chunk_pts);
    float4* Xs = reinterpret_cast<float4*>(Jsm + nterms((PART == 1 ? 2 : 4) + E) * kTile);
    const double2* Wd = W + (long long)d * ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const double2 v = Wd[i];
        const df re = df_from_double(v.x), im = df_from_double(v.y);
        wsm[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const Tile tl = tiles[tix];
    double* Jp_dc = Jp + ((long long)d * nchunks + cidx) * lay.total;
    const SState* init_c = init + (long long)cidx * npairs;
#define FTCJ_J_TILE(c) j_tile_split<(c) + E, ORTHO, CUT, (c)>(tl, lay, cst, init_c, lines, ch, wsm, Jp_dc, Jsm, Xs, nx)
    if (PART == 1) {
        switch (tl.cls) {
            case 0: FTCJ_J_TILE(0); break;
            case 1: FTCJ_J_TILE(1); break;
            default: FTCJ_J_TILE(2); break;
        }
    } else if (PART == 2) {
        if (tl.cls == 3) FTCJ_J_TILE(3);
        else FTCJ_J_TILE(4);
    } else {
        switch (tl.cls) {
            case 0: FTCJ_J_TILE(0); break;
            case 1: FTCJ_J_TILE(1); break;
            case 2: FTCJ_J_TILE(2); break;
            case 3: FTCJ_J_TILE(3); break;
            default: FTCJ_J_TILE(4); break;
        }
    }
#undef FTCJ_J_TILE
}

Layout make_layout(const ftcj_plan* P) {
    Layout l;
    for (int c = 0; c <= kNclass; ++c) l.start[c] = P->class_start[c];
    for (int c = 0; c < kNclass; ++c) l.base[c] = P->term_base[c];
    l.total = P->total_terms;
    return l;
}

Layout make_grad_layout(const ftcj_plan* P) {
    Layout l;
    for (int c = 0; c <= kNclass; ++c) l.start[c] = P->class_start[c];
    for (int c = 0; c < kNclass; ++c) l.base[c] = P->term_base_g[c];
    l.total = P->total_terms_g;
    return l;
}

// entries of the half X(n1) table, n1 = 0 .. max(|n1_min|, n1_max)
int xtab_entries(const ftcj_plan* P) { return std::max(-P->n1_min, P->n1_max) + 1; }

// orthorhombic cells with a short enough n1 range use the per-record X(n1) table
bool use_xtab(const ftcj_plan* P) { return P->ortho && xtab_entries(P) <= 24; }

size_t xtab_bytes(const ftcj_plan* P) {
    return use_xtab(P) ? sizeof(float4) * (size_t)xtab_entries(P) * kTile : 0;
}

size_t rho_smem(const ftcj_plan* P, int part = 0) {
    return sizeof(float4) * ((size_t)kSBatch * (kTile + 1) + kTile + (size_t)std::max(P->max_chunk_pts, 1)) +
           sizeof(float2) * (size_t)nterms(part == 1 ? 2 : 4) * kTile + xtab_bytes(P);
}

size_t j_smem(const ftcj_plan* P, int part, int e = 0) {
    const int hi = (part == 1 ? 2 : 4) + e;
    return sizeof(float4) * (size_t)std::max(P->max_chunk_pts, 1) + sizeof(float2) * (size_t)nterms(hi) * kTile +
           xtab_bytes(P);
}

// the walk kernels for the plan's shape: X(n1) table or recurrence, with or without per-pair cutoffs
using RhoKernel = decltype(&k_rho_walk_split<true, true, 0>);
using JKernel = decltype(&k_j_walk_split<true, true, 0, 0>);

template <int PART>
RhoKernel rho_kernel_part(const ftcj_plan* P) {
    const bool c = P->d_rec_gcut != nullptr;
    if (use_xtab(P)) return c ? k_rho_walk_split<true, true, PART> : k_rho_walk_split<true, false, PART>;
    return c ? k_rho_walk_split<false, true, PART> : k_rho_walk_split<false, false, PART>;
}

RhoKernel rho_kernel(const ftcj_plan* P, int part = 0) {
    return part == 1 ? rho_kernel_part<1>(P) : (part == 2 ? rho_kernel_part<2>(P) : rho_kernel_part<0>(P));
}

template <int PART, int E>
JKernel j_kernel_part(const ftcj_plan* P) {
    const bool c = P->d_rec_gcut != nullptr;
    if (use_xtab(P)) return c ? k_j_walk_split<true, true, PART, E> : k_j_walk_split<true, false, PART, E>;
    return c ? k_j_walk_split<false, true, PART, E> : k_j_walk_split<false, false, PART, E>;
}

JKernel j_kernel(const ftcj_plan* P, int part) {
    return part == 1 ? j_kernel_part<1, 0>(P) : (part == 2 ? j_kernel_part<2, 0>(P) : j_kernel_part<0, 0>(P));
}

// the gradient's walk always runs as its two class parts (the 56-term slice of
// classes 3-4 would hold a one-kernel walk to few blocks per SM)
JKernel j_grad_kernel(const ftcj_plan* P, int part) {
    return part == 1 ? j_kernel_part<1, 1>(P) : j_kernel_part<2, 1>(P);
}


// ---- one persistent launch over a batch of cells (form 2) -------------------
//
// Work items of every cell of a batch share one queue (a global counter):
// structure-factor items (cell, persistent block b of the cell's LPT
// schedule, chunk, density), the same work one block of the cell's own walk
// launch does, writing that block's rho row, and back-contraction items
// (cell, tile, chunk, density), all structure-factor items first.  The phase
// change is per cell: the CTA that finishes a cell's last structure-factor
// item sums its rows in fixed order, forms W = 2 v conj rho and E_J, and
// raises the cell's ready flag; a CTA holding a back-contraction item of that
// cell waits for the flag (every structure-factor item was taken before any
// back-contraction item, by CTAs that wait on nothing, so the wait ends).  The wait is bounded: past the
// budget the CTA raises the batch's error word and skips the item.  Data
// written inside the launch (rows, W) is read through L2 (ld.global.cg),
// never through the read-only path.

struct BatchCell {
    const Tile* tiles;
    const int* sched;
    int npb, nchunks, nx, ndens;
    Layout lay;
    const float2* Dp;
    const SConst* cst;
    const SState* init;
    long long npairs;
    const WLine* lines;
    const WChunk* chunks;
    double2* rho_part;   // [dens][npb][ng_half]
    const double* vg;
    double2* W;          // [dens][ng_half]
    double* EJ;          // [dens]
    double* Jp;          // [dens][nchunks][total]
    long long ng_half;
};

// one tile of one class, out of line: each class's walk gets its own register allocation
template <int Lc, bool ORTHO>
__device__ __noinline__ void batch_rho_tile(const Tile tl, const BatchCell* C, const float2* __restrict__ Dp_d,
                                            const SState* __restrict__ init_c, const WChunk ch, float4* buf,
                                            float4* red, float4* row, float2* Dsm, float4* Xs, int* spt) {
    rho_tile_split<Lc, ORTHO, false>(tl, C->lay, Dp_d, C->cst, init_c, C->lines, ch, buf, red, row, Dsm, Xs, C->nx,
                                     spt);
}

template <int Lc, bool ORTHO>
__device__ __noinline__ void batch_j_tile(const Tile tl, const BatchCell* C, const SState* __restrict__ init_c,
                                          const WChunk ch, const float4* wsm, double* Jp_dc, float2* Jsm,
                                          float4* Xs) {
    j_tile_split<Lc, ORTHO, false, Lc>(tl, C->lay, C->cst, init_c, C->lines, ch, wsm, Jp_dc, Jsm, Xs, C->nx);
}

template <bool ORTHO>
__device__ __forceinline__ void batch_rho_item(const BatchCell& C, int b, int cidx, int d, float4* ssm, int* spt) {
    const WChunk ch = C.chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    float4* buf = ssm;
    float4* red = buf + kSBatch * (kTile + 1);
    float2* Dsm = reinterpret_cast<float2*>(red + kTile);
    float4* Xs = reinterpret_cast<float4*>(Dsm + nterms(4) * kTile);
    float4* row = Xs + (ORTHO ? C.nx * kTile : 0);
    for (int i = threadIdx.x; i < npts; i += blockDim.x) row[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const float2* Dp_d = C.Dp + (long long)d * C.lay.total;
    const SState* init_c = C.init + (long long)cidx * C.npairs;
    for (int j = C.sched[b]; j < C.sched[b + 1]; ++j) {
        const Tile tl = C.tiles[C.sched[C.npb + 1 + j]];
#define FTCJ_BRHO(Lc) batch_rho_tile<Lc, ORTHO>(tl, &C, Dp_d, init_c, ch, buf, red, row, Dsm, Xs, spt)
        switch (tl.cls) {
            case 0: FTCJ_BRHO(0); break;
            case 1: FTCJ_BRHO(1); break;
            case 2: FTCJ_BRHO(2); break;
            case 3: FTCJ_BRHO(3); break;
            default: FTCJ_BRHO(4); break;
        }
#undef FTCJ_BRHO
    }
    __syncthreads();
    double2* out = C.rho_part + ((long long)d * C.npb + b) * C.ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const float4 v = row[i];
        out[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
    __syncthreads();
}

template <bool ORTHO>
__device__ __forceinline__ void batch_j_item(const BatchCell& C, int tix, int cidx, int d, float4* ssm) {
    const WChunk ch = C.chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    float4* wsm = ssm;
    float2* Jsm = reinterpret_cast<float2*>(ssm + npts);
    float4* Xs = reinterpret_cast<float4*>(Jsm + nterms(4) * kTile);
    const double2* Wd = C.W + (long long)d * C.ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const double2 v = __ldcg(Wd + i);  // written in this launch: through L2
        const df re = df_from_double(v.x), im = df_from_double(v.y);
        wsm[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const Tile tl = C.tiles[tix];
    double* Jp_dc = C.Jp + ((long long)d * C.nchunks + cidx) * C.lay.total;
    const SState* init_c = C.init + (long long)cidx * C.npairs;
#define FTCJ_BJ(c) batch_j_tile<(c), ORTHO>(tl, &C, init_c, ch, wsm, Jp_dc, Jsm, Xs)
    switch (tl.cls) {
        case 0: FTCJ_BJ(0); break;
        case 1: FTCJ_BJ(1); break;
        case 2: FTCJ_BJ(2); break;
        case 3: FTCJ_BJ(3); break;
        default: FTCJ_BJ(4); break;
    }
#undef FTCJ_BJ
    __syncthreads();
}

// rho = the cell's rows summed in fixed order, W = 2 v conj rho, E_J = sum v |rho|^2 (one CTA)
__device__ __noinline__ void batch_reduce_cell(const BatchCell& C, double* se) {
    for (int d = 0; d < C.ndens; ++d) {
        double e = 0.0;
        for (long long p = threadIdx.x; p < C.ng_half; p += blockDim.x) {
            const double2* src = C.rho_part + (long long)d * C.npb * C.ng_half + p;
            double rr = 0.0, ri = 0.0;
            for (int q = 0; q < C.npb; ++q) {
                const double2 u = __ldcg(src + (long long)q * C.ng_half);
                rr += u.x;
                ri += u.y;
            }
            const double v = C.vg[p];
            C.W[(long long)d * C.ng_half + p] = make_double2(2.0 * v * rr, -2.0 * v * ri);
            e += v * (rr * rr + ri * ri);
        }
        se[threadIdx.x] = e;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) C.EJ[d] = se[0];
        __syncthreads();
    }
}

// CTAs per SM the batch kernel is compiled for (registers: 3 -> 168, 2 -> 255)
#ifndef FTCJ_BATCH_MINB
#define FTCJ_BATCH_MINB 3
#endif

template <bool ORTHO>
__global__ void __launch_bounds__(kTile, FTCJ_BATCH_MINB) k_batch_walks(const BatchCell* __restrict__ cells,
                                                           const int4* __restrict__ items, int nitems,
                                                           int* counter, int* remaining, int* ready, int* err,
                                                           long long spin) {
    extern __shared__ float4 ssm[];
    __shared__ int spt[2 * kSBatch];
    __shared__ double se[kTile];
    __shared__ int s_item, s_go;
    __shared__ BatchCell sc;  // the item's cell, read from shared memory rather than held in registers
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int4 in = items[it];
        if (threadIdx.x < (int)(sizeof(BatchCell) / 8))
            reinterpret_cast<long long*>(&sc)[threadIdx.x] = reinterpret_cast<const long long*>(cells + in.x)[threadIdx.x];
        __syncthreads();
        const BatchCell& C = sc;
        const int d = in.w & 0xffff;
        if ((in.w >> 16) == 0) {
            batch_rho_item<ORTHO>(C, in.y, in.z, d, ssm, spt);
            // the last structure-factor item of the cell does its reduction
            __threadfence();
            if (threadIdx.x == 0) s_go = atomicSub(remaining + in.x, 1) == 1;
            __syncthreads();
            if (s_go) {
                __threadfence();
                batch_reduce_cell(C, se);
                __threadfence();
                if (threadIdx.x == 0) atomicExch(ready + in.x, 1);
            }
            __syncthreads();
        } else {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                int ok = 1;
                while (atomicAdd(ready + in.x, 0) == 0) {
                    if (*(volatile int*)err || clock64() - t0 > spin) {
                        atomicOr(err, 1);
                        ok = 0;
                        break;
                    }
                }
                __threadfence();
                s_go = ok;
            }
            __syncthreads();
            if (s_go) batch_j_item<ORTHO>(C, in.y, in.z, d, ssm);
            __syncthreads();
        }
    }
}

// shared memory of the batch kernel for one cell: the larger of its two walks' (one-kernel shapes)
size_t batch_cell_smem(const ftcj_plan* P) { return std::max(rho_smem(P, 0), j_smem(P, 0)); }

}  // namespace

int split_xtab_entries(const ftcj_plan* P) { return use_xtab(P) ? xtab_entries(P) : 0; }

size_t split_rho_smem(const ftcj_plan* P, int part) { return rho_smem(P, part); }

int setup_split(ftcj_plan* P) {
    const size_t nch = P->chunks.size();
    const size_t np = (size_t)std::max<int64_t>(P->npairs, 1);
    FTCJ_CUDA(cudaMalloc(&P->d_split_init, sizeof(SState) * np * std::max<size_t>(nch, 1)));
    P->device_bytes += sizeof(SState) * np * std::max<size_t>(nch, 1);
    FTCJ_CUDA(cudaMalloc(&P->d_split_const, sizeof(SConst) * np));
    P->device_bytes += sizeof(SConst) * np;
    if (P->npairs > 0 && nch > 0) {
        dim3 g((unsigned)((P->npairs + 127) / 128), (unsigned)nch);
        k_split_setup<<<g, 128>>>(P->d_walk, P->npairs, P->d_lines, P->d_chunks, (int)nch,
                                  reinterpret_cast<SState*>(P->d_split_init),
                                  reinterpret_cast<SConst*>(P->d_split_const), P->cc);
        FTCJ_CUDA(cudaGetLastError());
    }
    int rc = FTCJ_OK;
    for (int part = 0; part < 3 && !rc; ++part) rc = allow_dynamic_smem((const void*)rho_kernel(P, part), rho_smem(P, part));
    if (rc) return rc;
    for (int part = 0; part < 3 && !rc; ++part) rc = allow_dynamic_smem((const void*)j_kernel(P, part), j_smem(P, part));
    if (rc) return rc;
    for (int part = 1; part < 3 && !rc; ++part)
        rc = allow_dynamic_smem((const void*)j_grad_kernel(P, part), j_smem(P, part, 1));
    if (rc) return rc;
    // split the walk by class only where shared memory holds the one-kernel walk below three blocks per SM
    int dev = 0, per_sm = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    int nhi = 0;  // tiles are ordered by decreasing class: classes 3-4 lead
    while (nhi < (int)P->tiles.size() && P->tiles[nhi].cls >= 3) ++nhi;
    const bool smem_bound = (size_t)per_sm / (j_smem(P, 0) + 1024) < 3;
    P->ntiles_hi = smem_bound && nhi > 0 && nhi < (int)P->tiles.size() ? nhi : 0;
    const bool rho_smem_bound = (size_t)per_sm / (rho_smem(P, 0) + 1024) < 3;
    P->rho_hi_tiles = rho_smem_bound && nhi > 0 && nhi < (int)P->tiles.size() ? nhi : 0;
    if (!P->aux) {
        // the heavy classes' stream has the highest priority, so that their blocks take SM slots first
        int lo_prio = 0, hi_prio = 0;
        FTCJ_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        FTCJ_CUDA(cudaStreamCreateWithPriority(&P->aux, cudaStreamNonBlocking, hi_prio));
        FTCJ_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
        FTCJ_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    }
    return FTCJ_OK;
}

int rho_walk_split_blocks_per_sm(ftcj_plan* P, int part, int* out) {
    int n = 0;
    FTCJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rho_kernel(P, part), kTile, rho_smem(P, part)));
    *out = n > 0 ? n : 1;
    return FTCJ_OK;
}

int launch_rho_walk_split(ftcj_plan* P, int ndens, cudaStream_t s) {
    if (P->ng_half == 0 || P->tiles.empty()) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_rho_part, 0, sizeof(double2) * (size_t)ndens * P->npb * P->ng_half, s));
        return FTCJ_OK;
    }
    const int nx = use_xtab(P) ? xtab_entries(P) : 0;
    auto go = [&](int part, int b0, int nblk) {
        rho_kernel(P, part)<<<dim3((unsigned)nblk, (unsigned)P->chunks.size(), ndens), kTile, rho_smem(P, part), s>>>(
            P->d_tiles, b0, make_layout(P), reinterpret_cast<const float2*>(P->d_Dp),
            reinterpret_cast<const SConst*>(P->d_split_const), reinterpret_cast<const SState*>(P->d_split_init),
            P->npairs, P->d_lines, P->d_chunks, P->npb, reinterpret_cast<double2*>(P->d_rho_part), P->ng_half,
            P->d_sched, nx);
    };
    if (P->rho_hi_tiles > 0) {
        go(2, 0, P->npb_hi);
        FTCJ_CUDA(cudaGetLastError());
        go(1, P->npb_hi, P->npb - P->npb_hi);
    } else {
        go(0, 0, P->npb);
    }
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int split_j_launches(const ftcj_plan* P) { return P->ntiles_hi > 0 ? 2 : 1; }

int launch_j_walk_split(ftcj_plan* P, int ndens, const double* W, cudaStream_t s) {
    const int nch = (int)P->chunks.size();
    if (P->tiles.empty()) return FTCJ_OK;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_Jp, 0, sizeof(double) * (size_t)ndens * std::max(nch, 1) * P->total_terms, s));
        return FTCJ_OK;
    }
    const int nx = use_xtab(P) ? xtab_entries(P) : 0;
    const int nhi = P->ntiles_hi, nlo = (int)P->tiles.size() - nhi;
    auto go = [&](int part, int tile0, int ntiles, cudaStream_t st) {
        j_kernel(P, part)<<<dim3((unsigned)ntiles, nch, ndens), kTile, j_smem(P, part), st>>>(
            P->d_tiles, tile0, make_layout(P), reinterpret_cast<const SConst*>(P->d_split_const),
            reinterpret_cast<const SState*>(P->d_split_init), P->npairs, P->d_lines, P->d_chunks, nch,
            reinterpret_cast<const double2*>(W), P->ng_half, nx, P->max_chunk_pts, P->d_Jp);
    };
    if (nhi > 0 && nlo > 0) {
        // classes 3-4 on the plan's second stream, beside classes 0-2 on the caller's (event fork and join)
        FTCJ_CUDA(cudaEventRecord(P->ev_fork, s));
        FTCJ_CUDA(cudaStreamWaitEvent(P->aux, P->ev_fork, 0));
        go(2, 0, nhi, P->aux);
        FTCJ_CUDA(cudaGetLastError());
        go(1, nhi, nlo, s);
        FTCJ_CUDA(cudaGetLastError());
        FTCJ_CUDA(cudaEventRecord(P->ev_join, P->aux));
        FTCJ_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));
    } else {
        go(0, 0, (int)P->tiles.size(), s);
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}

bool split_grad_walk_exact(const ftcj_plan* P) { return P->n_abs_max <= kSplitGradNmax; }

// The degree-(L+1) back-contraction of the nuclear gradient in double-float,
// into d_Jg (FP64, the gradient's term layout).  Both class parts run side by
// side (classes 3-4 on the plan's second stream), each over its own tiles.
int launch_j_walk_grad_split(ftcj_plan* P, int ndens, const double* W, cudaStream_t s) {
    const int nch = (int)P->chunks.size();
    if (P->tiles.empty()) return FTCJ_OK;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_Jg, 0, sizeof(double) * (size_t)ndens * std::max(nch, 1) * P->total_terms_g, s));
        return FTCJ_OK;
    }
    const int nx = use_xtab(P) ? xtab_entries(P) : 0;
    int nhi = 0;  // tiles are ordered by decreasing class: classes 3-4 lead
    while (nhi < (int)P->tiles.size() && P->tiles[nhi].cls >= 3) ++nhi;
    const int nlo = (int)P->tiles.size() - nhi;
    auto go = [&](int part, int tile0, int ntiles, cudaStream_t st) {
        j_grad_kernel(P, part)<<<dim3((unsigned)ntiles, nch, ndens), kTile, j_smem(P, part, 1), st>>>(
            P->d_tiles, tile0, make_grad_layout(P), reinterpret_cast<const SConst*>(P->d_split_const),
            reinterpret_cast<const SState*>(P->d_split_init), P->npairs, P->d_lines, P->d_chunks, nch,
            reinterpret_cast<const double2*>(W), P->ng_half, nx, P->max_chunk_pts, P->d_Jg);
    };
    if (nhi > 0 && nlo > 0) {
        FTCJ_CUDA(cudaEventRecord(P->ev_fork, s));
        FTCJ_CUDA(cudaStreamWaitEvent(P->aux, P->ev_fork, 0));
        go(2, 0, nhi, P->aux);
        FTCJ_CUDA(cudaGetLastError());
        go(1, nhi, nlo, s);
        FTCJ_CUDA(cudaGetLastError());
        FTCJ_CUDA(cudaEventRecord(P->ev_join, P->aux));
        FTCJ_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));
    } else {
        go(nhi > 0 ? 2 : 1, 0, (int)P->tiles.size(), s);
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}


// ---- the batch kernel's host side -----------------------------------------

struct BatchWalks {
    BatchCell* d_cells = nullptr;
    int4* d_items = nullptr;
    int* d_remaining0 = nullptr;  // structure-factor items per cell
    int* d_state = nullptr;       // queue counter, error word, [ncell] remaining, [ncell] ready
    int ncell = 0, nrho = 0, nitems = 0, grid = 0;
    bool ortho = false;
    size_t smem = 0;
};

void batch_walks_destroy(BatchWalks* bw) {
    if (!bw) return;
    void* ptrs[] = {bw->d_cells, bw->d_items, bw->d_remaining0, bw->d_state};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete bw;
}

int batch_walks_create(const std::vector<ftcj_plan*>& plans, BatchWalks** out) {
    *out = nullptr;
    const int n = (int)plans.size();
    std::vector<BatchCell> cells(n);
    struct It {
        int4 v;
        double cost, key;
    };
    std::vector<It> rho, jit;
    std::vector<int> rem(n, 0);
    size_t smem = 0;
    const bool ortho = n > 0 && use_xtab(plans[0]);
    for (int c = 0; c < n; ++c) {
        const ftcj_plan* P = plans[c];
        if (use_xtab(P) != ortho)
            return fail(FTCJ_EUNSUPPORTED, "a persistent batch takes cells that all walk with the X(n1) table "
                                           "(orthorhombic) or all without it");
        if (P->precision != FTCJ_PREC_SPLIT || P->d_rec_gcut || P->tc)
            return fail(FTCJ_EUNSUPPORTED, "the persistent batch runs the double-float walks over whole spheres "
                                           "(split precision, no per-pair cutoffs, walk contraction)");
        BatchCell& C = cells[c];
        C.tiles = P->d_tiles;
        C.sched = P->d_sched;
        C.npb = P->npb;
        C.nchunks = (int)P->chunks.size();
        C.nx = use_xtab(P) ? xtab_entries(P) : 0;
        C.ndens = P->max_dens;
        C.lay = make_layout(P);
        C.Dp = reinterpret_cast<const float2*>(P->d_Dp);
        C.cst = reinterpret_cast<const SConst*>(P->d_split_const);
        C.init = reinterpret_cast<const SState*>(P->d_split_init);
        C.npairs = P->npairs;
        C.lines = P->d_lines;
        C.chunks = P->d_chunks;
        C.rho_part = reinterpret_cast<double2*>(P->d_rho_part);
        C.vg = P->d_vg;
        C.W = reinterpret_cast<double2*>(P->d_W);
        C.EJ = P->d_EJ_stage;
        C.Jp = P->d_Jp;
        C.ng_half = P->ng_half;
        smem = std::max(smem, batch_cell_smem(P));
        if (P->ng_half == 0 || P->tiles.empty()) continue;  // no work: W and J' stay zero (below)
        // per-tile cost, the walks' constants (38L + 100 per point)
        auto tcost = [&](int t) { return (double)P->tiles[t].count * (38.0 * P->tiles[t].cls + 100.0); };
        for (int b = 0; b < P->npb; ++b) {
            double bc = 0.0;
            for (int j = P->rho_sched[b]; j < P->rho_sched[b + 1]; ++j) bc += tcost(P->rho_sched[P->npb + 1 + j]);
            for (int ch = 0; ch < C.nchunks; ++ch)
                for (int d = 0; d < C.ndens; ++d) {
                    rho.push_back({make_int4(c, b, ch, d), bc * (P->chunks[ch].p1 - P->chunks[ch].p0), 0.0});
                    ++rem[c];
                }
        }
        for (int t = 0; t < (int)P->tiles.size(); ++t)
            for (int ch = 0; ch < C.nchunks; ++ch)
                for (int d = 0; d < C.ndens; ++d)
                    jit.push_back({make_int4(c, t, ch, d), tcost(t) * (P->chunks[ch].p1 - P->chunks[ch].p0), 0.0});
    }
    // The queue: every structure-factor item first, largest first (the grid stays busy to the end of
    // that phase); then the back-contraction items, by the queue position of their cell's last
    // structure-factor item (the order in which the cells become ready), largest first within a cell.
    // Every structure-factor item precedes every back-contraction item, and items are taken in queue
    // order by CTAs that wait on nothing else, so a waiting item's cell is being finished.
    std::stable_sort(rho.begin(), rho.end(), [](const It& a, const It& b) { return a.cost > b.cost; });
    std::vector<double> last(n, 0.0);
    for (size_t i = 0; i < rho.size(); ++i) last[rho[i].v.x] = (double)i;
    for (It& x : jit) x.key = last[x.v.x];
    std::stable_sort(jit.begin(), jit.end(), [](const It& a, const It& b) {
        return a.key != b.key ? a.key < b.key : a.cost > b.cost;
    });
    std::vector<int4> items;
    for (const It& x : rho) items.push_back(x.v);
    for (const It& x : jit) items.push_back(make_int4(x.v.x, x.v.y, x.v.z, x.v.w | (1 << 16)));
    BatchWalks* bw = new (std::nothrow) BatchWalks();
    if (!bw) return fail(FTCJ_ENOMEM, "host allocation failed");
    bw->ncell = n;
    bw->nrho = (int)rho.size();
    bw->nitems = (int)items.size();
    bw->smem = smem;
    bw->ortho = ortho;
    const void* kern = ortho ? (const void*)k_batch_walks<true> : (const void*)k_batch_walks<false>;
    cudaError_t e = cudaMalloc(&bw->d_cells, sizeof(BatchCell) * std::max(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&bw->d_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&bw->d_remaining0, sizeof(int) * std::max(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&bw->d_state, sizeof(int) * (2 + 2 * (size_t)std::max(n, 1)));
    if (e == cudaSuccess) e = cudaMemcpy(bw->d_cells, cells.data(), sizeof(BatchCell) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(bw->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bw->d_remaining0, rem.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    int rc = e == cudaSuccess ? FTCJ_OK : cuda_fail(e, "batch work queue");
    if (!rc) rc = allow_dynamic_smem(kern, smem);
    int per_sm = 0;
    if (!rc) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTile, smem);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch kernel occupancy");
        else if (per_sm < 1) rc = fail(FTCJ_EUNSUPPORTED, "the batch's walks do not fit one SM");
    }
    if (rc) {
        batch_walks_destroy(bw);
        return rc;
    }
    bw->grid = std::max(1, std::min(bw->nitems, per_sm * plans[0]->num_sms));
    *out = bw;
    return FTCJ_OK;
}

int batch_walks_launch(BatchWalks* bw, const std::vector<ftcj_plan*>& plans, long long spin, cudaStream_t s) {
    const int n = bw->ncell;
    FTCJ_CUDA(cudaMemsetAsync(bw->d_state, 0, sizeof(int) * (2 + 2 * (size_t)n), s));
    FTCJ_CUDA(cudaMemcpyAsync(bw->d_state + 2, bw->d_remaining0, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    // cells without work: their potential, energy and J' are zero
    for (ftcj_plan* P : plans)
        if (P->ng_half == 0 || P->tiles.empty()) {
            FTCJ_CUDA(cudaMemsetAsync(P->d_EJ_stage, 0, sizeof(double) * P->max_dens, s));
            FTCJ_CUDA(cudaMemsetAsync(P->d_Jp, 0,
                                      sizeof(double) * (size_t)P->max_dens * std::max<size_t>(P->chunks.size(), 1) *
                                          P->total_terms,
                                      s));
        }
    if (bw->nitems == 0) return FTCJ_OK;
    auto kern = bw->ortho ? k_batch_walks<true> : k_batch_walks<false>;
    kern<<<(unsigned)bw->grid, kTile, bw->smem, s>>>(bw->d_cells, bw->d_items, bw->nitems, bw->d_state,
                                                     bw->d_state + 2, bw->d_state + 2 + n, bw->d_state + 1, spin);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int batch_walks_error(BatchWalks* bw, int* word, cudaStream_t s) {
    FTCJ_CUDA(cudaMemcpyAsync(word, bw->d_state + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTCJ_CUDA(cudaStreamSynchronize(s));
    return FTCJ_OK;
}

int batch_walks_launches(const BatchWalks* bw) { return bw->nitems ? 1 : 0; }

}  // namespace ftcj
