// Steps a4, a5 and a6: the structure-factor pass rho(G) (Alg. 1), the
// potential W(G) = 2 v(G) conj rho(G) with E_J, and the back-contraction
// J'_ijk (Alg. S1), in FP64.
//
// Layout of the work: one thread per pair record, 128 records of one class
// L = l_a + l_b per block, all threads walking the same G points in lock step
// (the per-G data is a warp-uniform broadcast).  The half sphere is walked as
// lines along b_1 at fixed (n2, n3), each from n1 = 0 outwards, lines of a
// plane from n2 = 0 outwards, planes n3 = 0, 1, ...  Along that walk every
// pair factor is advanced by multiplications only (the per-axis intermediates
// of Eqs. "intermediate in relative coordinate" and "non-separable
// exponential term"):
//   g(n) = exp(-|G|^2/4p): its ratio to the previous point is itself a
//          geometric sequence (ratio multipliers q_i, x_ij, y_ij);
//   ph(n) = exp(-2 pi i n.f): multiplied by exp(-2 pi i f_j) per step.
// Transcendentals are evaluated only where a chunk of lines starts.
//
// rho: each point's 128 pair contributions are summed in shared memory in
// batches of 32 points (transpose + column sums), accumulated into a per-block
// row, and the rows of all blocks are added in a fixed order by k_rho_reduce
// (deterministic, no atomics).
// J: the thread accumulates sum over a line of t(n1) n1^i, then folds the
// line into J'_ijk with n2^j n3^k; nothing is shared between threads.
#include <cmath>

#include "ftcj_internal.h"

namespace ftcj {
namespace {


struct Layout {
    long long start[kNclass + 1];
    long long base[kNclass];
    long long total;
};

constexpr int kPw = kLpair + 2;  // powers n1^0..n1^(L+1) in the J walks' table

struct WalkState {
    double gC, TF, RF0, RB0, rF0, rB0, phCr, phCi;  // plane centre (0, 0, n3)
    double gL, Rd, rF, rB, phLr, phLi;              // line centre (0, n2, n3)
};

__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double& cr, double& ci) {
    double r = ar * br - ai * bi;
    double i = ar * bi + ai * br;
    cr = r;
    ci = i;
}

__device__ __forceinline__ void phase(double th, double& re, double& im) {
    th -= rint(th);
    double s, c;
    sincospi(2.0 * th, &s, &c);
    re = c;
    im = -s;  // exp(-2 pi i th)
}

// state at line (n2, n3) and its plane centre, from closed forms
__device__ __noinline__ void state_first(const PairWalk& w, const double* M6, int n2, int n3, WalkState& s) {
    const double c = w.c;
    const double M11 = M6[0], M22 = M6[1], M33 = M6[2], M12 = M6[3], M13 = M6[4], M23 = M6[5];
    const double a2 = (double)n2, a3 = (double)n3;
    s.gC = exp(-c * M33 * a3 * a3);
    s.TF = exp(-c * M33 * (2.0 * a3 + 1.0));
    s.RF0 = exp(-c * (M22 + 2.0 * M23 * a3));
    s.RB0 = exp(-c * (M22 - 2.0 * M23 * a3));
    s.rF0 = exp(-c * (M11 + 2.0 * M13 * a3));
    s.rB0 = exp(-c * (M11 - 2.0 * M13 * a3));
    phase(a3 * w.f3, s.phCr, s.phCi);
    double Q = M22 * a2 * a2 + 2.0 * M23 * a2 * a3 + M33 * a3 * a3;
    s.gL = exp(-c * Q);
    s.Rd = (n2 >= 0) ? exp(-c * (M22 * (2.0 * a2 + 1.0) + 2.0 * M23 * a3))
                     : exp(-c * (M22 * (1.0 - 2.0 * a2) - 2.0 * M23 * a3));
    double beta = M12 * a2 + M13 * a3;
    s.rF = exp(-c * (M11 + 2.0 * beta));
    s.rB = exp(-c * (M11 - 2.0 * beta));
    phase(a2 * w.f2 + a3 * w.f3, s.phLr, s.phLi);
}

__device__ __forceinline__ void state_step(const PairWalk& w, const double* M6, int op, int n2, int n3,
                                           WalkState& s) {
    switch (op) {
        case OP_FIRST:
            state_first(w, M6, n2, n3, s);
            break;
        case OP_N2F:
            s.gL *= s.Rd;
            s.Rd *= w.q2;
            s.rF *= w.x12;
            s.rB *= w.y12;
            cmul(s.phLr, s.phLi, w.e2r, w.e2i, s.phLr, s.phLi);
            break;
        case OP_NEGSTART:
            s.gL = s.gC * s.RB0;
            s.Rd = s.RB0 * w.q2;
            s.rF = s.rF0 * w.y12;
            s.rB = s.rB0 * w.x12;
            cmul(s.phCr, s.phCi, w.e2r, -w.e2i, s.phLr, s.phLi);
            break;
        case OP_N2B:
            s.gL *= s.Rd;
            s.Rd *= w.q2;
            s.rF *= w.y12;
            s.rB *= w.x12;
            cmul(s.phLr, s.phLi, w.e2r, -w.e2i, s.phLr, s.phLi);
            break;
        default:  // OP_N3
            s.gC *= s.TF;
            s.TF *= w.q3;
            s.RF0 *= w.x23;
            s.RB0 *= w.y23;
            s.rF0 *= w.x13;
            s.rB0 *= w.y13;
            cmul(s.phCr, s.phCi, w.e3r, w.e3i, s.phCr, s.phCi);
            s.gL = s.gC;
            s.Rd = s.RF0;
            s.rF = s.rF0;
            s.rB = s.rB0;
            s.phLr = s.phCr;
            s.phLi = s.phCi;
            break;
    }
}

__device__ __forceinline__ PairWalk idle_walk() {
    PairWalk w;
    w.c = 0.0;
    w.f1 = w.f2 = w.f3 = 0.0;
    w.q1 = w.q2 = w.q3 = 1.0;
    w.x12 = w.y12 = w.x13 = w.y13 = w.x23 = w.y23 = 1.0;
    w.e1r = w.e2r = w.e3r = 1.0;
    w.e1i = w.e2i = w.e3i = 0.0;
    w.pad = 0.0;
    return w;
}

// products n2^j n3^k for j + k <= L
template <int L>
__device__ __forceinline__ void powers23(int n2, int n3, double pq[L + 1][L + 1]) {
    double p2[L + 1], p3[L + 1];
    p2[0] = 1.0;
    p3[0] = 1.0;
#pragma unroll
    for (int j = 1; j <= L; ++j) {
        p2[j] = p2[j - 1] * (double)n2;
        p3[j] = p3[j - 1] * (double)n3;
    }
#pragma unroll
    for (int j = 0; j <= L; ++j)
#pragma unroll
        for (int k = 0; k + j <= L; ++k) pq[j][k] = p2[j] * p3[k];
}

// ---- rho -----------------------------------------------------------------

// Per-pair cutoffs: the tile's part of a line under its G radius, the n1
// with qa n1^2 + 2 qb n1 + qc < R2, intersected with [lo, hi] (the same FP32
// test as the split form's walks).
__device__ __forceinline__ void cut_range(const WLine& ln, float R2, int& lo, int& hi) {
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

// index within the chunk of the point n1 = m of line ln (stored order:
// n1 = max(lo, 0) .. hi, then min(hi, -1) .. lo)
__device__ __forceinline__ int point_index(const WLine& ln, int p0, int m) {
    const int f = max(ln.lo, 0);
    if (m >= 0) return ln.pt - p0 + (m - f);
    const int n0 = ln.hi >= f ? ln.hi - f + 1 : 0;
    return ln.pt - p0 + n0 + (min(ln.hi, -1) - m);
}

// idx: the batch's point indices in the row (per-pair cutoffs), else consecutive from rbase
__device__ __forceinline__ void rho_flush(double2* buf, double2* red, double2* row, const int* idx, int rbase,
                                          int nvalid) {
    __syncthreads();
    const int tid = threadIdx.x, j = tid & 31, wv = tid >> 5;
    if (j < nvalid) {
        double sr = 0.0, si = 0.0;
        const double2* b = buf + j * (kTile + 1) + wv * 32;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            double2 v = b[k];
            sr += v.x;
            si += v.y;
        }
        red[wv * 32 + j] = make_double2(sr, si);
    }
    __syncthreads();
    if (tid < nvalid) {
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int q = 0; q < kTile / 32; ++q) {
            double2 v = red[q * 32 + tid];
            sr += v.x;
            si += v.y;
        }
        const int r = idx ? idx[tid] : rbase + tid;
        const double2 o = row[r];
        row[r] = make_double2(o.x + sr, o.y + si);
    }
}

template <int L, bool CUT>
__device__ void rho_tile(const double* M6, const Tile& tl, const Layout& lay, const double* __restrict__ Dp_d,
                         const PairWalk* __restrict__ walk, const WLine* __restrict__ lines, const WChunk ch,
                         double2* buf, double2* red, double2* row, int* spt) {
    constexpr int NT = nterms(L);
    const int tid = threadIdx.x;
    const bool valid = tid < tl.count;
    const long long pi = (long long)tl.first + tid;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long loc = pi - lay.start[L];
    double D[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) D[t] = valid ? Dp_d[lay.base[L] + (long long)t * cnt + loc] : 0.0;
    const PairWalk w = valid ? walk[pi] : idle_walk();
    WalkState s;
    int slot = 0, par = 0;
    int rbase = 0;
    for (int li = ch.l0; li < ch.l1; ++li) {
        const WLine ln = lines[li];
        state_step(w, M6, ln.op, ln.n2, ln.n3, s);
        int lo = ln.lo, hi = ln.hi;
        if (CUT) cut_range(ln, tl.gcut2, lo, hi);
        if (lo > hi) continue;
        // c_i = sum_{j,k} (-i)^{i+j+k} D'_ijk n2^j n3^k
        double cr[L + 1], ci[L + 1];
        {
            double pq[L + 1][L + 1];
            powers23<L>(ln.n2, ln.n3, pq);
#pragma unroll
            for (int i = 0; i <= L; ++i) {
                cr[i] = 0.0;
                ci[i] = 0.0;
            }
            int t = 0;
#pragma unroll
            for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                for (int i = lam; i >= 0; --i)
#pragma unroll
                    for (int j = lam - i; j >= 0; --j) {
                        const int k = lam - i - j;
                        const double v = D[t] * pq[j][k];
                        switch (lam & 3) {
                            case 0: cr[i] += v; break;
                            case 1: ci[i] -= v; break;
                            case 2: cr[i] -= v; break;
                            default: ci[i] += v; break;
                        }
                        ++t;
                    }
        }
        // forward half of the line: n1 = 0, 1, ..., hi
        if (hi >= 0) {
            double g = s.gL, r = s.rF, pr = s.phLr, pim = s.phLi, x = 0.0;
            for (int m = 0; m <= hi; ++m) {
                if (m >= lo) {
                    double ar = cr[L], ai = ci[L];
#pragma unroll
                    for (int i = L - 1; i >= 0; --i) {
                        ar = fma(ar, x, cr[i]);
                        ai = fma(ai, x, ci[i]);
                    }
                    const double gr = g * pr, gi = g * pim;
                    buf[slot * (kTile + 1) + tid] = make_double2(gr * ar - gi * ai, gr * ai + gi * ar);
                    if (CUT && tid == 0) spt[par * kBatch + slot] = point_index(ln, ch.p0, m);
                    if (++slot == kBatch) {
                        rho_flush(buf, red, row, CUT ? spt + par * kBatch : nullptr, rbase, kBatch);
                        rbase += kBatch;
                        slot = 0;
                        par ^= 1;
                    }
                }
                g *= r;
                r *= w.q1;
                cmul(pr, pim, w.e1r, w.e1i, pr, pim);
                x += 1.0;
            }
        }
        // backward half: n1 = -1, -2, ..., lo
        if (lo <= -1) {
            double g = s.gL * s.rB, r = s.rB * w.q1, pr, pim, x = -1.0;
            cmul(s.phLr, s.phLi, w.e1r, -w.e1i, pr, pim);
            for (int m = -1; m >= lo; --m) {
                if (m <= hi) {
                    double ar = cr[L], ai = ci[L];
#pragma unroll
                    for (int i = L - 1; i >= 0; --i) {
                        ar = fma(ar, x, cr[i]);
                        ai = fma(ai, x, ci[i]);
                    }
                    const double gr = g * pr, gi = g * pim;
                    buf[slot * (kTile + 1) + tid] = make_double2(gr * ar - gi * ai, gr * ai + gi * ar);
                    if (CUT && tid == 0) spt[par * kBatch + slot] = point_index(ln, ch.p0, m);
                    if (++slot == kBatch) {
                        rho_flush(buf, red, row, CUT ? spt + par * kBatch : nullptr, rbase, kBatch);
                        rbase += kBatch;
                        slot = 0;
                        par ^= 1;
                    }
                }
                g *= r;
                r *= w.q1;
                cmul(pr, pim, w.e1r, -w.e1i, pr, pim);
                x -= 1.0;
            }
        }
    }
    if (slot > 0) rho_flush(buf, red, row, CUT ? spt + par * kBatch : nullptr, rbase, slot);
    __syncthreads();
}

template <bool CUT>
__global__ void __launch_bounds__(kTile) k_rho_walk(const Tile* __restrict__ tiles, int ntiles, Layout lay,
                                                    const double* __restrict__ Dp, const PairWalk* __restrict__ walk,
                                                    const WLine* __restrict__ lines,
                                                    const WChunk* __restrict__ chunks, int npb,
                                                    double2* __restrict__ rho_part, long long ng_half, CellConst cc,
                                                    const int* __restrict__ sched) {
    extern __shared__ double2 smem[];
    __shared__ int spt[2 * kBatch];  // point indices of the current and the previous batch (per-pair cutoffs)
    const int b = blockIdx.x, cidx = blockIdx.y, d = blockIdx.z;
    const WChunk ch = chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    double2* buf = smem;
    double2* red = buf + kBatch * (kTile + 1);
    double2* row = red + kTile;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) row[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const double* Dp_d = Dp + (long long)d * lay.total;
    // this block's tiles: sched[b] .. sched[b+1] index the list after the npb+1 offsets
    for (int j = sched[b]; j < sched[b + 1]; ++j) {
        const Tile tl = tiles[sched[npb + 1 + j]];
        switch (tl.cls) {
            case 0: rho_tile<0, CUT>(cc.M6, tl, lay, Dp_d, walk, lines, ch, buf, red, row, spt); break;
            case 1: rho_tile<1, CUT>(cc.M6, tl, lay, Dp_d, walk, lines, ch, buf, red, row, spt); break;
            case 2: rho_tile<2, CUT>(cc.M6, tl, lay, Dp_d, walk, lines, ch, buf, red, row, spt); break;
            case 3: rho_tile<3, CUT>(cc.M6, tl, lay, Dp_d, walk, lines, ch, buf, red, row, spt); break;
            default: rho_tile<4, CUT>(cc.M6, tl, lay, Dp_d, walk, lines, ch, buf, red, row, spt); break;
        }
    }
    __syncthreads();
    double2* out = rho_part + ((long long)d * npb + b) * ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) out[i] = row[i];
}

// rho = sum over the block rows; optional W = 2 v conj(rho) and per-block
// partial sums of v |rho|^2.  A block takes kRedPoints consecutive points and
// 256 / kRedPoints row groups (group g sums rows g, g + groups, ... with two
// accumulators); the groups are added in a fixed tree, so the result does not
// depend on scheduling.  With nparts = 1 and part = rho this is the potential
// step on a given rho.
__global__ void __launch_bounds__(256) k_rho_reduce(const double2* __restrict__ part, int nparts,
                                                    long long ng_half, const double* __restrict__ vg,
                                                    double2* __restrict__ rho_out, double2* __restrict__ W_out,
                                                    double* __restrict__ Epart, int nEblocks) {
    constexpr int kGroups = 256 / kRedPoints;
    __shared__ double2 sred[kGroups][kRedPoints];
    __shared__ double se[kRedPoints];
    const int d = blockIdx.y;
    const int pt = threadIdx.x % kRedPoints, g = threadIdx.x / kRedPoints;
    const long long p = (long long)blockIdx.x * kRedPoints + pt;
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    if (p < ng_half) {
        const double2* src = part + (long long)d * nparts * ng_half + p;
        int q = g;
        for (; q + kGroups < nparts; q += 2 * kGroups) {
            const double2 u = src[(long long)q * ng_half];
            const double2 v = src[(long long)(q + kGroups) * ng_half];
            ar += u.x;
            ai += u.y;
            br += v.x;
            bi += v.y;
        }
        if (q < nparts) {
            const double2 u = src[(long long)q * ng_half];
            ar += u.x;
            ai += u.y;
        }
    }
    sred[g][pt] = make_double2(ar + br, ai + bi);
    __syncthreads();
    for (int o = kGroups / 2; o > 0; o >>= 1) {
        if (g < o) {
            const double2 a = sred[g][pt], b = sred[g + o][pt];
            sred[g][pt] = make_double2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
    }
    if (g == 0) {
        double e = 0.0;
        if (p < ng_half) {
            const double2 r = sred[0][pt];
            if (rho_out) rho_out[(long long)d * ng_half + p] = r;
            if (W_out) {
                const double v = vg[p];
                W_out[(long long)d * ng_half + p] = make_double2(2.0 * v * r.x, -2.0 * v * r.y);
                e = v * (r.x * r.x + r.y * r.y);
            }
        }
        se[pt] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0 && Epart) {
        double t = 0.0;
        for (int k = 0; k < kRedPoints; ++k) t += se[k];
        Epart[(long long)d * nEblocks + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_energy_final(const double* __restrict__ Epart, int nEblocks,
                                                      double* __restrict__ EJ) {
    __shared__ double se[256];
    const int d = blockIdx.x;
    double e = 0.0;
    for (int i = threadIdx.x; i < nEblocks; i += blockDim.x) e += Epart[(long long)d * nEblocks + i];
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) EJ[d] = se[0];
}

// ---- J -------------------------------------------------------------------

// L is the polynomial degree walked (the record's class, or class + 1 for the
// gradient); the term layout is that of the record's class tl.cls.
template <int L, bool CUT>
__device__ void j_tile(const double* M6, const Tile& tl, const Layout& lay, const PairWalk* __restrict__ walk,
                       const WLine* __restrict__ lines, const WChunk ch, const double2* __restrict__ wsm,
                       const double* __restrict__ pw, int n1min, double* __restrict__ Jp_dc) {
    constexpr int NT = nterms(L);
    const int tid = threadIdx.x;
    const bool valid = tid < tl.count;
    const long long pi = (long long)tl.first + tid;
    const long long cnt = lay.start[tl.cls + 1] - lay.start[tl.cls];
    const long long loc = pi - lay.start[tl.cls];
    const PairWalk w = valid ? walk[pi] : idle_walk();
    double J[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) J[t] = 0.0;
    WalkState s;
    for (int li = ch.l0; li < ch.l1; ++li) {
        const WLine ln = lines[li];
        state_step(w, M6, ln.op, ln.n2, ln.n3, s);
        int lo = ln.lo, hi = ln.hi;
        if (CUT) cut_range(ln, tl.gcut2, lo, hi);
        if (lo > hi) continue;
        double Ar[L + 1], Ai[L + 1];
#pragma unroll
        for (int i = 0; i <= L; ++i) {
            Ar[i] = 0.0;
            Ai[i] = 0.0;
        }
        int q = point_index(ln, ch.p0, max(lo, 0));
        if (hi >= 0) {
            double g = s.gL, r = s.rF, pr = s.phLr, pim = s.phLi;
            for (int m = 0; m <= hi; ++m) {
                if (m >= lo) {
                    const double2 W = wsm[q++];
                    const double gr = g * pr, gi = g * pim;
                    const double tr = gr * W.x - gi * W.y, ti = gr * W.y + gi * W.x;
                    Ar[0] += tr;
                    Ai[0] += ti;
                    const double* pwm = pw + (m - n1min) * kPw;
#pragma unroll
                    for (int i = 1; i <= L; ++i) {
                        Ar[i] = fma(tr, pwm[i], Ar[i]);
                        Ai[i] = fma(ti, pwm[i], Ai[i]);
                    }
                }
                g *= r;
                r *= w.q1;
                cmul(pr, pim, w.e1r, w.e1i, pr, pim);
            }
        }
        if (lo <= -1) {
            q = point_index(ln, ch.p0, min(hi, -1));
            double g = s.gL * s.rB, r = s.rB * w.q1, pr, pim;
            cmul(s.phLr, s.phLi, w.e1r, -w.e1i, pr, pim);
            for (int m = -1; m >= lo; --m) {
                if (m <= hi) {
                    const double2 W = wsm[q++];
                    const double gr = g * pr, gi = g * pim;
                    const double tr = gr * W.x - gi * W.y, ti = gr * W.y + gi * W.x;
                    Ar[0] += tr;
                    Ai[0] += ti;
                    const double* pwm = pw + (m - n1min) * kPw;
#pragma unroll
                    for (int i = 1; i <= L; ++i) {
                        Ar[i] = fma(tr, pwm[i], Ar[i]);
                        Ai[i] = fma(ti, pwm[i], Ai[i]);
                    }
                }
                g *= r;
                r *= w.q1;
                cmul(pr, pim, w.e1r, -w.e1i, pr, pim);
            }
        }
        // J'_ijk += Re[(-i)^{i+j+k} A_i] n2^j n3^k
        double pq[L + 1][L + 1];
        powers23<L>(ln.n2, ln.n3, pq);
        int t = 0;
#pragma unroll
        for (int lam = 0; lam <= L; ++lam)
#pragma unroll
            for (int i = lam; i >= 0; --i)
#pragma unroll
                for (int j = lam - i; j >= 0; --j) {
                    const int k = lam - i - j;
                    double a;
                    switch (lam & 3) {
                        case 0: a = Ar[i]; break;
                        case 1: a = Ai[i]; break;
                        case 2: a = -Ar[i]; break;
                        default: a = -Ai[i]; break;
                    }
                    J[t] = fma(a, pq[j][k], J[t]);
                    ++t;
                }
    }
    if (valid) {
#pragma unroll
        for (int t = 0; t < NT; ++t) Jp_dc[lay.base[tl.cls] + (long long)t * cnt + loc] = J[t];
    }
}

// EXTRA = 0: the back-contraction of degree L; EXTRA = 1: degree L + 1, the
// sums the nuclear gradient needs (one more power of G from d/dR).
template <int EXTRA, bool CUT>
__global__ void __launch_bounds__(kTile) k_j_walk(const Tile* __restrict__ tiles, Layout lay,
                                                  const PairWalk* __restrict__ walk, const WLine* __restrict__ lines,
                                                  const WChunk* __restrict__ chunks, int nchunks,
                                                  const double2* __restrict__ W, long long ng_half, int n1min,
                                                  int n1cnt, int max_chunk_pts, double* __restrict__ Jp, CellConst cc) {
    extern __shared__ double2 smem[];
    const int tix = blockIdx.x, cidx = blockIdx.y, d = blockIdx.z;
    const WChunk ch = chunks[cidx];
    const int npts = ch.p1 - ch.p0;
    double2* wsm = smem;
    double* pw = reinterpret_cast<double*>(smem + max_chunk_pts);
    const double2* Wd = W + (long long)d * ng_half + ch.p0;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) wsm[i] = Wd[i];
    for (int i = threadIdx.x; i < n1cnt * kPw; i += blockDim.x) {
        const double x = (double)(n1min + i / kPw);
        double v = 1.0;
        for (int e = 0; e < i % kPw; ++e) v *= x;
        pw[i] = v;
    }
    __syncthreads();
    const Tile tl = tiles[tix];
    double* Jp_dc = Jp + ((long long)d * nchunks + cidx) * lay.total;
    switch (tl.cls + EXTRA) {
        case 0: j_tile<0, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc); break;
        case 1: j_tile<1, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc); break;
        case 2: j_tile<2, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc); break;
        case 3: j_tile<3, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc); break;
        case 4: j_tile<4, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc); break;
        default:
            if (EXTRA) j_tile<5, CUT>(cc.M6, tl, lay, walk, lines, ch, wsm, pw, n1min, Jp_dc);
            break;
    }
}

__global__ void k_vg(const int* __restrict__ gvec, long long n, double* __restrict__ vg, CellConst cc) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double n1 = gvec[3 * p], n2 = gvec[3 * p + 1], n3 = gvec[3 * p + 2];
    const double g2 = cc.M6[0] * n1 * n1 + cc.M6[1] * n2 * n2 + cc.M6[2] * n3 * n3 +
                      2.0 * (cc.M6[3] * n1 * n2 + cc.M6[4] * n1 * n3 + cc.M6[5] * n2 * n3);
    vg[p] = cc.vpar[0] * exp(-g2 * cc.vpar[1]) / g2;
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

size_t rho_smem_bytes(const ftcj_plan* P) {
    return sizeof(double2) * ((size_t)kBatch * (kTile + 1) + kTile + (size_t)std::max(P->max_chunk_pts, 1));
}

size_t j_smem_bytes(const ftcj_plan* P) {
    int n1cnt = P->n1_max - P->n1_min + 1;
    return sizeof(double2) * (size_t)std::max(P->max_chunk_pts, 1) + sizeof(double) * kPw * (size_t)n1cnt;
}

}  // namespace

int upload_walk_tables(ftcj_plan* P) {
    int rc = allow_dynamic_smem((const void*)k_rho_walk<false>, rho_smem_bytes(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_rho_walk<true>, rho_smem_bytes(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_j_walk<0, false>, j_smem_bytes(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_j_walk<0, true>, j_smem_bytes(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_j_walk<1, false>, j_smem_bytes(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_j_walk<1, true>, j_smem_bytes(P));
    return rc;
}

int rho_walk_blocks_per_sm(ftcj_plan* P, int* out) {
    int n = 0;
    FTCJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rho_walk<false>, kTile, rho_smem_bytes(P)));
    *out = n > 0 ? n : 1;
    return FTCJ_OK;
}

int launch_vg(ftcj_plan* P) {
    if (P->ng_half == 0) return FTCJ_OK;
    k_vg<<<(unsigned)((P->ng_half + 255) / 256), 256>>>(P->d_gvec, P->ng_half, P->d_vg, P->cc);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_rho_walk(ftcj_plan* P, int ndens, cudaStream_t s) {
    if (P->ng_half == 0 || P->tiles.empty()) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_rho_part, 0, sizeof(double2) * (size_t)ndens * P->npb * P->ng_half, s));
        return FTCJ_OK;
    }
    dim3 g(P->npb, (unsigned)P->chunks.size(), ndens);
    auto kern = P->d_rec_gcut ? k_rho_walk<true> : k_rho_walk<false>;
    kern<<<g, kTile, rho_smem_bytes(P), s>>>(P->d_tiles, (int)P->tiles.size(), make_layout(P), P->d_Dp,
                                                   P->d_walk, P->d_lines, P->d_chunks, P->npb,
                                                   reinterpret_cast<double2*>(P->d_rho_part), P->ng_half, P->cc,
                                                   P->d_sched);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_rho_reduce(ftcj_plan* P, int ndens, double* rho_out, double* W_out, double* EJ_out, const double* rho_in,
                      cudaStream_t s) {
    const double2* part = rho_in ? reinterpret_cast<const double2*>(rho_in)
                                 : reinterpret_cast<const double2*>(P->d_rho_part);
    int nparts = rho_in ? 1 : P->rho_rows;
    if (P->ng_half > 0) {
        dim3 g(P->nEblocks, ndens);
        k_rho_reduce<<<g, 256, 0, s>>>(part, nparts, P->ng_half, P->d_vg, reinterpret_cast<double2*>(rho_out),
                                       reinterpret_cast<double2*>(W_out), EJ_out ? P->d_Epart : nullptr,
                                       P->nEblocks);
        FTCJ_CUDA(cudaGetLastError());
    }
    if (EJ_out) {
        if (P->ng_half == 0) {
            FTCJ_CUDA(cudaMemsetAsync(EJ_out, 0, sizeof(double) * ndens, s));
        } else {
            k_energy_final<<<ndens, 256, 0, s>>>(P->d_Epart, P->nEblocks, EJ_out);
            FTCJ_CUDA(cudaGetLastError());
        }
    }
    return FTCJ_OK;
}

int launch_j_walk(ftcj_plan* P, int ndens, const double* W, cudaStream_t s) {
    int nch = (int)P->chunks.size();
    if (P->tiles.empty()) return FTCJ_OK;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_Jp, 0, sizeof(double) * (size_t)ndens * std::max(nch, 1) * P->total_terms, s));
        return FTCJ_OK;
    }
    dim3 g((unsigned)P->tiles.size(), nch, ndens);
    int n1cnt = P->n1_max - P->n1_min + 1;
    auto kern = P->d_rec_gcut ? k_j_walk<0, true> : k_j_walk<0, false>;
    kern<<<g, kTile, j_smem_bytes(P), s>>>(P->d_tiles, make_layout(P), P->d_walk, P->d_lines, P->d_chunks, nch,
                                               reinterpret_cast<const double2*>(W), P->ng_half, P->n1_min, n1cnt,
                                               P->max_chunk_pts, P->d_Jp, P->cc);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

}  // namespace ftcj

namespace ftcj {

// the degree-(L+1) back-contraction sums of the nuclear gradient, into d_Jg
int launch_j_walk_grad(ftcj_plan* P, int ndens, const double* W, cudaStream_t s) {
    int nch = (int)P->chunks.size();
    if (P->tiles.empty()) return FTCJ_OK;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(P->d_Jg, 0, sizeof(double) * (size_t)ndens * std::max(nch, 1) * P->total_terms_g, s));
        return FTCJ_OK;
    }
    dim3 g((unsigned)P->tiles.size(), nch, ndens);
    int n1cnt = P->n1_max - P->n1_min + 1;
    auto kern = P->d_rec_gcut ? k_j_walk<1, true> : k_j_walk<1, false>;
    kern<<<g, kTile, j_smem_bytes(P), s>>>(P->d_tiles, make_grad_layout(P), P->d_walk, P->d_lines,
                                                  P->d_chunks, nch, reinterpret_cast<const double2*>(W), P->ng_half,
                                                  P->n1_min, n1cnt, P->max_chunk_pts, P->d_Jg, P->cc);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

}  // namespace ftcj
