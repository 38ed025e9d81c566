// Steps a2 and a8: the k <-> BvK transforms (Eqs. "FT for D" and "FT of J")
//   D^{0n} = Re (1/Nk) sum_k exp(-i k.R_n) D^k,
//   J^k    = sum_n exp(+i k.R_n) J^{0n},
// done as one small DFT per mesh axis (separable over the Gamma-centred
// mesh), each stage a coalesced pass over the [dens][cell][nao*nao] array
// with the AO-pair index fastest.
#include <algorithm>
#include <vector>

#include "df.cuh"
#include "ftcj_internal.h"

namespace ftcj {
namespace {

constexpr int kTw = 16;  // twiddle table edge (k-mesh dimensions <= 16)

__global__ void k_twiddles(double2* __restrict__ tw, int n0, int n1, int n2) {
    int a = blockIdx.x;
    int N = a == 0 ? n0 : (a == 1 ? n1 : n2);
    int m = threadIdx.y, n = threadIdx.x;
    double2 v = make_double2(0.0, 0.0);
    if (m < N && n < N) {
        int r = (m * n) % N;
        double s, c;
        sincospi(2.0 * (double)r / (double)N, &s, &c);
        v = make_double2(c, -s);  // exp(-2 pi i m n / N)
    }
    tw[(a * kTw + m) * kTw + n] = v;
}

// One axis of the separable transform.  Element idx = ((d*nk + cell)*E + e);
// out(.., n_axis, ..) = scale * sum_m w(m, n_axis) in(.., m, ..), with
// w = tw or conj(tw).  IN_REAL / OUT_REAL select double or interleaved complex.
template <bool IN_REAL, bool OUT_REAL>
__global__ void k_dft_axis(const double* __restrict__ in, double* __restrict__ out, long long total, long long E,
                           int N1, int N2, int N3, int axis, const double2* __restrict__ tw, int conj_tw,
                           double scale) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int nk = N1 * N2 * N3;
    long long e = idx % E;
    long long t = idx / E;
    int cell = (int)(t % nk);
    long long d = t / nk;
    int i3 = cell % N3, i2 = (cell / N3) % N2, i1 = cell / (N2 * N3);
    int na, Na;
    long long stride;
    if (axis == 0) {
        na = i1;
        Na = N1;
        stride = (long long)N2 * N3 * E;
    } else if (axis == 1) {
        na = i2;
        Na = N2;
        stride = (long long)N3 * E;
    } else {
        na = i3;
        Na = N3;
        stride = E;
    }
    long long base = (d * nk + cell) * E + e - (long long)na * stride;
    const double2* w = tw + axis * kTw * kTw;
    double sr = 0.0, si = 0.0;
    for (int m = 0; m < Na; ++m) {
        double2 c = w[m * kTw + na];
        double wr = c.x, wi = conj_tw ? -c.y : c.y;
        long long q = base + (long long)m * stride;
        if (IN_REAL) {
            double x = in[q];
            sr = fma(wr, x, sr);
            si = fma(wi, x, si);
        } else {
            double2 x = reinterpret_cast<const double2*>(in)[q];
            sr = fma(wr, x.x, fma(-wi, x.y, sr));
            si = fma(wr, x.y, fma(wi, x.x, si));
        }
    }
    if (OUT_REAL) {
        out[idx] = scale * sr;
    } else {
        reinterpret_cast<double2*>(out)[idx] = make_double2(scale * sr, scale * si);
    }
}

__global__ void k_complex_to_real(const double2* __restrict__ in, double* __restrict__ out, long long n, double s) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * in[i].x;
}

__global__ void k_real_to_complex(const double* __restrict__ in, double2* __restrict__ out, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i], 0.0);
}

__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// max |Im D^{0n}| and max |Re D^{0n}_{mu nu} - Re D^{0,-n}_{nu mu}| over a complex fold
__global__ void k_check(const double2* __restrict__ D, long long ndens, int N1, int N2, int N3, int nao,
                        double* __restrict__ out) {
    long long nn = (long long)nao * nao;
    int nk = N1 * N2 * N3;
    long long total = ndens * nk * nn;
    double mi = 0.0, ma = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long e = i % nn;
        long long t = i / nn;
        int cell = (int)(t % nk);
        long long d = t / nk;
        int mu = (int)(e / nao), nu = (int)(e % nao);
        int i3 = cell % N3, i2 = (cell / N3) % N2, i1 = cell / (N2 * N3);
        int mcell = (((N1 - i1) % N1) * N2 + ((N2 - i2) % N2)) * N3 + ((N3 - i3) % N3);
        double2 a = D[i];
        double2 b = D[(d * nk + mcell) * nn + (long long)nu * nao + mu];
        mi = fmax(mi, fabs(a.y));
        ma = fmax(ma, fabs(a.x - b.x));
    }
    atomic_max_nonneg(out, mi);
    atomic_max_nonneg(out + 1, ma);
}

inline unsigned nblocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// ---- fused transform: every axis in one pass over HBM -------------------
// Each thread owns one AO-pair element of one density and keeps its whole
// column over the mesh (nk complex values) in a thread-private slice of
// shared memory (stride kFusedT, so a warp's accesses hit distinct banks).
// The mesh axes are transformed in place: length 2 and 4 by butterflies
// (only additions; the twiddles are +-1, +-i), other lengths by a direct sum
// with the twiddle table.
constexpr int kFusedT = 32;
constexpr int kFusedMaxNk = 256;

__device__ __forceinline__ void dft_line(double2* col, int base, int stride, int Na, const double2* __restrict__ w,
                                         bool inverse) {
    if (Na == 2) {
        double2 x0 = col[base * kFusedT], x1 = col[(base + stride) * kFusedT];
        col[base * kFusedT] = make_double2(x0.x + x1.x, x0.y + x1.y);
        col[(base + stride) * kFusedT] = make_double2(x0.x - x1.x, x0.y - x1.y);
        return;
    }
    if (Na == 4) {
        double2 x0 = col[base * kFusedT], x1 = col[(base + stride) * kFusedT];
        double2 x2 = col[(base + 2 * stride) * kFusedT], x3 = col[(base + 3 * stride) * kFusedT];
        double2 a = make_double2(x0.x + x2.x, x0.y + x2.y), b = make_double2(x0.x - x2.x, x0.y - x2.y);
        double2 c = make_double2(x1.x + x3.x, x1.y + x3.y), d = make_double2(x1.x - x3.x, x1.y - x3.y);
        // forward (exp(-2 pi i mn/4)): y1 = b - i d, y3 = b + i d; inverse swaps them
        double2 bmid = make_double2(b.x + d.y, b.y - d.x);  // b - i d
        double2 bpid = make_double2(b.x - d.y, b.y + d.x);  // b + i d
        col[base * kFusedT] = make_double2(a.x + c.x, a.y + c.y);
        col[(base + 2 * stride) * kFusedT] = make_double2(a.x - c.x, a.y - c.y);
        col[(base + stride) * kFusedT] = inverse ? bpid : bmid;
        col[(base + 3 * stride) * kFusedT] = inverse ? bmid : bpid;
        return;
    }
    double2 x[kTw];
    for (int m = 0; m < Na; ++m) x[m] = col[(base + m * stride) * kFusedT];
    for (int n = 0; n < Na; ++n) {
        double sr = 0.0, si = 0.0;
        for (int m = 0; m < Na; ++m) {
            double2 c = w[m * kTw + n];
            double wi = inverse ? -c.y : c.y;
            sr = fma(c.x, x[m].x, fma(-wi, x[m].y, sr));
            si = fma(c.x, x[m].y, fma(wi, x[m].x, si));
        }
        col[(base + n * stride) * kFusedT] = make_double2(sr, si);
    }
}

__device__ void dft_mesh(double2* col, int N1, int N2, int N3, const double2* __restrict__ tw, bool inverse) {
    // axis 2 (stride 1), axis 1 (stride N3), axis 0 (stride N2*N3)
    if (N3 > 1)
        for (int o = 0; o < N1 * N2; ++o) dft_line(col, o * N3, 1, N3, tw + 2 * kTw * kTw, inverse);
    if (N2 > 1)
        for (int i1 = 0; i1 < N1; ++i1)
            for (int i3 = 0; i3 < N3; ++i3) dft_line(col, i1 * N2 * N3 + i3, N3, N2, tw + kTw * kTw, inverse);
    if (N1 > 1)
        for (int o = 0; o < N2 * N3; ++o) dft_line(col, o, N2 * N3, N1, tw, inverse);
}

// D^{0n} = Re (1/nk) sum_k exp(-i k.R_n) D^k for one (density, element) per thread
__global__ void __launch_bounds__(kFusedT) k_fold_fused(const double2* __restrict__ Dk, double* __restrict__ D0n,
                                                        long long E, int N1, int N2, int N3,
                                                        const double2* __restrict__ tw) {
    extern __shared__ double2 fsm[];
    const int nk = N1 * N2 * N3;
    const long long e = (long long)blockIdx.x * kFusedT + threadIdx.x;
    const long long d = blockIdx.y;
    double2* col = fsm + threadIdx.x;
    if (e < E) {
        const double2* src = Dk + d * nk * E + e;
        for (int k = 0; k < nk; ++k) col[k * kFusedT] = src[(long long)k * E];
        dft_mesh(col, N1, N2, N3, tw, false);
        const double s = 1.0 / nk;
        double* dst = D0n + d * nk * E + e;
        for (int n = 0; n < nk; ++n) dst[(long long)n * E] = s * col[n * kFusedT].x;
    }
}

// J^k = sum_n exp(+i k.R_n) J^{0n} for one (density, element) per thread
__global__ void __launch_bounds__(kFusedT) k_unfold_fused(const double* __restrict__ J0n, double2* __restrict__ Jk,
                                                          long long E, int N1, int N2, int N3,
                                                          const double2* __restrict__ tw) {
    extern __shared__ double2 fsm[];
    const int nk = N1 * N2 * N3;
    const long long e = (long long)blockIdx.x * kFusedT + threadIdx.x;
    const long long d = blockIdx.y;
    double2* col = fsm + threadIdx.x;
    if (e < E) {
        const double* src = J0n + d * nk * E + e;
        for (int n = 0; n < nk; ++n) col[n * kFusedT] = make_double2(src[(long long)n * E], 0.0);
        dft_mesh(col, N1, N2, N3, tw, true);
        double2* dst = Jk + d * nk * E + e;
        for (int k = 0; k < nk; ++k) dst[(long long)k * E] = col[k * kFusedT];
    }
}

// ---- split-precision register transform ----------------------------------


// The transform's sums are at most 9 additions deep (three axes of length 3 or
// 4), so they run without renormalisation (df.cuh "_u" forms); the outputs are
// rebuilt as exact double sums of both parts.
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf_add_u(a, b); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{df_add_u(a.re, df_neg(b.re)), df_add_u(a.im, df_neg(b.im))}; }

// -i v (forward twiddle of a length-4 axis) and +i v (inverse)
__device__ __forceinline__ cdf mul_mi(cdf v) { return cdf{v.im, df_neg(v.re)}; }
__device__ __forceinline__ cdf mul_pi(cdf v) { return cdf{df_neg(v.im), v.re}; }

// sqrt(3)/2 as a double-float (hi = the nearest float, lo = the nearest float to the rest)
__device__ __forceinline__ df sqrt3_half() { return df{__uint_as_float(1063105495u), __uint_as_float(847611083u)}; }

__device__ __forceinline__ cdf halve(cdf v) {
    return cdf{{0.5f * v.re.hi, 0.5f * v.re.lo}, {0.5f * v.im.hi, 0.5f * v.im.lo}};  // exact
}

// Length-3 DFT from t1 = x1 + x2, t2 = x1 - x2: y0 = x0 + t1 and
// y1, y2 = x0 - t1/2 -+ i (sqrt3/2) t2 (forward; the inverse swaps the signs).
template <bool INV>
__device__ __forceinline__ void dft3(cdf x0, cdf x1, cdf x2, cdf& y0, cdf& y1, cdf& y2) {
    const cdf t1 = cadd(x1, x2), t2 = csub(x1, x2);
    const df c = sqrt3_half();
    const cdf is = mul_pi(cdf{df_mul_u(t2.re, c), df_mul_u(t2.im, c)});  // +i (sqrt3/2) t2
    const cdf m1 = csub(x0, halve(t1));
    y0 = cadd(x0, t1);
    y1 = INV ? cadd(m1, is) : csub(m1, is);
    y2 = INV ? csub(m1, is) : cadd(m1, is);
}

// in-register DFT of v[base + m*stride], m < N (N = 1, 2, 3, 4), in natural order
template <int N, bool INV>
__device__ __forceinline__ void dft_reg(cdf* v, int base, int stride) {
    if (N == 2) {
        const cdf x0 = v[base], x1 = v[base + stride];
        v[base] = cadd(x0, x1);
        v[base + stride] = csub(x0, x1);
    } else if (N == 3) {
        dft3<INV>(v[base], v[base + stride], v[base + 2 * stride], v[base], v[base + stride], v[base + 2 * stride]);
    } else if (N == 4) {
        const cdf x0 = v[base], x1 = v[base + stride], x2 = v[base + 2 * stride], x3 = v[base + 3 * stride];
        const cdf a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = csub(x1, x3);
        const cdf wd = INV ? mul_pi(d) : mul_mi(d);  // y1 = b + w d, y3 = b - w d
        v[base] = cadd(a, c);
        v[base + 2 * stride] = csub(a, c);
        v[base + stride] = cadd(b, wd);
        v[base + 3 * stride] = csub(b, wd);
    }
}

__device__ __forceinline__ cdf shfl_xor_cdf(cdf v, int mask) {
    return cdf{{__shfl_xor_sync(0xffffffffu, v.re.hi, mask), __shfl_xor_sync(0xffffffffu, v.re.lo, mask)},
               {__shfl_xor_sync(0xffffffffu, v.im.hi, mask), __shfl_xor_sync(0xffffffffu, v.im.lo, mask)}};
}

__device__ __forceinline__ cdf shfl_cdf(cdf v, int src) {
    return cdf{{__shfl_sync(0xffffffffu, v.re.hi, src), __shfl_sync(0xffffffffu, v.re.lo, src)},
               {__shfl_sync(0xffffffffu, v.im.hi, src), __shfl_sync(0xffffffffu, v.im.lo, src)}};
}

// Axis-1 DFT across the N1 lanes of a column group (lane j of the group holds
// x_j); returns the output of index out_index(j).  N1 = 2, 3: y_j.  N1 = 4:
// two radix-2 exchanges; lane j ends with y of the bit-reversed index.  G3
// (N1 = 3) is a template flag so that the other kernels carry no code for it.
template <bool INV, bool G3>
__device__ __forceinline__ cdf dft_lanes(cdf x, int j, int N1) {
    if (G3) {  // N1 == 3
        const int g0 = (int)(threadIdx.x & 31) - j;  // lane of x_0
        cdf y[3];
        dft3<INV>(shfl_cdf(x, g0), shfl_cdf(x, g0 + 1), shfl_cdf(x, g0 + 2), y[0], y[1], y[2]);
        return j == 0 ? y[0] : (j == 1 ? y[1] : y[2]);
    }
    if (N1 == 2) {
        const cdf o = shfl_xor_cdf(x, 1);
        return j == 0 ? cadd(x, o) : csub(o, x);
    }
    if (N1 == 4) {
        // lanes 0,1: a_j = x_j + x_{j+2}; lanes 2,3: b_{j-2} = x_{j-2} - x_j
        cdf o = shfl_xor_cdf(x, 2);
        const cdf t = j < 2 ? cadd(x, o) : csub(o, x);
        // y0 = a0 + a1, y2 = a0 - a1, y1 = b0 + w b1, y3 = b0 - w b1
        o = shfl_xor_cdf(t, 1);
        switch (j) {
            case 0: return cadd(t, o);
            case 1: return csub(o, t);
            case 2: return cadd(t, INV ? mul_pi(o) : mul_mi(o));
            default: return csub(o, INV ? mul_pi(t) : mul_mi(t));
        }
    }
    return x;
}

__device__ __forceinline__ int out_index(int j, int N1) { return N1 == 4 ? ((j & 1) << 1) | (j >> 1) : j; }

constexpr int kRegBlock = 128;

// Lanes of a warp form 32 / N1 groups of N1 (lanes 30, 31 idle when N1 = 3);
// group g of warp w of block b owns column (b * 4 + w) * (32 / N1) + g.
struct LaneGroup {
    long long col;
    int j;
    bool live;
};

__device__ __forceinline__ LaneGroup lane_group(int N1) {
    const int lane = threadIdx.x & 31, cpw = 32 / N1;
    const int g = lane / N1;
    LaneGroup r;
    r.j = lane - g * N1;
    r.live = g < cpw;
    r.col = ((long long)blockIdx.x * (kRegBlock / 32) + (threadIdx.x >> 5)) * cpw + g;
    return r;
}

inline unsigned reg_blocks(long long ncol, int N1) { return nblocks(ncol, (kRegBlock / 32) * (32 / N1)); }

// Split-form transforms for meshes whose axes are 1, 2, 3 or 4 long (the
// twiddles are +-1, +-i and -1/2 +- i sqrt3/2), in complex double-float on
// the FP32 pipe.  N1 lanes share one AO-pair column of one density; lane j
// holds the i1 = j plane of N2 x N3 values in registers, transforms it along
// axes 3 and 2, and the axis-1 transform runs across the lanes with shuffles.
// MODE 0: fold, D^{0n} = Re (1/nk) sum_k exp(-i k.R_n) D^k; MODE 1: unfold,
// J^k = sum_n exp(+i k.R_n) J^{0n}.
template <int MODE, int N2, int N3, bool G3>
__global__ void __launch_bounds__(kRegBlock) k_fold_reg(const void* __restrict__ in, void* __restrict__ out,
                                                        long long E, int N1, df inv_nk) {
    constexpr int P = N2 * N3;
    constexpr bool INV = MODE == 1;
    const LaneGroup lg = lane_group(N1);
    const int j = lg.j;
    const long long e = lg.col;
    const long long d = blockIdx.y;
    const int nk = N1 * P;
    const bool valid = lg.live && e < E;
    cdf v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const long long idx = (d * nk + (long long)j * P + q) * E + e;
        if (MODE == 0) {
            const double2 x = valid ? static_cast<const double2*>(in)[idx] : make_double2(0.0, 0.0);
            v[q] = cdf{split_double(x.x), split_double(x.y)};
        } else {
            const double x = valid ? static_cast<const double*>(in)[idx] : 0.0;
            v[q] = cdf{split_double(x), {0.f, 0.f}};
        }
    }
#pragma unroll
    for (int i2 = 0; i2 < N2; ++i2) dft_reg<N3, INV>(v, i2 * N3, 1);
#pragma unroll
    for (int i3 = 0; i3 < N3; ++i3) dft_reg<N2, INV>(v, i3, N3);
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = dft_lanes<INV, G3>(v[q], j, N1);
    if (!valid) return;
    const long long base = (d * nk + (long long)out_index(j, N1) * P) * E + e;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        if (MODE == 0)
            static_cast<double*>(out)[base + (long long)q * E] = join_df(df_mul(v[q].re, inv_nk));
        else
            static_cast<double2*>(out)[base + (long long)q * E] = make_double2(join_df(v[q].re), join_df(v[q].im));
    }
}

// (mu, nu), mu <= nu, of the t-th element of the row-major upper triangle of an
// n x n matrix (row mu starts at mu n - mu (mu - 1) / 2); FP32 estimate, then
// integer correction
__device__ __forceinline__ void tri_index(long long t, int n, int& mu, int& nu) {
    const float b = 2.f * n + 1.f;
    int m = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.f * (float)t, 0.f))));
    m = min(max(m, 0), n - 1);
    auto start = [n](int r) { return (long long)r * n - (long long)r * (r - 1) / 2; };
    while (m > 0 && start(m) > t) --m;
    while (m + 1 < n && start(m + 1) <= t) ++m;
    mu = m;
    nu = m + (int)(t - start(m));
}

// The fold of a Hermitian D^k (D^k_{nu mu} = conj D^k_{mu nu}): then
// D^{0n}_{nu mu} = D^{0,-n}_{mu nu}, so only the upper triangle mu <= nu is read
// and transformed, and each result is also written, transposed, at cell -n.
// Same arithmetic and lane layout as k_fold_reg<0, N2, N3, G3>.  Six blocks
// per SM (80 registers): a 240-AO cell's 904 blocks then run in one wave.
template <int N2, int N3, bool G3>
__global__ void __launch_bounds__(kRegBlock, G3 ? 1 : 6) k_fold_reg_herm(const double2* __restrict__ in, double* __restrict__ out,
                                                             int nao, long long T, int N1, df inv_nk) {
    constexpr int P = N2 * N3;
    const LaneGroup lg = lane_group(N1);
    const int j = lg.j;
    const long long t = lg.col;
    const long long d = blockIdx.y;
    const int nk = N1 * P;
    const long long E = (long long)nao * nao;
    const bool valid = lg.live && t < T;
    int mu = 0, nu = 0;
    if (valid) tri_index(t, nao, mu, nu);
    const long long e = (long long)mu * nao + nu;
    cdf v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const double2 x = valid ? in[(d * nk + (long long)j * P + q) * E + e] : make_double2(0.0, 0.0);
        v[q] = cdf{split_double(x.x), split_double(x.y)};
    }
#pragma unroll
    for (int i2 = 0; i2 < N2; ++i2) dft_reg<N3, false>(v, i2 * N3, 1);
#pragma unroll
    for (int i3 = 0; i3 < N3; ++i3) dft_reg<N2, false>(v, i3, N3);
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = dft_lanes<false, G3>(v[q], j, N1);
    if (!valid) return;
    const int o1 = out_index(j, N1), m1 = (N1 - o1) % N1;
    const long long et = (long long)nu * nao + mu;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const double val = join_df(df_mul(v[q].re, inv_nk));
        out[(d * nk + (long long)o1 * P + q) * E + e] = val;
        if (mu != nu) {
            const int i2 = q / N3, i3 = q % N3;
            const int qm = ((N2 - i2) % N2) * N3 + (N3 - i3) % N3;
            out[(d * nk + (long long)m1 * P + qm) * E + et] = val;
        }
    }
}

int axis_code(int n) { return n >= 1 && n <= 4 ? n - 1 : -1; }

// runs f.template run<N2, N3>() for the plan's (N2, N3), both in 1..4
template <class F>
void by_plane(const ftcj_plan* P, const F& f) {
    switch (axis_code(P->km[1]) * 4 + axis_code(P->km[2])) {
        case 0: f.template run<1, 1>(); break;
        case 1: f.template run<1, 2>(); break;
        case 2: f.template run<1, 3>(); break;
        case 3: f.template run<1, 4>(); break;
        case 4: f.template run<2, 1>(); break;
        case 5: f.template run<2, 2>(); break;
        case 6: f.template run<2, 3>(); break;
        case 7: f.template run<2, 4>(); break;
        case 8: f.template run<3, 1>(); break;
        case 9: f.template run<3, 2>(); break;
        case 10: f.template run<3, 3>(); break;
        case 11: f.template run<3, 4>(); break;
        case 12: f.template run<4, 1>(); break;
        case 13: f.template run<4, 2>(); break;
        case 14: f.template run<4, 3>(); break;
        default: f.template run<4, 4>(); break;
    }
}

template <int MODE>
struct RegLaunch {
    dim3 g;
    cudaStream_t s;
    const void* in;
    void* out;
    long long E;
    int N1;
    df inv;
    template <int N2, int N3>
    void run() const {
        if (N1 == 3) k_fold_reg<MODE, N2, N3, true><<<g, kRegBlock, 0, s>>>(in, out, E, N1, inv);
        else k_fold_reg<MODE, N2, N3, false><<<g, kRegBlock, 0, s>>>(in, out, E, N1, inv);
    }
};

struct HermLaunch {
    dim3 g;
    cudaStream_t s;
    const double2* in;
    double* out;
    int nao;
    long long T;
    int N1;
    df inv;
    template <int N2, int N3>
    void run() const {
        if (N1 == 3) k_fold_reg_herm<N2, N3, true><<<g, kRegBlock, 0, s>>>(in, out, nao, T, N1, inv);
        else k_fold_reg_herm<N2, N3, false><<<g, kRegBlock, 0, s>>>(in, out, nao, T, N1, inv);
    }
};

template <int MODE>
int launch_fold_reg(const ftcj_plan* P, int ndens, const void* in, void* out, cudaStream_t s) {
    const long long E = (long long)P->nao * P->nao;
    const int N1 = P->km[0];
    by_plane(P, RegLaunch<MODE>{dim3(reg_blocks(E, N1), ndens), s, in, out, E, N1, df_from_double(1.0 / P->nk)});
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_fold_herm(const ftcj_plan* P, int ndens, const double* Dk, double* D0n, cudaStream_t s) {
    const long long T = (long long)P->nao * (P->nao + 1) / 2;
    const int N1 = P->km[0];
    by_plane(P, HermLaunch{dim3(reg_blocks(T, N1), ndens), s, reinterpret_cast<const double2*>(Dk), D0n, P->nao, T,
                           N1, df_from_double(1.0 / P->nk)});
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

// the split form's register transform covers meshes with every axis 1 to 4 long
bool reg_fold_supported(const ftcj_plan* P) {
    return P->precision == FTCJ_PREC_SPLIT && P->nk > 1 && axis_code(P->km[0]) >= 0 && axis_code(P->km[1]) >= 0 &&
           axis_code(P->km[2]) >= 0;
}

}  // namespace

int launch_twiddles(ftcj_plan* P) {
    k_twiddles<<<3, dim3(kTw, kTw)>>>(reinterpret_cast<double2*>(P->d_tw), P->km[0], P->km[1], P->km[2]);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

// Runs the stages over the axes with N > 1.  mode 0: fold (complex in, real
// out, scale 1/nk, exp(-i..)); mode 1: unfold (real in, complex out,
// exp(+i..)); mode 2: fold keeping the complex result (for the input check).
static int run_stages(ftcj_plan* P, int ndens, const double* in, double* out, int mode, cudaStream_t s) {
    long long E = (long long)P->nao * P->nao;
    long long total = (long long)ndens * P->nk * E;
    const double2* tw = reinterpret_cast<const double2*>(P->d_tw);
    std::vector<int> axes;
    if (mode == 1) {
        for (int a = 0; a < 3; ++a)
            if (P->km[a] > 1) axes.push_back(a);
    } else {
        for (int a = 2; a >= 0; --a)
            if (P->km[a] > 1) axes.push_back(a);
    }
    const int B = 256;
    if (total == 0) return FTCJ_OK;
    if (axes.empty()) {
        if (mode == 0) k_complex_to_real<<<nblocks(total, B), B, 0, s>>>(reinterpret_cast<const double2*>(in), out,
                                                                         total, 1.0);
        else if (mode == 1) k_real_to_complex<<<nblocks(total, B), B, 0, s>>>(in, reinterpret_cast<double2*>(out),
                                                                              total);
        else FTCJ_CUDA(cudaMemcpyAsync(out, in, sizeof(double) * 2 * total, cudaMemcpyDeviceToDevice, s));
        FTCJ_CUDA(cudaGetLastError());
        return FTCJ_OK;
    }
    double* bufs[2] = {P->d_cbuf0, P->d_cbuf1};
    int conj = mode == 1 ? 1 : 0;
    for (size_t st = 0; st < axes.size(); ++st) {
        bool first = st == 0, last = st + 1 == axes.size();
        const double* src = first ? in : bufs[(st - 1) & 1];
        double* dst = last ? out : bufs[st & 1];
        double scale = (last && mode != 1) ? 1.0 / P->nk : 1.0;
        int ax = axes[st];
        unsigned g = nblocks(total, B);
        if (mode == 1 && first) {
            k_dft_axis<true, false><<<g, B, 0, s>>>(src, dst, total, E, P->km[0], P->km[1], P->km[2], ax, tw, conj,
                                                    scale);
        } else if (mode == 0 && last) {
            k_dft_axis<false, true><<<g, B, 0, s>>>(src, dst, total, E, P->km[0], P->km[1], P->km[2], ax, tw, conj,
                                                    scale);
        } else {
            k_dft_axis<false, false><<<g, B, 0, s>>>(src, dst, total, E, P->km[0], P->km[1], P->km[2], ax, tw, conj,
                                                     scale);
        }
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}

static size_t fused_smem(const ftcj_plan* P) { return sizeof(double2) * (size_t)kFusedT * P->nk; }

int fused_fold_supported(const ftcj_plan* P) { return P->nk > 1 && P->nk <= kFusedMaxNk; }

int setup_fold(ftcj_plan* P) {
    if (!fused_fold_supported(P)) return FTCJ_OK;
    int rc = allow_dynamic_smem((const void*)k_fold_fused, fused_smem(P));
    if (!rc) rc = allow_dynamic_smem((const void*)k_unfold_fused, fused_smem(P));
    return rc;
}

int launch_fold(ftcj_plan* P, int ndens, const double* Dk, double* D0n, cudaStream_t s) {
    if (reg_fold_supported(P)) return launch_fold_reg<0>(P, ndens, Dk, D0n, s);
    if (!fused_fold_supported(P)) return run_stages(P, ndens, Dk, D0n, 0, s);
    long long E = (long long)P->nao * P->nao;
    dim3 g(nblocks(E, kFusedT), ndens);
    k_fold_fused<<<g, kFusedT, fused_smem(P), s>>>(reinterpret_cast<const double2*>(Dk), D0n, E, P->km[0], P->km[1],
                                                   P->km[2], reinterpret_cast<const double2*>(P->d_tw));
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

// The build's fold: D^k is Hermitian by the contract, which the split form's
// register transform uses to read and transform half of it.
int launch_fold_build(ftcj_plan* P, int ndens, const double* Dk, double* D0n, cudaStream_t s) {
    if (reg_fold_supported(P)) return launch_fold_herm(P, ndens, Dk, D0n, s);
    return launch_fold(P, ndens, Dk, D0n, s);
}

int launch_unfold(ftcj_plan* P, int ndens, const double* J0n, double* Jk, cudaStream_t s) {
    if (reg_fold_supported(P)) return launch_fold_reg<1>(P, ndens, J0n, Jk, s);
    if (!fused_fold_supported(P)) return run_stages(P, ndens, J0n, Jk, 1, s);
    long long E = (long long)P->nao * P->nao;
    dim3 g(nblocks(E, kFusedT), ndens);
    k_unfold_fused<<<g, kFusedT, fused_smem(P), s>>>(J0n, reinterpret_cast<double2*>(Jk), E, P->km[0], P->km[1],
                                                     P->km[2], reinterpret_cast<const double2*>(P->d_tw));
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_check_density(ftcj_plan* P, int ndens, const double* Dk, double* out2, cudaStream_t s) {
    // the complex fold goes to the host-variant staging buffer, which is free here
    double* full = P->d_Jk_stage;
    int rc = run_stages(P, ndens, Dk, full, 2, s);
    if (rc) return rc;
    FTCJ_CUDA(cudaMemsetAsync(out2, 0, 2 * sizeof(double), s));
    k_check<<<256, 256, 0, s>>>(reinterpret_cast<const double2*>(full), ndens, P->km[0], P->km[1], P->km[2], P->nao,
                                out2);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

}  // namespace ftcj
