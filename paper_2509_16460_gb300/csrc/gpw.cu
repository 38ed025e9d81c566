// The GPW route of the diffuse-diffuse (DD) pair densities (Sec. 2.6, App. E).
//
// A classified plan keeps its compact pair records (CC and CD) in the
// long-range walks and gives the DD records a plan of their own (P->dd): the
// same a3 / a7 maps turn D^{0n} into their relative-coordinate Hermite terms
// D'_ijk and their J'_ijk back into J^{0n}, but their structure factor and
// back-contraction run on a uniform real-space grid of the cell,
//   r_m = sum_i (m_i / N_i) a_i,  m_i = 0..N_i-1.
//
// Collocation.  A record's density, written in the walks' form
//   rho_r(G) = e^{-G^2/4p} e^{-iG.P} sum_ijk (-i)^{i+j+k} D'_ijk n1^i n2^j n3^k,
// is in real space sum_ijk D'_ijk c_ijk(r) with
//   c_ijk(r) = (2 pi)^{-(i+j+k)} (p/pi)^{3/2} H_ijk(s) e^{-p s.g s},
// s the fractional coordinates of r - P (summed over the lattice images),
// g_ab = a_a . a_b, and H the Hermite polynomials of that metric,
//   H_{m+e_a} = 2p (g s)_a H_m - 2p sum_b g_ab m_b H_{m-e_b},  H_0 = 1,
// so that (-d/ds)^m e^{-p s.g s} = H_m(s) e^{-p s.g s}: each derivative d/dF_a
// of the centre's fractional coordinate brings down -2 pi i n_a.  In an
// orthorhombic cell g is diagonal and every factor separates by axis (App. E,
// "Orthorhombic unit cells"): per record and axis a table of
//   T_a[i][m_a] = (2 pi)^{-i} sum_t H^{(a)}_i(s_a - t) e^{-p g_aa (s_a - t)^2}
// (the lattice images summed on the line, then wrapped into the cell), and
//   rho_D(m) = sum_r sum_i T_1[i][m1] sum_jk D'_ijk T_2[j][m2] T_3[k][m3],
// contracted axis by axis as the paper describes.  Other cells evaluate the
// Gaussian point by point with the lattice images in reach (App. E,
// "Non-orthorhombic unit cells", written with the product Gaussian of the pair).
//
// Transforms.  rho_D(G) = (Omega/N) sum_m rho_D(r_m) e^{-iG.r_m} for the half
// sphere's G = sum n_i b_i, where G.r_m = 2 pi sum_i n_i m_i / N_i separates:
// three passes, over m1 (all n1 of the sphere), m2 (all n2) and m3 (the sphere's
// points).  The grid is fine enough that every alias G + K of a sphere point
// (K = sum k_i N_i b_i != 0) has |G + K| >= Gcut + sqrt(184 p_max), where a DD
// transform is below e^{-46} of its peak.  The back-contraction runs the
// adjoint passes: V(r_m) = (Omega/N) Re sum_{half} W_D(G) e^{-iG.r_m}, and
// J'_ijk = sum_m c_ijk(r_m) V(r_m) (with W_D = 2 v_FR conj(rho_C + rho_D) this is
// 2 Re sum_half of the record's transform times W_D, as in the walks).
//
// Potentials (Sec. 2.6): integrals between two compact densities keep
// v_LR(G) = 4 pi e^{-G^2/4w^2} / (Omega G^2), every other one takes
// v_FR(G) = 4 pi / (Omega G^2):
//   W_C = 2 [v_LR conj(rho_C) + v_FR conj(rho_D)]   (the compact records' walks)
//   W_D = 2 v_FR conj(rho_C + rho_D)                (the DD records, on the grid)
//   E_J = sum_half v_LR |rho_C|^2 + v_FR (2 Re rho_C conj(rho_D) + |rho_D|^2).
//
// The FP64 form runs everything in FP64.  The split form runs the two grid
// contractions (collocation and integration, the route's flops) in
// double-float on the FP32 pipe, with tables and V(r_m) stored as (hi, lo)
// float pairs; the transforms, potentials and sums stay FP64.  The partial
// grids of the collocation and the energy partials are summed in a fixed
// order (no atomics).
#include <algorithm>
#include <cmath>
#include <vector>

#include "df.cuh"
#include "ftcj_internal.h"

namespace ftcj {

struct Gpw {
    int N[3] = {0, 0, 0};     // grid points along a_1..a_3
    long long npts = 0;       // N1 N2 N3
    int nlo[3] = {0, 0, 0};   // the half sphere's n_i run over [nlo_i, nlo_i + ncnt_i)
    int ncnt[3] = {0, 0, 0};
    bool sep = false;         // orthorhombic: per-axis tables
    int lmax = 0;             // highest class of the DD records
    int nsplit = 1;           // record splits of the collocation (partial grids)
    long long tstride = 0;    // table entries of one record: (lmax + 1)(N1 + N2 + N3)
    double gnorm = 0.0;       // Omega / (N1 N2 N3)
    bool df = false;          // split form: the grid contractions in double-float on the FP32 pipe
    double* d_tab = nullptr;    // [tstride][nrec], the record index fastest
    float2* d_tabf = nullptr;   // the same tables as double-float (hi, lo), split form
    float2* d_tabfr = nullptr;  // [nrec][tstride]: the double-float tables record by record (collocation)
    float2* d_vf = nullptr;     // [max_dens][npts]: V(r_m) as double-float, split form
    double* d_part = nullptr;   // [nsplit][max_dens][npts]
    double* d_grid = nullptr;   // [max_dens][npts]: rho_D(r_m), then V(r_m)
    double2* d_t1 = nullptr;    // [max_dens][ncnt0][N2][N3]
    double2* d_t2 = nullptr;    // [max_dens][ncnt0][ncnt1][N3]
    double2* d_rhoD = nullptr;  // [max_dens][ng_half]
    double2* d_WD = nullptr;    // [max_dens][ng_half]
    double* d_vfr = nullptr;    // [ng_half]
    double* d_Epart = nullptr;  // [max_dens][nEb]
    double2* d_tw = nullptr;    // e^{-2 pi i k / N_a} for k < N_a, the three axes one after the other
    int nsj = 1;                // splits of the m2 rows in the integration (partial J' summed in order)
    size_t vplane_bytes = 0;    // shared memory of the double-float integration: one plane V(., m2, .)
    double* d_jpart = nullptr;  // [nsj][max_dens][total_terms of the DD records]
    int* d_cstart = nullptr;    // [ncnt0 ncnt1 + 1]: the half sphere's points by (n1, n2)
    int* d_clist = nullptr;     // [ng_half]
    int nEb = 0;
    size_t bytes = 0;
};

namespace {

constexpr int kGpwThreads = 128;
constexpr int kM1 = 32;  // m1 values a collocation thread holds at a time
constexpr double kGaussCut = 50.0;  // images with p |r - P|^2 above this are dropped (e^{-50})

struct DdLayout {
    long long start[kNclass + 1];
    long long base[kNclass];
    long long total;
};

struct Lattice {
    double A[9];    // rows a_i
    double g[9];    // a_i . a_j
    double bn[3];   // |b_i| / (2 pi)
};

// exp(-2 pi i k / n) from the axis's table, k reduced into [0, n) exactly
__device__ __forceinline__ void twiddle(const double2* __restrict__ tw, long long k, int n, double& c, double& s) {
    long long r = k % n;
    if (r < 0) r += n;
    const double2 v = __ldg(tw + r);
    c = v.x;
    s = v.y;
}

__global__ void k_gpw_twiddles(int N0, int N1, int N2, double2* __restrict__ tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N0 + N1 + N2) return;
    const int n = k < N0 ? N0 : (k < N0 + N1 ? N1 : N2);
    const int j = k < N0 ? k : (k < N0 + N1 ? k - N0 : k - N0 - N1);
    double sn, cs;
    sincospi(2.0 * (double)j / (double)n, &sn, &cs);
    tw[k] = make_double2(cs, -sn);
}

// fractional coordinates of the record's product centre P
__device__ __forceinline__ void centre_frac(const PairDev& pr, const CellConst& cc, double F[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
        F[a] = cc.Bt[3 * a] * pr.P[0] + cc.Bt[3 * a + 1] * pr.P[1] + cc.Bt[3 * a + 2] * pr.P[2];
}

// ---- per-axis tables of the separable form (plan setup) --------------------

// One thread per (record, axis, grid index): T_a[i][m] for i <= class.
__global__ void k_gpw_tables(const PairDev* __restrict__ pairs, long long nrec, int lmax, int N0, int N1, int N2,
                             Lattice lat, CellConst cc, double* __restrict__ tab, float2* __restrict__ tabf,
                             float2* __restrict__ tabfr) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Nt = N0 + N1 + N2;
    if (tid >= nrec * Nt) return;
    const long long r = tid / Nt;
    int m = (int)(tid % Nt), ax = 0, n = N0, off = 0;
    if (m >= N0 + N1) {
        ax = 2;
        m -= N0 + N1;
        n = N2;
        off = (lmax + 1) * (N0 + N1);
    } else if (m >= N0) {
        ax = 1;
        m -= N0;
        n = N1;
        off = (lmax + 1) * N0;
    }
    const PairDev pr = pairs[r];
    const int L = pr.cls;
    double F[3];
    centre_frac(pr, cc, F);
    const double p = pr.p, gaa = lat.g[4 * ax];
    const double s0 = (double)m / (double)n - F[ax];
    const double reach = sqrt(kGaussCut / (p * gaa));
    const long long tlo = (long long)ceil(s0 - reach), thi = (long long)floor(s0 + reach);
    double acc[kLpair + 1];
#pragma unroll
    for (int i = 0; i <= kLpair; ++i) acc[i] = 0.0;
    const double two_pg = 2.0 * p * gaa;
    for (long long t = tlo; t <= thi; ++t) {
        const double s = s0 - (double)t;
        const double e = exp(-p * gaa * s * s);
        double hm = 0.0, h = 1.0;  // H_{i-1}, H_i
        acc[0] += e;
        for (int i = 1; i <= L; ++i) {
            const double hn = two_pg * s * h - two_pg * (double)(i - 1) * hm;
            hm = h;
            h = hn;
            acc[i] += h * e;
        }
    }
    double scale = ax == 0 ? pow(p / M_PI, 1.5) : 1.0;
    for (int i = 0; i <= lmax; ++i) {
        const double v = i <= L ? acc[i] * scale : 0.0;
        const long long e = ((long long)off + (long long)i * n + m) * nrec + r;
        tab[e] = v;
        if (tabf) {
            const float hi = (float)v;
            tabf[e] = make_float2(hi, (float)(v - (double)hi));
            tabfr[r * ((long long)(lmax + 1) * (N0 + N1 + N2)) + off + (long long)i * n + m] = tabf[e];
        }
        scale *= 1.0 / (2.0 * M_PI);
    }
}

// ---- collocation ------------------------------------------------------------

// Separable form, the records of class L: one thread per grid line (m2, m3)
// and up to kM1 values of m1 at a time; blockIdx.y splits the records,
// blockIdx.z is the density.  Each record adds
//   sum_i T_1[i][m1] w_i,  w_i = sum_jk D'_ijk T_2[j][m2] T_3[k][m3]
// to its split's partial grid (the first class launched writes it, the later
// ones add to it, in launch order).
template <int L>
__global__ void __launch_bounds__(kGpwThreads) k_gpw_collocate_sep(const double* __restrict__ tab, long long nrec,
                                                                  int lmax, int N0, int N1, int N2,
                                                                  const double* __restrict__ Dp, DdLayout lay,
                                                                  int nsplit, int nd, long long npts, bool add,
                                                                  double* __restrict__ part) {
    const int d = blockIdx.z, split = blockIdx.y;
    const int lines = N1 * N2;
    const int line = blockIdx.x * kGpwThreads + threadIdx.x;
    if (line >= lines) return;
    const int m2 = line / N2, m3 = line % N2;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long r0 = lay.start[L] + cnt * split / nsplit, r1 = lay.start[L] + cnt * (split + 1) / nsplit;
    const long long off1 = (long long)(lmax + 1) * N0, off2 = (long long)(lmax + 1) * (N0 + N1);
    const double* Dd = Dp + (long long)d * lay.total + lay.base[L] - lay.start[L];
    double* out = part + ((long long)split * nd + d) * npts + line;
    constexpr int M = L == 0 ? kM1 : (L <= 2 ? kM1 / 2 : kM1 / 4);  // registers: every T_1 load is hoisted
    for (int mb = 0; mb < N0; mb += M) {
        const int mcnt = min(M, N0 - mb);
        double acc[M];
#pragma unroll
        for (int q = 0; q < M; ++q) acc[q] = 0.0;
        for (long long r = r0; r < r1; ++r) {
            double t2[L + 1], t3[L + 1], w[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) {
                t2[i] = __ldg(tab + (off1 + (long long)i * N1 + m2) * nrec + r);
                t3[i] = __ldg(tab + (off2 + (long long)i * N2 + m3) * nrec + r);
                w[i] = 0.0;
            }
            int t = 0;
#pragma unroll
            for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                for (int a = lam; a >= 0; --a)
#pragma unroll
                    for (int b = lam - a; b >= 0; --b, ++t)
                        w[a] = fma(__ldg(Dd + (long long)t * cnt + r), t2[b] * t3[lam - a - b], w[a]);
            const double* T1 = tab + (long long)mb * nrec + r;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                if (q < mcnt) {
                    double v = acc[q];
#pragma unroll
                    for (int a = 0; a <= L; ++a) v = fma(__ldg(T1 + ((long long)a * N0 + q) * nrec), w[a], v);
                    acc[q] = v;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < M; ++q)
            if (q < mcnt) {
                double* o = out + (long long)(mb + q) * lines;
                *o = add ? *o + acc[q] : acc[q];
            }
    }
}

__device__ __forceinline__ df ld_df(const float2* p) {
    const float2 v = __ldg(p);
    return df{v.x, v.y};
}

// The separable collocation in double-float (split form): the same sums as
// k_gpw_collocate_sep, every product and sum an error-free double-float step
// on the FP32 pipe (D'_ijk split from FP64 with integer operations); the
// accumulators are renormalised every four records and joined to FP64 once.
// The block stages the T_1 rows and D' terms of 32 records at a time in
// shared memory (one coalesced load per chunk instead of a dependent load per
// record); each thread reads its T_2[j][m2] and T_3[k][m3] from the
// record-major tables (tabfr), a few contiguous lines per warp, loading the
// next record's while the current one is added.
constexpr int kColChunk = 32;

template <int L>
__global__ void __launch_bounds__(kGpwThreads) k_gpw_collocate_sep_df(const float2* __restrict__ tabfr, long long nrec,
                                                                     int lmax, int N0, int N1, int N2,
                                                                     const double* __restrict__ Dp, DdLayout lay,
                                                                     int nsplit, int nd, long long npts, bool add,
                                                                     double* __restrict__ part) {
    constexpr int NT = nterms(L);
    constexpr int M = L == 0 ? kM1 : (L <= 2 ? kM1 / 2 : kM1 / 4);
    __shared__ float2 sT1[kColChunk][L + 1][M];
    __shared__ double sD[kColChunk][NT];
    const int d = blockIdx.z, split = blockIdx.y;
    const int lines = N1 * N2;
    const int line = blockIdx.x * kGpwThreads + threadIdx.x;
    const bool live = line < lines;
    const int m2 = live ? line / N2 : 0, m3 = live ? line % N2 : 0;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long r0 = lay.start[L] + cnt * split / nsplit, r1 = lay.start[L] + cnt * (split + 1) / nsplit;
    const long long tstride = (long long)(lmax + 1) * (N0 + N1 + N2);
    const long long off1 = (long long)(lmax + 1) * N0, off2 = (long long)(lmax + 1) * (N0 + N1);
    const double* Dd = Dp + (long long)d * lay.total + lay.base[L] - lay.start[L];
    double* out = part + ((long long)split * nd + d) * npts + line;
    for (int mb = 0; mb < N0; mb += M) {
        const int mcnt = min(M, N0 - mb);
        df acc[M];
#pragma unroll
        for (int q = 0; q < M; ++q) acc[q] = df{0.f, 0.f};
        float2 n2[L + 1], n3[L + 1];
        if (r0 < r1) {
            const float2* row = tabfr + r0 * tstride;
#pragma unroll
            for (int i = 0; i <= L; ++i) {
                n2[i] = __ldg(row + off1 + (long long)i * N1 + m2);
                n3[i] = __ldg(row + off2 + (long long)i * N2 + m3);
            }
        }
        for (long long c0 = r0; c0 < r1; c0 += kColChunk) {
            const int kc = (int)min((long long)kColChunk, r1 - c0);
            __syncthreads();  // the previous chunk is consumed
            for (int e = threadIdx.x; e < kc * (L + 1) * M; e += kGpwThreads) {
                const int rec = e / ((L + 1) * M), a = (e / M) % (L + 1), q = e % M;
                sT1[rec][a][q] = q < mcnt ? __ldg(tabfr + (c0 + rec) * tstride + (long long)a * N0 + mb + q)
                                          : make_float2(0.f, 0.f);
            }
            for (int e = threadIdx.x; e < kc * NT; e += kGpwThreads) {
                const int rec = e / NT, t = e % NT;
                sD[rec][t] = __ldg(Dd + (long long)t * cnt + c0 + rec);
            }
            __syncthreads();
            for (int rec = 0; rec < kc; ++rec) {
                const long long r = c0 + rec;
                df t2[L + 1], t3[L + 1], w[L + 1];
#pragma unroll
                for (int i = 0; i <= L; ++i) {
                    t2[i] = df{n2[i].x, n2[i].y};
                    t3[i] = df{n3[i].x, n3[i].y};
                    w[i] = df{0.f, 0.f};
                }
                if (r + 1 < r1) {
                    const float2* row = tabfr + (r + 1) * tstride;
#pragma unroll
                    for (int i = 0; i <= L; ++i) {
                        n2[i] = __ldg(row + off1 + (long long)i * N1 + m2);
                        n3[i] = __ldg(row + off2 + (long long)i * N2 + m3);
                    }
                }
                int t = 0;
#pragma unroll
                for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                    for (int a = lam; a >= 0; --a)
#pragma unroll
                        for (int b = lam - a; b >= 0; --b, ++t)
                            w[a] = df_add_u(w[a], df_mul_u(split_double(sD[rec][t]), df_mul_u(t2[b], t3[lam - a - b])));
#pragma unroll
                for (int a = 0; a <= L; ++a) w[a] = df_norm(w[a]);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    df v = acc[q];
#pragma unroll
                    for (int a = 0; a <= L; ++a) {
                        const float2 x = sT1[rec][a][q];
                        v = df_add_u(v, df_mul_u(df{x.x, x.y}, w[a]));
                    }
                    acc[q] = v;
                }
                if ((rec & 3) == 3) {
#pragma unroll
                    for (int q = 0; q < M; ++q) acc[q] = df_norm(acc[q]);
                }
            }
        }
        if (live) {
#pragma unroll
            for (int q = 0; q < M; ++q)
                if (q < mcnt) {
                    double* o = out + (long long)(mb + q) * lines;
                    const double v = join_df(df_norm(acc[q]));
                    *o = add ? *o + v : v;
                }
        }
    }
}

// Hermite polynomials of the metric g at the fractional displacement s, up to
// degree L, in the Hermite-term order (degree lam, then n1 power a = lam..0,
// n2 power b = lam-a..0): H_{m+e_x} = 2p (g s)_x H_m - 2p sum_y g_xy m_y H_{m-e_y}.
__device__ void hermite_metric(int L, double p, const double* g, const double s[3], double* H) {
    double gs[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) gs[x] = g[3 * x] * s[0] + g[3 * x + 1] * s[1] + g[3 * x + 2] * s[2];
    H[0] = 1.0;
    const double tp = 2.0 * p;
    for (int lam = 1; lam <= L; ++lam) {
        int t = lam_offset(lam);
        for (int a = lam; a >= 0; --a)
            for (int b = lam - a; b >= 0; --b, ++t) {
                const int c = lam - a - b;
                int m[3] = {a, b, c};
                const int x = a > 0 ? 0 : (b > 0 ? 1 : 2);  // the step: m = (a, b, c) - e_x
                --m[x];
                const int lm = lam - 1;
                double v = tp * gs[x] * H[lam_offset(lm) + mono_index(lm, m[0], m[1])];
                for (int y = 0; y < 3; ++y) {
                    if (m[y] == 0) continue;
                    int q[3] = {m[0], m[1], m[2]};
                    --q[y];
                    v -= tp * g[3 * x + y] * (double)m[y] * H[lam_offset(lm - 1) + mono_index(lm - 1, q[0], q[1])];
                }
                H[t] = v;
            }
    }
}

// General cell: one thread per grid point; every record's images within
// p |r - P - T|^2 <= 50 (blockIdx.y splits the records, blockIdx.z the density).
__global__ void __launch_bounds__(kGpwThreads) k_gpw_collocate_gen(const PairDev* __restrict__ pairs, long long nrec,
                                                                  int N0, int N1, int N2, const double* __restrict__ Dp,
                                                                  DdLayout lay, Lattice lat, CellConst cc, int nsplit,
                                                                  int nd, long long npts, double* __restrict__ part) {
    const int d = blockIdx.z, split = blockIdx.y;
    const long long m = (long long)blockIdx.x * kGpwThreads + threadIdx.x;
    if (m >= npts) return;
    const int m1 = (int)(m / ((long long)N1 * N2)), m2 = (int)((m / N2) % N1), m3 = (int)(m % N2);
    const double f[3] = {(double)m1 / N0, (double)m2 / N1, (double)m3 / N2};
    const long long r0 = nrec * split / nsplit, r1 = nrec * (split + 1) / nsplit;
    const double* Dd = Dp + (long long)d * lay.total;
    double H[kMaxTerms];
    double acc = 0.0;
    for (long long r = r0; r < r1; ++r) {
        const PairDev pr = pairs[r];
        const int L = pr.cls;
        const long long cnt = lay.start[L + 1] - lay.start[L], loc = r - lay.start[L];
        double F[3];
        centre_frac(pr, cc, F);
        const double p = pr.p, rs = sqrt(kGaussCut / p);
        int tlo[3], thi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double s0 = f[a] - F[a], reach = rs * lat.bn[a];
            tlo[a] = (int)ceil(s0 - reach);
            thi[a] = (int)floor(s0 + reach);
        }
        const double pref = pow(p / M_PI, 1.5);
        for (int t1 = tlo[0]; t1 <= thi[0]; ++t1)
            for (int t2 = tlo[1]; t2 <= thi[1]; ++t2)
                for (int t3 = tlo[2]; t3 <= thi[2]; ++t3) {
                    const double s[3] = {f[0] - F[0] - t1, f[1] - F[1] - t2, f[2] - F[2] - t3};
                    double q = 0.0;
#pragma unroll
                    for (int x = 0; x < 3; ++x)
#pragma unroll
                        for (int y = 0; y < 3; ++y) q += lat.g[3 * x + y] * s[x] * s[y];
                    if (p * q > kGaussCut) continue;
                    const double e = pref * exp(-p * q);
                    hermite_metric(L, p, lat.g, s, H);
                    double v = 0.0, sc = 1.0;
                    int t = 0;
                    for (int lam = 0; lam <= L; ++lam, sc *= 1.0 / (2.0 * M_PI))
                        for (int i = 0; i < nmono(lam); ++i, ++t)
                            v += sc * H[t] * __ldg(Dd + lay.base[L] + (long long)t * cnt + loc);
                    acc += e * v;
                }
    }
    part[((long long)split * nd + d) * npts + m] = acc;
}

// rho_D(r_m) = sum over the record splits, in split order
__global__ void k_gpw_reduce(const double* __restrict__ part, int nsplit, int nd, long long npts,
                             double* __restrict__ grid) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (m >= npts) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += part[((long long)q * nd + d) * npts + m];
    grid[(long long)d * npts + m] = s;
}

// ---- grid <-> sphere transforms ---------------------------------------------

// pass 1: t1[n1][m2][m3] = sum_m1 rho(m1, m2, m3) e^{-2 pi i n1 m1 / N0}
__global__ void k_gpw_dft1(const double* __restrict__ grid, const double2* __restrict__ tw, int N0, int N1, int N2,
                           int nlo0, int ncnt0, long long npts, double2* __restrict__ t1) {
    const int d = blockIdx.y;
    const long long lines = (long long)N1 * N2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncnt0 * lines) return;
    const int n1 = nlo0 + (int)(idx / lines);
    const long long line = idx % lines;
    const double* src = grid + (long long)d * npts + line;
    double re = 0.0, im = 0.0;
    for (int m1 = 0; m1 < N0; ++m1) {
        double c, s;
        twiddle(tw, (long long)n1 * m1, N0, c, s);
        const double v = src[(long long)m1 * lines];
        re = fma(v, c, re);
        im = fma(v, s, im);
    }
    t1[(long long)d * ncnt0 * lines + idx] = make_double2(re, im);
}

// pass 2: t2[n1][n2][m3] = sum_m2 t1[n1][m2][m3] e^{-2 pi i n2 m2 / N1}
__global__ void k_gpw_dft2(const double2* __restrict__ t1, const double2* __restrict__ tw, int N1, int N2, int ncnt0,
                           int nlo1, int ncnt1, double2* __restrict__ t2) {
    const int d = blockIdx.y;
    const long long total = (long long)ncnt0 * ncnt1 * N2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int m3 = (int)(idx % N2);
    const int n2i = (int)((idx / N2) % ncnt1), n1i = (int)(idx / ((long long)N2 * ncnt1));
    const int n2 = nlo1 + n2i;
    const double2* src = t1 + ((long long)d * ncnt0 + n1i) * N1 * N2 + m3;
    double re = 0.0, im = 0.0;
    for (int m2 = 0; m2 < N1; ++m2) {
        double c, s;
        twiddle(tw, (long long)n2 * m2, N1, c, s);
        const double2 v = src[(long long)m2 * N2];
        re += v.x * c - v.y * s;
        im += v.x * s + v.y * c;
    }
    t2[(long long)d * total + idx] = make_double2(re, im);
}

// pass 3: rho_D(G_p) = (Omega/N) sum_m3 t2[n1][n2][m3] e^{-2 pi i n3 m3 / N2}
__global__ void k_gpw_dft3(const double2* __restrict__ t2, const double2* __restrict__ tw, const int* __restrict__ gvec,
                           long long ng, int N2, int nlo0, int ncnt0, int nlo1, int ncnt1, double gnorm,
                           double2* __restrict__ rho) {
    const int d = blockIdx.y;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ng) return;
    const int n1 = gvec[3 * p], n2 = gvec[3 * p + 1], n3 = gvec[3 * p + 2];
    const double2* src = t2 + (((long long)d * ncnt0 + (n1 - nlo0)) * ncnt1 + (n2 - nlo1)) * N2;
    double re = 0.0, im = 0.0;
    for (int m3 = 0; m3 < N2; ++m3) {
        double c, s;
        twiddle(tw, (long long)n3 * m3, N2, c, s);
        const double2 v = src[m3];
        re += v.x * c - v.y * s;
        im += v.x * s + v.y * c;
    }
    rho[(long long)d * ng + p] = make_double2(gnorm * re, gnorm * im);
}

// ---- potentials and energy (Sec. 2.6) ---------------------------------------

__global__ void __launch_bounds__(256) k_gpw_potential(const double2* __restrict__ rhoC, const double2* __restrict__ rhoD,
                                                      const double* __restrict__ vlr, const double* __restrict__ vfr,
                                                      long long ng, double2* __restrict__ WC, double2* __restrict__ WD,
                                                      double* __restrict__ Epart, int nEb) {
    __shared__ double se[256];
    const int d = blockIdx.y;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (p < ng) {
        const double2 c = rhoC[(long long)d * ng + p], q = rhoD[(long long)d * ng + p];
        const double vl = vlr[p], vf = vfr[p];
        WC[(long long)d * ng + p] = make_double2(2.0 * (vl * c.x + vf * q.x), -2.0 * (vl * c.y + vf * q.y));
        WD[(long long)d * ng + p] = make_double2(2.0 * vf * (c.x + q.x), -2.0 * vf * (c.y + q.y));
        e = vl * (c.x * c.x + c.y * c.y) + vf * (2.0 * (c.x * q.x + c.y * q.y) + q.x * q.x + q.y * q.y);
    }
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) Epart[(long long)d * nEb + blockIdx.x] = se[0];
}

__global__ void __launch_bounds__(256) k_gpw_energy(const double* __restrict__ Epart, int nEb, double* __restrict__ EJ) {
    __shared__ double se[256];
    const int d = blockIdx.x;
    double e = 0.0;
    for (int i = threadIdx.x; i < nEb; i += blockDim.x) e += Epart[(long long)d * nEb + i];
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) EJ[d] = se[0];
}

__global__ void k_gpw_vfr(const int* __restrict__ gvec, long long n, CellConst cc, double* __restrict__ vfr) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double n1 = gvec[3 * p], n2 = gvec[3 * p + 1], n3 = gvec[3 * p + 2];
    const double g2 = cc.M6[0] * n1 * n1 + cc.M6[1] * n2 * n2 + cc.M6[2] * n3 * n3 +
                      2.0 * (cc.M6[3] * n1 * n2 + cc.M6[4] * n1 * n3 + cc.M6[5] * n2 * n3);
    vfr[p] = cc.vpar[0] / g2;
}

// ---- adjoint passes: V(r_m) = (Omega/N) Re sum_half W_D(G) e^{-iG.r_m} -----------

// pass 3^T: u2[n1][n2][m3] = sum over the points of (n1, n2) of W_D e^{-2 pi i n3 m3 / N2}
__global__ void k_gpw_adj3(const double2* __restrict__ WD, const double2* __restrict__ tw, const int* __restrict__ gvec,
                           long long ng, const int* __restrict__ cstart, const int* __restrict__ clist, int N2,
                           int ncnt0, int ncnt1, double2* __restrict__ u2) {
    const int d = blockIdx.y;
    const long long total = (long long)ncnt0 * ncnt1 * N2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int m3 = (int)(idx % N2);
    const long long cell = idx / N2;
    double re = 0.0, im = 0.0;
    for (int k = cstart[cell]; k < cstart[cell + 1]; ++k) {
        const int p = clist[k];
        double c, s;
        twiddle(tw, (long long)gvec[3 * p + 2] * m3, N2, c, s);
        const double2 w = WD[(long long)d * ng + p];
        re += w.x * c - w.y * s;
        im += w.x * s + w.y * c;
    }
    u2[(long long)d * total + idx] = make_double2(re, im);
}

// pass 2^T: u1[n1][m2][m3] = sum_n2 u2[n1][n2][m3] e^{-2 pi i n2 m2 / N1}
__global__ void k_gpw_adj2(const double2* __restrict__ u2, const double2* __restrict__ tw, int N1, int N2, int ncnt0,
                           int nlo1, int ncnt1, double2* __restrict__ u1) {
    const int d = blockIdx.y;
    const long long total = (long long)ncnt0 * N1 * N2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int m3 = (int)(idx % N2), m2 = (int)((idx / N2) % N1), n1i = (int)(idx / ((long long)N1 * N2));
    const double2* src = u2 + ((long long)d * ncnt0 + n1i) * ncnt1 * N2 + m3;
    double re = 0.0, im = 0.0;
    for (int n2i = 0; n2i < ncnt1; ++n2i) {
        double c, s;
        twiddle(tw, (long long)(nlo1 + n2i) * m2, N1, c, s);
        const double2 v = src[(long long)n2i * N2];
        re += v.x * c - v.y * s;
        im += v.x * s + v.y * c;
    }
    u1[(long long)d * total + idx] = make_double2(re, im);
}

// pass 1^T: V[m1][m2][m3] = (Omega/N) Re sum_n1 u1[n1][m2][m3] e^{-2 pi i n1 m1 / N0}
__global__ void k_gpw_adj1(const double2* __restrict__ u1, const double2* __restrict__ tw, int N0, int N1, int N2,
                           int nlo0, int ncnt0, long long npts, double gnorm, double* __restrict__ V,
                           float2* __restrict__ Vf) {
    const int d = blockIdx.y;
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= npts) return;
    const long long lines = (long long)N1 * N2;
    const int m1 = (int)(m / lines);
    const long long line = m % lines;
    const double2* src = u1 + (long long)d * ncnt0 * lines + line;
    double re = 0.0;
    for (int n1i = 0; n1i < ncnt0; ++n1i) {
        double c, s;
        twiddle(tw, (long long)(nlo0 + n1i) * m1, N0, c, s);
        const double2 v = src[(long long)n1i * lines];
        re += v.x * c - v.y * s;
    }
    const double v = gnorm * re;
    V[(long long)d * npts + m] = v;
    if (Vf) {
        const float hi = (float)v;
        Vf[(long long)d * npts + m] = make_float2(hi, (float)(v - (double)hi));
    }
}

// ---- integration: J'_ijk = sum_m c_ijk(r_m) V(r_m) ---------------------------------

// Separable form, one thread per record of class L (blockIdx.y the density):
// per grid line a_i = sum_m1 T_1[i][m1] V(m1, m2, m3), then every term
// J'_ijk += a_i T_2[j][m2] T_3[k][m3].
template <int L>
__global__ void __launch_bounds__(kGpwThreads) k_gpw_integrate_sep(const double* __restrict__ tab, long long nrec,
                                                                  int lmax, int N0, int N1, int N2, DdLayout lay,
                                                                  const double* __restrict__ V, long long npts,
                                                                  double* __restrict__ Jp) {
    constexpr int NT = nterms(L);
    const int d = blockIdx.y, sj = blockIdx.z, nsj = gridDim.z;
    const int m2lo = N1 * sj / nsj, m2hi = N1 * (sj + 1) / nsj;
    const long long loc = (long long)blockIdx.x * kGpwThreads + threadIdx.x;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    if (loc >= cnt) return;
    const long long r = lay.start[L] + loc;
    const long long off1 = (long long)(lmax + 1) * N0, off2 = (long long)(lmax + 1) * (N0 + N1);
    const long long lines = (long long)N1 * N2;
    const double* Vd = V + (long long)d * npts;
    double J[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) J[t] = 0.0;
    for (int m2 = m2lo; m2 < m2hi; ++m2) {
        double t2[L + 1];
#pragma unroll
        for (int j = 0; j <= L; ++j) t2[j] = __ldg(tab + (off1 + (long long)j * N1 + m2) * nrec + r);
        for (int m3 = 0; m3 < N2; ++m3) {
            const long long line = (long long)m2 * N2 + m3;
            double a[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) a[i] = 0.0;
            for (int m1 = 0; m1 < N0; ++m1) {
                const double v = __ldg(Vd + (long long)m1 * lines + line);
#pragma unroll
                for (int i = 0; i <= L; ++i) a[i] = fma(__ldg(tab + ((long long)i * N0 + m1) * nrec + r), v, a[i]);
            }
            double t3[L + 1];
#pragma unroll
            for (int k = 0; k <= L; ++k) t3[k] = __ldg(tab + (off2 + (long long)k * N2 + m3) * nrec + r);
            int t = 0;
#pragma unroll
            for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                for (int i = lam; i >= 0; --i)
#pragma unroll
                    for (int j = lam - i; j >= 0; --j, ++t) J[t] = fma(a[i], t2[j] * t3[lam - i - j], J[t]);
        }
    }
    double* out = Jp + ((long long)sj * gridDim.y + d) * lay.total + lay.base[L] + loc;
#pragma unroll
    for (int t = 0; t < NT; ++t) out[(long long)t * cnt] = J[t];
}

// The separable integration in double-float (split form): per grid line
// a_i = sum_m1 T_1[i][m1] V(m1, m2, m3) and J'_ijk += a_i T_2[j][m2] T_3[k][m3]
// as error-free double-float steps.  For each m2 row the block stages the
// plane V(., m2, .) in shared memory (one coalesced load; every thread then
// reads the same values); a class-0 record keeps its T_1 row in registers
// when N0 <= 32.  Threads past the class's records take part in the staging.
template <int L>
__global__ void __launch_bounds__(kGpwThreads) k_gpw_integrate_sep_df(const float2* __restrict__ tabf, long long nrec,
                                                                     int lmax, int N0, int N1, int N2, DdLayout lay,
                                                                     const float2* __restrict__ Vf, long long npts,
                                                                     double* __restrict__ Jp) {
    constexpr int NT = nterms(L);
    constexpr int R = 32;  // T_1 entries a class-0 thread keeps in registers
    extern __shared__ float2 sV[];  // [N0][N2]: V(m1, m2, m3) of the current m2
    const int d = blockIdx.y, sj = blockIdx.z, nsj = gridDim.z;
    const int m2lo = N1 * sj / nsj, m2hi = N1 * (sj + 1) / nsj;
    const long long loc = (long long)blockIdx.x * kGpwThreads + threadIdx.x;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const bool live = loc < cnt;
    const long long r = lay.start[L] + (live ? loc : 0);
    const long long off1 = (long long)(lmax + 1) * N0, off2 = (long long)(lmax + 1) * (N0 + N1);
    const long long lines = (long long)N1 * N2;
    const float2* Vd = Vf + (long long)d * npts;
    const bool regs = L == 0 && N0 <= R;
    df t1r[L == 0 ? R : 1];
    if (regs) {
#pragma unroll
        for (int q = 0; q < (L == 0 ? R : 1); ++q)
            t1r[q] = q < N0 && live ? ld_df(tabf + (long long)q * nrec + r) : df{0.f, 0.f};
    }
    df J[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) J[t] = df{0.f, 0.f};
    for (int m2 = m2lo; m2 < m2hi; ++m2) {
        __syncthreads();  // the previous plane is consumed
        for (int e = threadIdx.x; e < N0 * N2; e += kGpwThreads) {
            const int m1 = e / N2, m3 = e % N2;
            sV[e] = __ldg(Vd + (long long)m1 * lines + (long long)m2 * N2 + m3);
        }
        __syncthreads();
        if (!live) continue;
        df t2[L + 1];
#pragma unroll
        for (int j = 0; j <= L; ++j) t2[j] = ld_df(tabf + (off1 + (long long)j * N1 + m2) * nrec + r);
        for (int m3 = 0; m3 < N2; ++m3) {
            df t3[L + 1];
#pragma unroll
            for (int k = 0; k <= L; ++k) t3[k] = ld_df(tabf + (off2 + (long long)k * N2 + m3) * nrec + r);
            df a[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) a[i] = df{0.f, 0.f};
            if (regs) {
#pragma unroll
                for (int q = 0; q < (L == 0 ? R : 1); ++q) {
                    if (q < N0) {
                        const float2 v = sV[q * N2 + m3];
                        a[0] = df_add_u(a[0], df_mul_u(t1r[q], df{v.x, v.y}));
                        if ((q & 7) == 7) a[0] = df_norm(a[0]);
                    }
                }
            } else {
                for (int m1 = 0; m1 < N0; ++m1) {
                    const float2 v = sV[m1 * N2 + m3];
#pragma unroll
                    for (int i = 0; i <= L; ++i)
                        a[i] = df_add_u(a[i], df_mul_u(ld_df(tabf + ((long long)i * N0 + m1) * nrec + r), df{v.x, v.y}));
                    if ((m1 & 7) == 7) {
#pragma unroll
                        for (int i = 0; i <= L; ++i) a[i] = df_norm(a[i]);
                    }
                }
            }
            int t = 0;
#pragma unroll
            for (int lam = 0; lam <= L; ++lam)
#pragma unroll
                for (int i = lam; i >= 0; --i)
#pragma unroll
                    for (int j = lam - i; j >= 0; --j, ++t)
                        J[t] = df_norm(df_add_u(J[t], df_mul_u(df_norm(a[i]), df_mul_u(t2[j], t3[lam - i - j]))));
        }
    }
    if (!live) return;
    double* out = Jp + ((long long)sj * gridDim.y + d) * lay.total + lay.base[L] + loc;
#pragma unroll
    for (int t = 0; t < NT; ++t) out[(long long)t * cnt] = join_df(J[t]);
}

// J'_t = the partial sums of the m2 splits, in split order
__global__ void k_gpw_jsum(const double* __restrict__ part, int nsj, int nd, long long total, double* __restrict__ Jp) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (e >= total) return;
    double v = 0.0;
    for (int q = 0; q < nsj; ++q) v += part[((long long)q * nd + d) * total + e];
    Jp[(long long)d * total + e] = v;
}

// General cell: one thread per record, every grid point and lattice image in reach.
__global__ void __launch_bounds__(kGpwThreads) k_gpw_integrate_gen(const PairDev* __restrict__ pairs, long long nrec,
                                                                  int N0, int N1, int N2, DdLayout lay, Lattice lat,
                                                                  CellConst cc, const double* __restrict__ V,
                                                                  long long npts, double* __restrict__ Jp) {
    const int d = blockIdx.y;
    const long long r = (long long)blockIdx.x * kGpwThreads + threadIdx.x;
    if (r >= nrec) return;
    const PairDev pr = pairs[r];
    const int L = pr.cls;
    const int NT = nterms(L);
    const long long cnt = lay.start[L + 1] - lay.start[L], loc = r - lay.start[L];
    double F[3];
    centre_frac(pr, cc, F);
    const double p = pr.p, rs = sqrt(kGaussCut / p), pref = pow(p / M_PI, 1.5);
    const double* Vd = V + (long long)d * npts;
    double J[kMaxTerms], H[kMaxTerms];
    for (int t = 0; t < NT; ++t) J[t] = 0.0;
    for (long long m = 0; m < npts; ++m) {
        const int m1 = (int)(m / ((long long)N1 * N2)), m2 = (int)((m / N2) % N1), m3 = (int)(m % N2);
        const double f[3] = {(double)m1 / N0, (double)m2 / N1, (double)m3 / N2};
        const double v = __ldg(Vd + m);
        int tlo[3], thi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double s0 = f[a] - F[a], reach = rs * lat.bn[a];
            tlo[a] = (int)ceil(s0 - reach);
            thi[a] = (int)floor(s0 + reach);
        }
        for (int t1 = tlo[0]; t1 <= thi[0]; ++t1)
            for (int t2 = tlo[1]; t2 <= thi[1]; ++t2)
                for (int t3 = tlo[2]; t3 <= thi[2]; ++t3) {
                    const double s[3] = {f[0] - F[0] - t1, f[1] - F[1] - t2, f[2] - F[2] - t3};
                    double q = 0.0;
#pragma unroll
                    for (int x = 0; x < 3; ++x)
#pragma unroll
                        for (int y = 0; y < 3; ++y) q += lat.g[3 * x + y] * s[x] * s[y];
                    if (p * q > kGaussCut) continue;
                    const double ev = pref * exp(-p * q) * v;
                    hermite_metric(L, p, lat.g, s, H);
                    double sc = 1.0;
                    int t = 0;
                    for (int lam = 0; lam <= L; ++lam, sc *= 1.0 / (2.0 * M_PI))
                        for (int i = 0; i < nmono(lam); ++i, ++t) J[t] = fma(sc * H[t], ev, J[t]);
                }
    }
    for (int t = 0; t < NT; ++t) Jp[(long long)d * lay.total + lay.base[L] + (long long)t * cnt + loc] = J[t];
}

DdLayout dd_layout(const ftcj_plan* D) {
    DdLayout l;
    for (int c = 0; c <= kNclass; ++c) l.start[c] = D->class_start[c];
    for (int c = 0; c < kNclass; ++c) l.base[c] = D->term_base[c];
    l.total = D->total_terms;
    return l;
}

Lattice lattice_of(const ftcj_plan* P) {
    Lattice lat;
    for (int i = 0; i < 9; ++i) lat.A[i] = P->A[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            lat.g[3 * i + j] = P->A[3 * i] * P->A[3 * j] + P->A[3 * i + 1] * P->A[3 * j + 1] + P->A[3 * i + 2] * P->A[3 * j + 2];
    for (int i = 0; i < 3; ++i) lat.bn[i] = std::sqrt(P->M[4 * i]) / (2.0 * M_PI);
    return lat;
}

}  // namespace

namespace {

template <class T>
int galloc(ftcj_plan* P, Gpw* g, T** ptr, size_t count) {
    if (count == 0) count = 1;
    const size_t bytes = sizeof(T) * count;
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(FTCJ_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) +
                                     " bytes for the GPW grid failed: " + cudaGetErrorString(e));
    }
    g->bytes += bytes;
    P->device_bytes += bytes;
    return FTCJ_OK;
}

// the DD records' plan: the same cell, basis and sphere, FP64 maps, only the
// records whose two primitives are diffuse
int make_dd_plan(ftcj_plan* P, ftcj_plan* D) {
    for (int i = 0; i < 9; ++i) {
        D->A[i] = P->A[i];
        D->B[i] = P->B[i];
        D->M[i] = P->M[i];
    }
    D->vol = P->vol;
    D->omega = P->omega;
    D->gcut = P->gcut;
    for (int i = 0; i < 3; ++i) D->km[i] = P->km[i];
    D->nk = P->nk;
    D->params = P->params;
    D->params.pair_gcut_eps = 0.0;
    D->params.precision = FTCJ_PREC_FP64;
    D->params.contraction = FTCJ_CONTRACT_WALK;
    D->params.shard_count = 1;
    D->params.shard_index = 0;
    D->precision = FTCJ_PREC_FP64;
    D->max_dens = P->max_dens;
    D->nao = P->nao;
    D->nshell = P->nshell;
    D->ngroup = P->ngroup;
    D->nmember = P->nmember;
    D->ncentre = P->ncentre;
    D->groups = P->groups;
    D->members = P->members;
    D->member_shell = P->member_shell;
    D->member_prim = P->member_prim;
    D->member_group = P->member_group;
    D->num_sms = P->num_sms;
    D->cc = P->cc;
    D->ortho = P->ortho;
    D->rec_filter = 2;
    D->alpha_cut = P->alpha_cut;
    D->jp_fixed = 1;
    FTCJ_CUDA(cudaMalloc(&D->d_groups, sizeof(GroupDev) * D->groups.size()));
    FTCJ_CUDA(cudaMemcpy(D->d_groups, D->groups.data(), sizeof(GroupDev) * D->groups.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaMalloc(&D->d_members, sizeof(MemberDev) * D->members.size()));
    FTCJ_CUDA(cudaMemcpy(D->d_members, D->members.data(), sizeof(MemberDev) * D->members.size(),
                         cudaMemcpyHostToDevice));
    D->device_bytes += sizeof(GroupDev) * D->groups.size() + sizeof(MemberDev) * D->members.size();
    int rc = screen_and_sort(D);
    if (rc) return rc;
    D->total_terms = 0;
    for (int c = 0; c < kNclass; ++c) {
        D->term_base[c] = D->total_terms;
        D->total_terms += (D->class_start[c + 1] - D->class_start[c]) * nterms(c);
    }
    if (D->npairs == 0) return FTCJ_OK;
    if ((rc = upload_hermite_tables(D))) return rc;
    if ((rc = build_maps(D))) return rc;
    const size_t terms = (size_t)D->max_dens * (size_t)D->total_terms;
    FTCJ_CUDA(cudaMalloc(&D->d_Dp, sizeof(double) * terms));
    FTCJ_CUDA(cudaMalloc(&D->d_Jp, sizeof(double) * terms));
    D->device_bytes += 2 * sizeof(double) * terms;
    return FTCJ_OK;
}

}  // namespace

int setup_gpw(ftcj_plan* P) {
    ftcj_plan* D = new (std::nothrow) ftcj_plan();
    if (!D) return fail(FTCJ_ENOMEM, "host allocation failed");
    P->dd = D;  // released with P, also on failure
    int rc = make_dd_plan(P, D);
    if (rc) return rc;
    P->device_bytes += D->device_bytes;
    if (D->npairs == 0) return FTCJ_OK;  // nothing diffuse: the plain long-range build

    Gpw* g = new (std::nothrow) Gpw();
    if (!g) return fail(FTCJ_ENOMEM, "host allocation failed");
    P->gpw = g;
    // the half sphere's index ranges
    int nmax[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int64_t p = 0; p < P->ng_half; ++p)
        for (int a = 0; a < 3; ++a) {
            const int v = P->gvec[3 * p + a];
            nmax[a] = std::max(nmax[a], std::abs(v));
            lo[a] = std::min(lo[a], v);
            hi[a] = std::max(hi[a], v);
        }
    // the grid: every alias of a DD transform below e^{-46} on the sphere
    double amax = 0.0;
    for (const GroupDev& gr : P->groups)
        if (gr.alpha < P->alpha_cut) amax = std::max(amax, gr.alpha);
    const double reach = P->gcut + std::sqrt(184.0 * 2.0 * amax);
    for (int a = 0; a < 3; ++a) {
        const double an = std::sqrt(P->A[3 * a] * P->A[3 * a] + P->A[3 * a + 1] * P->A[3 * a + 1] +
                                    P->A[3 * a + 2] * P->A[3 * a + 2]);
        const int need = 2 * nmax[a] + 1;
        int n = P->params.gpw_grid[a];
        if (n > 0) {
            if (n < need) return fail(FTCJ_EINVAL, "gpw_grid below 2 max|n_i| + 1 along an axis: sphere points alias");
        } else {
            n = std::max(need, (int)std::ceil(reach * an / (2.0 * M_PI)));
        }
        if (n > 4096) return fail(FTCJ_EUNSUPPORTED, "GPW grid above 4096 points along an axis");
        g->N[a] = n;
        g->nlo[a] = lo[a];
        g->ncnt[a] = std::max(1, hi[a] - lo[a] + 1);
    }
    g->npts = (long long)g->N[0] * g->N[1] * g->N[2];
    g->gnorm = P->vol / (double)g->npts;
    g->sep = P->ortho;
    g->df = g->sep && P->precision == FTCJ_PREC_SPLIT;
    if (g->df) {
        g->vplane_bytes = sizeof(float2) * (size_t)g->N[0] * g->N[2];
        const void* kerns[] = {(const void*)k_gpw_integrate_sep_df<0>, (const void*)k_gpw_integrate_sep_df<1>,
                               (const void*)k_gpw_integrate_sep_df<2>, (const void*)k_gpw_integrate_sep_df<3>,
                               (const void*)k_gpw_integrate_sep_df<4>};
        for (const void* k : kerns)
            if ((rc = allow_dynamic_smem(k, g->vplane_bytes))) return rc;
    }
    g->lmax = 0;
    for (int c = 0; c < kNclass; ++c)
        if (D->class_start[c + 1] > D->class_start[c]) g->lmax = c;
    const long long nrec = D->npairs;
    const int md = P->max_dens;
    // record splits: about four blocks per SM, at least 8 records a split,
    // partial grids within 1 GB
    const long long lines = (long long)g->N[1] * g->N[2];
    const long long blocks = g->sep ? (lines + kGpwThreads - 1) / kGpwThreads : (g->npts + kGpwThreads - 1) / kGpwThreads;
    long long ns = (4LL * P->num_sms + blocks * md - 1) / (blocks * md);
    ns = std::min<long long>(ns, std::max<long long>(1, nrec / 8));
    ns = std::min<long long>(ns, std::max<long long>(1, (1LL << 27) / ((long long)md * g->npts)));
    g->nsplit = (int)std::max<long long>(1, std::min<long long>(ns, 65535));
    if (g->sep) {
        g->tstride = (long long)(g->lmax + 1) * (g->N[0] + g->N[1] + g->N[2]);
        if ((rc = galloc(P, g, &g->d_tab, (size_t)(g->tstride * nrec)))) return rc;
        if (g->df && (rc = galloc(P, g, &g->d_tabf, (size_t)(g->tstride * nrec)))) return rc;
        if (g->df && (rc = galloc(P, g, &g->d_tabfr, (size_t)(g->tstride * nrec)))) return rc;
        const long long nt = nrec * (g->N[0] + g->N[1] + g->N[2]);
        k_gpw_tables<<<(unsigned)((nt + 255) / 256), 256>>>(D->d_pairs, nrec, g->lmax, g->N[0], g->N[1], g->N[2],
                                                            lattice_of(P), P->cc, g->d_tab, g->d_tabf, g->d_tabfr);
        FTCJ_CUDA(cudaGetLastError());
    }
    if (g->sep) {
        // row splits of the integration: about four blocks per SM
        const long long rb = (nrec + kGpwThreads - 1) / kGpwThreads;
        g->nsj = (int)std::max<long long>(1, std::min<long long>(g->N[1], (4LL * P->num_sms + rb * md - 1) / (rb * md)));
        if ((rc = galloc(P, g, &g->d_jpart, (size_t)g->nsj * md * D->total_terms))) return rc;
    }
    if ((rc = galloc(P, g, &g->d_tw, (size_t)(g->N[0] + g->N[1] + g->N[2])))) return rc;
    k_gpw_twiddles<<<(unsigned)((g->N[0] + g->N[1] + g->N[2] + 255) / 256), 256>>>(g->N[0], g->N[1], g->N[2], g->d_tw);
    FTCJ_CUDA(cudaGetLastError());
    if ((rc = galloc(P, g, &g->d_part, (size_t)g->nsplit * md * g->npts))) return rc;
    if ((rc = galloc(P, g, &g->d_grid, (size_t)md * g->npts))) return rc;
    if (g->df && (rc = galloc(P, g, &g->d_vf, (size_t)md * g->npts))) return rc;
    if ((rc = galloc(P, g, &g->d_t1, (size_t)md * g->ncnt[0] * lines))) return rc;
    if ((rc = galloc(P, g, &g->d_t2, (size_t)md * g->ncnt[0] * g->ncnt[1] * g->N[2]))) return rc;
    if ((rc = galloc(P, g, &g->d_rhoD, (size_t)md * P->ng_half))) return rc;
    if ((rc = galloc(P, g, &g->d_WD, (size_t)md * P->ng_half))) return rc;
    if ((rc = galloc(P, g, &g->d_vfr, (size_t)P->ng_half))) return rc;
    g->nEb = (int)std::max<int64_t>(1, (P->ng_half + 255) / 256);
    if ((rc = galloc(P, g, &g->d_Epart, (size_t)md * g->nEb))) return rc;
    if (P->ng_half > 0) {
        k_gpw_vfr<<<(unsigned)((P->ng_half + 255) / 256), 256>>>(P->d_gvec, P->ng_half, P->cc, g->d_vfr);
        FTCJ_CUDA(cudaGetLastError());
    }
    // the half sphere's points grouped by (n1, n2), for the adjoint of pass 3
    const long long ncell = (long long)g->ncnt[0] * g->ncnt[1];
    std::vector<int> cstart((size_t)ncell + 1, 0), clist((size_t)std::max<int64_t>(1, P->ng_half));
    for (int64_t p = 0; p < P->ng_half; ++p)
        ++cstart[(size_t)(P->gvec[3 * p] - g->nlo[0]) * g->ncnt[1] + (P->gvec[3 * p + 1] - g->nlo[1]) + 1];
    for (long long c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t p = 0; p < P->ng_half; ++p)
            clist[fill[(size_t)(P->gvec[3 * p] - g->nlo[0]) * g->ncnt[1] + (P->gvec[3 * p + 1] - g->nlo[1])]++] = (int)p;
    }
    if ((rc = galloc(P, g, &g->d_cstart, cstart.size()))) return rc;
    if ((rc = galloc(P, g, &g->d_clist, clist.size()))) return rc;
    FTCJ_CUDA(cudaMemcpy(g->d_cstart, cstart.data(), sizeof(int) * cstart.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaMemcpy(g->d_clist, clist.data(), sizeof(int) * clist.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaDeviceSynchronize());
    return FTCJ_OK;
}

void free_gpw(ftcj_plan* P) {
    Gpw* g = P->gpw;
    if (!g) return;
    void* ptrs[] = {g->d_tab, g->d_tabf, g->d_tabfr, g->d_vf, g->d_tw, g->d_jpart, g->d_part, g->d_grid, g->d_t1, g->d_t2, g->d_rhoD, g->d_WD, g->d_vfr, g->d_Epart,
                    g->d_cstart, g->d_clist};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete g;
    P->gpw = nullptr;
}

int launch_gpw_rho(ftcj_plan* P, int nd, cudaStream_t s) {
    Gpw* g = P->gpw;
    const ftcj_plan* D = P->dd;
    if (!g || P->ng_half == 0) return FTCJ_OK;
    const DdLayout lay = dd_layout(D);
    const long long lines = (long long)g->N[1] * g->N[2];
    if (g->sep) {
        dim3 grid((unsigned)((lines + kGpwThreads - 1) / kGpwThreads), g->nsplit, nd);
        bool add = false;
        for (int c = 0; c < kNclass; ++c) {
            if (D->class_start[c + 1] == D->class_start[c]) continue;
            if (g->df) {
                auto kern = c == 0 ? k_gpw_collocate_sep_df<0>
                          : c == 1 ? k_gpw_collocate_sep_df<1>
                          : c == 2 ? k_gpw_collocate_sep_df<2>
                          : c == 3 ? k_gpw_collocate_sep_df<3>
                                   : k_gpw_collocate_sep_df<4>;
                kern<<<grid, kGpwThreads, 0, s>>>(g->d_tabfr, D->npairs, g->lmax, g->N[0], g->N[1], g->N[2], D->d_Dp,
                                                  lay, g->nsplit, nd, g->npts, add, g->d_part);
            } else {
                auto kern = c == 0 ? k_gpw_collocate_sep<0>
                          : c == 1 ? k_gpw_collocate_sep<1>
                          : c == 2 ? k_gpw_collocate_sep<2>
                          : c == 3 ? k_gpw_collocate_sep<3>
                                   : k_gpw_collocate_sep<4>;
                kern<<<grid, kGpwThreads, 0, s>>>(g->d_tab, D->npairs, g->lmax, g->N[0], g->N[1], g->N[2], D->d_Dp,
                                                  lay, g->nsplit, nd, g->npts, add, g->d_part);
            }
            FTCJ_CUDA(cudaGetLastError());
            add = true;
        }
    } else {
        dim3 grid((unsigned)((g->npts + kGpwThreads - 1) / kGpwThreads), g->nsplit, nd);
        k_gpw_collocate_gen<<<grid, kGpwThreads, 0, s>>>(D->d_pairs, D->npairs, g->N[0], g->N[1], g->N[2], D->d_Dp,
                                                        lay, lattice_of(P), P->cc, g->nsplit, nd, g->npts, g->d_part);
    }
    FTCJ_CUDA(cudaGetLastError());
    k_gpw_reduce<<<dim3((unsigned)((g->npts + 255) / 256), nd), 256, 0, s>>>(g->d_part, g->nsplit, nd, g->npts,
                                                                           g->d_grid);
    FTCJ_CUDA(cudaGetLastError());
    const long long n1 = (long long)g->ncnt[0] * lines;
    k_gpw_dft1<<<dim3((unsigned)((n1 + 255) / 256), nd), 256, 0, s>>>(g->d_grid, g->d_tw, g->N[0], g->N[1], g->N[2],
                                                                    g->nlo[0], g->ncnt[0], g->npts, g->d_t1);
    FTCJ_CUDA(cudaGetLastError());
    const long long n2 = (long long)g->ncnt[0] * g->ncnt[1] * g->N[2];
    k_gpw_dft2<<<dim3((unsigned)((n2 + 255) / 256), nd), 256, 0, s>>>(g->d_t1, g->d_tw + g->N[0], g->N[1], g->N[2],
                                                                    g->ncnt[0], g->nlo[1], g->ncnt[1], g->d_t2);
    FTCJ_CUDA(cudaGetLastError());
    k_gpw_dft3<<<dim3((unsigned)((P->ng_half + 255) / 256), nd), 256, 0, s>>>(
        g->d_t2, g->d_tw + g->N[0] + g->N[1], P->d_gvec, P->ng_half, g->N[2], g->nlo[0], g->ncnt[0], g->nlo[1],
        g->ncnt[1], g->gnorm, g->d_rhoD);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_gpw_potential(ftcj_plan* P, int nd, double* EJ, cudaStream_t s) {
    Gpw* g = P->gpw;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(EJ, 0, sizeof(double) * nd, s));
        return FTCJ_OK;
    }
    k_gpw_potential<<<dim3(g->nEb, nd), 256, 0, s>>>(reinterpret_cast<const double2*>(P->d_rho), g->d_rhoD, P->d_vg,
                                                   g->d_vfr, P->ng_half, reinterpret_cast<double2*>(P->d_W), g->d_WD,
                                                   g->d_Epart, g->nEb);
    FTCJ_CUDA(cudaGetLastError());
    k_gpw_energy<<<nd, 256, 0, s>>>(g->d_Epart, g->nEb, EJ);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_gpw_j(ftcj_plan* P, int nd, cudaStream_t s) {
    Gpw* g = P->gpw;
    ftcj_plan* D = P->dd;
    if (!g) return FTCJ_OK;
    if (P->ng_half == 0) {
        FTCJ_CUDA(cudaMemsetAsync(D->d_Jp, 0, sizeof(double) * (size_t)nd * D->total_terms, s));
        return FTCJ_OK;
    }
    const long long lines = (long long)g->N[1] * g->N[2];
    const long long n2 = (long long)g->ncnt[0] * g->ncnt[1] * g->N[2];
    k_gpw_adj3<<<dim3((unsigned)((n2 + 255) / 256), nd), 256, 0, s>>>(g->d_WD, g->d_tw + g->N[0] + g->N[1], P->d_gvec,
                                                                    P->ng_half, g->d_cstart, g->d_clist, g->N[2],
                                                                    g->ncnt[0], g->ncnt[1], g->d_t2);
    FTCJ_CUDA(cudaGetLastError());
    const long long n1 = (long long)g->ncnt[0] * lines;
    k_gpw_adj2<<<dim3((unsigned)((n1 + 255) / 256), nd), 256, 0, s>>>(g->d_t2, g->d_tw + g->N[0], g->N[1], g->N[2],
                                                                    g->ncnt[0], g->nlo[1], g->ncnt[1], g->d_t1);
    FTCJ_CUDA(cudaGetLastError());
    k_gpw_adj1<<<dim3((unsigned)((g->npts + 255) / 256), nd), 256, 0, s>>>(g->d_t1, g->d_tw, g->N[0], g->N[1], g->N[2],
                                                                         g->nlo[0], g->ncnt[0], g->npts, g->gnorm,
                                                                         g->d_grid, g->d_vf);
    FTCJ_CUDA(cudaGetLastError());
    const DdLayout lay = dd_layout(D);
    if (g->sep) {
        for (int c = 0; c < kNclass; ++c) {
            const long long cnt = D->class_start[c + 1] - D->class_start[c];
            if (cnt == 0) continue;
            dim3 grid((unsigned)((cnt + kGpwThreads - 1) / kGpwThreads), nd, g->nsj);
            if (g->df) {
                auto kern = c == 0 ? k_gpw_integrate_sep_df<0>
                          : c == 1 ? k_gpw_integrate_sep_df<1>
                          : c == 2 ? k_gpw_integrate_sep_df<2>
                          : c == 3 ? k_gpw_integrate_sep_df<3>
                                   : k_gpw_integrate_sep_df<4>;
                kern<<<grid, kGpwThreads, g->vplane_bytes, s>>>(g->d_tabf, D->npairs, g->lmax, g->N[0], g->N[1],
                                                                g->N[2], lay, g->d_vf, g->npts, g->d_jpart);
            } else {
                auto kern = c == 0 ? k_gpw_integrate_sep<0>
                          : c == 1 ? k_gpw_integrate_sep<1>
                          : c == 2 ? k_gpw_integrate_sep<2>
                          : c == 3 ? k_gpw_integrate_sep<3>
                                   : k_gpw_integrate_sep<4>;
                kern<<<grid, kGpwThreads, 0, s>>>(g->d_tab, D->npairs, g->lmax, g->N[0], g->N[1], g->N[2], lay,
                                                  g->d_grid, g->npts, g->d_jpart);
            }
            FTCJ_CUDA(cudaGetLastError());
        }
        k_gpw_jsum<<<dim3((unsigned)((D->total_terms + 255) / 256), nd), 256, 0, s>>>(g->d_jpart, g->nsj, nd,
                                                                                      D->total_terms, D->d_Jp);
        FTCJ_CUDA(cudaGetLastError());
    } else {
        dim3 grid((unsigned)((D->npairs + kGpwThreads - 1) / kGpwThreads), nd);
        k_gpw_integrate_gen<<<grid, kGpwThreads, 0, s>>>(D->d_pairs, D->npairs, g->N[0], g->N[1], g->N[2], lay,
                                                        lattice_of(P), P->cc, g->d_grid, g->npts, D->d_Jp);
        FTCJ_CUDA(cudaGetLastError());
    }
    return FTCJ_OK;
}

int gpw_grid_dim(const ftcj_plan* P, int axis) { return P->gpw ? P->gpw->N[axis] : 0; }
int gpw_separable(const ftcj_plan* P) { return P->gpw && P->gpw->sep ? (P->gpw->df ? 2 : 1) : 0; }

int gpw_launches(const ftcj_plan* P, int nd) {
    (void)nd;
    const Gpw* g = P->gpw;
    if (!g || P->ng_half == 0) return 0;
    int integ = 0;
    if (g->sep) {
        for (int c = 0; c < kNclass; ++c) integ += P->dd->class_start[c + 1] > P->dd->class_start[c] ? 1 : 0;
    } else {
        integ = 1;
    }
    // collocation and integration (per class present in the separable form,
    // whose integration adds the sum of its row splits), reduction, three
    // passes, potential and energy, three adjoint passes, and the DD records'
    // a3 and a7 maps
    return integ + 1 + 3 + 2 + 3 + integ + (g->sep ? 1 : 0) + 2;
}

}  // namespace ftcj
