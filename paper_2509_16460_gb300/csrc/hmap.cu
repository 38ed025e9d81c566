// Per-record linear maps of Alg. 2 / Alg. S2, built once per plan.
//
// For a pair record and one (shell of group a, shell of group b) member pair,
// everything between the AO density block and the relative-coordinate Hermite
// densities is geometry only: the shells' coefficients and normalisation, the
// solid-harmonic (or Cartesian) components, the McMurchie-Davidson E
// coefficients of the Gaussian product, the expansion of Cartesian powers of G
// in n1^i n2^j n3^k, and the prefactor exp(-mu R^2)(pi/p)^{3/2}.  It is stored
// as M[f][q][term] (f over the a functions, q over the b functions, term over
// the record's D'_ijk, fastest), so that per build
//   D'_term = sum_{f,q} M[term][f][q] (D^{0[L]}_{fq} + D^{0[-L]}_{qf})      (a3)
//   J^{0[L]}_{fq} (and J^{0[-L]}_{qf}) += sum_term M[term][f][q] J'_term    (a7)
// are small dense products.  Each is spread over threads: one per (record,
// term) for a3 and one per (record, output element) for a7, so neighbouring
// threads read neighbouring map entries and share the record's density block
// (or J' terms) through broadcast loads.
#include <algorithm>
#include <cmath>
#include <vector>

#include "df.cuh"
#include "ftcj_internal.h"

namespace ftcj {
namespace {

__device__ __forceinline__ int nfunc_d(int l, int sph) { return sph ? 2 * l + 1 : (l + 1) * (l + 2) / 2; }

__device__ void ecoef_m(double PA, double PB, double a2p, int la, int lb, double E[3][3][5]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int t = 0; t < 5; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 1; i <= la; ++i)
        for (int t = 0; t <= i; ++t)
            E[i][0][t] = (t > 0 ? a2p * E[i - 1][0][t - 1] : 0.0) + PA * E[i - 1][0][t] +
                         (t + 1) * E[i - 1][0][t + 1];
    for (int i = 0; i <= la; ++i)
        for (int j = 1; j <= lb; ++j)
            for (int t = 0; t <= i + j; ++t)
                E[i][j][t] = (t > 0 ? a2p * E[i][j - 1][t - 1] : 0.0) + PB * E[i][j - 1][t] +
                             (t + 1 <= 4 ? (t + 1) * E[i][j - 1][t + 1] : 0.0);
}

__global__ void k_map_build(const PairDev* __restrict__ pairs, const GroupDev* __restrict__ G,
                            const MemberDev* __restrict__ mem, const long long* __restrict__ moff, long long npairs,
                            const double* __restrict__ Tm, const int* __restrict__ Toff, const double* __restrict__ Ut,
                            const int* __restrict__ cart, double* __restrict__ maps, CellConst cc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    const PairDev pr = pairs[i];
    const GroupDev A = G[pr.ga];
    const GroupDev B = G[pr.gb];
    double E[3][3][3][5];
    {
        const double Av[3] = {A.x, A.y, A.z};
        const double Bv[3] = {B.x, B.y, B.z};
        const double a2p = 0.5 / pr.p;
        for (int x = 0; x < 3; ++x) {
            const double Bs = Bv[x] + pr.L[0] * cc.A[x] + pr.L[1] * cc.A[3 + x] + pr.L[2] * cc.A[6 + x];
            ecoef_m(pr.P[x] - Av[x], pr.P[x] - Bs, a2p, A.lmax, B.lmax, E[x]);
        }
    }
    const int Lc = pr.cls;
    double* out = maps + moff[i];
    for (int ia = A.mem0; ia < A.mem1; ++ia) {
        const MemberDev ma = mem[ia];
        const int nfa = nfunc_d(ma.l, ma.sph), nca = (ma.l + 1) * (ma.l + 2) / 2;
        const double* Ua = Ut + ((ma.l * 2 + ma.sph) * kNcartMax) * kNcartMax;
        for (int ib = B.mem0; ib < B.mem1; ++ib) {
            const MemberDev mb = mem[ib];
            const int nfb = nfunc_d(mb.l, mb.sph), ncb = (mb.l + 1) * (mb.l + 2) / 2;
            const double* Ub = Ut + ((mb.l * 2 + mb.sph) * kNcartMax) * kNcartMax;
            const double scale = ma.coef * mb.coef * pr.K;
            int term = 0;
            for (int lam = 0; lam <= Lc; ++lam) {
                const int nm = nmono(lam);
                const double* T = Tm + Toff[lam];
                for (int b = 0; b < nm; ++b, ++term) {
                    // g[ca][cb] = sum_{tuv of degree lam} T[tuv][b] E^x_t E^y_u E^z_v
                    double g[kNcartMax][kNcartMax];
                    for (int ca = 0; ca < nca; ++ca) {
                        const int* xa = cart + (ma.l * kNcartMax + ca) * 3;
                        for (int cb = 0; cb < ncb; ++cb) {
                            const int* xb = cart + (mb.l * kNcartMax + cb) * 3;
                            double s = 0.0;
                            for (int t = 0; t <= xa[0] + xb[0] && t <= lam; ++t)
                                for (int u = 0; u <= xa[1] + xb[1] && t + u <= lam; ++u) {
                                    const int v = lam - t - u;
                                    if (v > xa[2] + xb[2]) continue;
                                    s += T[mono_index(lam, t, u) * nm + b] * E[0][xa[0]][xb[0]][t] *
                                         E[1][xa[1]][xb[1]][u] * E[2][xa[2]][xb[2]][v];
                                }
                            g[ca][cb] = s;
                        }
                    }
                    for (int f = 0; f < nfa; ++f)
                        for (int q = 0; q < nfb; ++q) {
                            double s = 0.0;
                            for (int ca = 0; ca < nca; ++ca) {
                                const double ua = Ua[f * kNcartMax + ca];
                                if (ua == 0.0) continue;
                                for (int cb = 0; cb < ncb; ++cb) s += ua * Ub[q * kNcartMax + cb] * g[ca][cb];
                            }
                            out[((long long)f * nfb + q) * nterms(Lc) + term] = scale * s;
                        }
                }
            }
            out += (long long)nterms(Lc) * nfa * nfb;
        }
    }
}

// thread index -> (class, record, slot) over the flattened per-class ranges
__device__ __forceinline__ bool locate(const MapThreads& mt, long long gid, int& cls, long long& rec, int& slot) {
    for (int c = 0; c < kNclass; ++c) {
        if (gid < mt.tstart[c + 1]) {
            if (mt.slots[c] == 0) return false;
            const long long loc = gid - mt.tstart[c];
            cls = c;
            rec = mt.rstart[c] + loc / mt.slots[c];
            slot = (int)(loc % mt.slots[c]);
            return true;
        }
    }
    return false;
}

// a3: one thread per (record, term): D'_term = sum over member pairs, f, q of
// M[f][q][term] times the combined density element
template <bool OUT_DF>
__global__ void __launch_bounds__(256) k_hermite_map(const PairDev* __restrict__ pairs,
                                                     const GroupDev* __restrict__ G,
                                                     const MemberDev* __restrict__ mem,
                                                     const long long* __restrict__ moff,
                                                     const double* __restrict__ maps, const double* __restrict__ D0n,
                                                     int nao, int nk, MapLayout lay, MapThreads mt,
                                                     double* __restrict__ Dp) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    int L, t;
    long long i;
    if (!locate(mt, gid, L, i, t)) return;
    const PairDev pr = pairs[i];
    const GroupDev A = G[pr.ga];
    const GroupDev B = G[pr.gb];
    const int NT = nterms(L);
    const long long nn = (long long)nao * nao;
    const double* Dc = D0n + ((long long)d * nk + pr.cell) * nn;
    const double* Dm = D0n + ((long long)d * nk + pr.mcell) * nn;
    const double* M = maps + moff[i];
    double acc = 0.0;
    for (int ia = A.mem0; ia < A.mem1; ++ia) {
        const MemberDev ma = mem[ia];
        const int nfa = nfunc_d(ma.l, ma.sph);
        for (int ib = B.mem0; ib < B.mem1; ++ib) {
            const MemberDev mb = mem[ib];
            const int nfb = nfunc_d(mb.l, mb.sph);
            for (int f = 0; f < nfa; ++f) {
                const double* drow = Dc + (long long)(ma.ao + f) * nao + mb.ao;
                for (int q = 0; q < nfb; ++q) {
                    double dv = __ldg(drow + q);
                    if (pr.weight == 2) dv += __ldg(Dm + (long long)(mb.ao + q) * nao + ma.ao + f);
                    acc = fma(__ldg(M + ((long long)f * nfb + q) * NT + t), dv, acc);
                }
            }
            M += (long long)NT * nfa * nfb;
        }
    }
    const long long off = (long long)d * lay.total + lay.base[L] + (i - lay.start[L]) +
                          (long long)t * (lay.start[L + 1] - lay.start[L]);
    if (OUT_DF) {
        const float hi = (float)acc;
        reinterpret_cast<float2*>(Dp)[off] = make_float2(hi, (float)(acc - (double)hi));
    } else {
        Dp[off] = acc;
    }
}

// a7: one thread per (record, output element of its member pairs):
// J_fq = sum_term M[f][q][term] J'_term (J' summed over the walk chunks),
// scattered into J^{0[L]} and, for a mirrored record, J^{0[-L]}
__global__ void __launch_bounds__(256) k_jtransform_map(const PairDev* __restrict__ pairs,
                                                        const GroupDev* __restrict__ G,
                                                        const MemberDev* __restrict__ mem,
                                                        const long long* __restrict__ moff,
                                                        const double* __restrict__ maps,
                                                        const double* __restrict__ Jp, int nchunks, int nao, int nk,
                                                        MapLayout lay, MapThreads mt, double* __restrict__ J0n) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    int L, slot;
    long long i;
    if (!locate(mt, gid, L, i, slot)) return;
    const PairDev pr = pairs[i];
    const GroupDev A = G[pr.ga];
    const GroupDev B = G[pr.gb];
    const int NT = nterms(L);
    // find this thread's (member pair, f, q)
    const double* M = maps + moff[i];
    int ia = A.mem0, ib = B.mem0, nfa = 0, nfb = 0;
    bool found = false;
    for (ia = A.mem0; ia < A.mem1 && !found; ++ia) {
        nfa = nfunc_d(mem[ia].l, mem[ia].sph);
        for (ib = B.mem0; ib < B.mem1; ++ib) {
            nfb = nfunc_d(mem[ib].l, mem[ib].sph);
            if (slot < nfa * nfb) {
                found = true;
                break;
            }
            slot -= nfa * nfb;
            M += (long long)NT * nfa * nfb;
        }
        if (found) break;
    }
    if (!found) return;  // a slot beyond this record's outputs
    const MemberDev ma = mem[ia], mb = mem[ib];
    const int f = slot / nfb, q = slot % nfb;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long loc = i - lay.start[L];
    const double* Mfq = M + ((long long)f * nfb + q) * NT;
    double s = 0.0;
    for (int t = 0; t < NT; ++t) {
        double jt = 0.0;
        for (int c = 0; c < nchunks; ++c)
            jt += __ldg(Jp + ((long long)d * nchunks + c) * lay.total + lay.base[L] + (long long)t * cnt + loc);
        s = fma(__ldg(Mfq + t), jt, s);
    }
    const long long nn = (long long)nao * nao;
    atomicAdd(J0n + ((long long)d * nk + pr.cell) * nn + (long long)(ma.ao + f) * nao + mb.ao + q, s);
    if (pr.weight == 2)
        atomicAdd(J0n + ((long long)d * nk + pr.mcell) * nn + (long long)(mb.ao + q) * nao + ma.ao + f, s);
}

// ---- split form: double-float maps, record-major blocks --------------------
// A block holds whole records of one class.  a3 stages each record's combined
// density elements (D^{0[L]}_{fq} + D^{0[-L]}_{qf}, split into double-float)
// once in shared memory and gives every term its own thread; a7 stages each
// record's J'_t (summed over the walk chunks) and gives every output element
// its own thread.  Arithmetic in double-float on the FP32 pipe.

// AO row and column of element e of a record (member pairs in order, then f, q)
__device__ __forceinline__ bool entry_ao(const GroupDev& A, const GroupDev& B, const MemberDev* __restrict__ mem,
                                         int e, int& row, int& col) {
    for (int ia = A.mem0; ia < A.mem1; ++ia) {
        const MemberDev ma = mem[ia];
        const int nfa = nfunc_d(ma.l, ma.sph);
        for (int ib = B.mem0; ib < B.mem1; ++ib) {
            const MemberDev mb = mem[ib];
            const int nfb = nfunc_d(mb.l, mb.sph);
            if (e < nfa * nfb) {
                row = ma.ao + e / nfb;
                col = mb.ao + e % nfb;
                return true;
            }
            e -= nfa * nfb;
        }
    }
    return false;
}

__device__ __forceinline__ int entries_of(const GroupDev& A, const GroupDev& B, const MemberDev* __restrict__ mem) {
    int n = 0;
    for (int ia = A.mem0; ia < A.mem1; ++ia)
        for (int ib = B.mem0; ib < B.mem1; ++ib)
            n += nfunc_d(mem[ia].l, mem[ia].sph) * nfunc_d(mem[ib].l, mem[ib].sph);
    return n;
}

__device__ __forceinline__ int block_class(const RecBlocks& rb) {
    int c = 0;
    while (c < kNclass - 1 && (int)blockIdx.x >= rb.bstart[c + 1]) ++c;
    return c;
}

__global__ void __launch_bounds__(256) k_hermite_map_df(const PairDev* __restrict__ pairs,
                                                        const GroupDev* __restrict__ G,
                                                        const MemberDev* __restrict__ mem,
                                                        const long long* __restrict__ moff,
                                                        const float2* __restrict__ maps,
                                                        const double* __restrict__ D0n, int nao, int nk,
                                                        MapLayout lay, RecBlocks rb, TermDest dst,
                                                        float2* __restrict__ Dp) {
    extern __shared__ float2 stage[];
    const int d = blockIdx.y;
    const int c = block_class(rb);
    const int NT = nterms(c), E = rb.stage[c], R = rb.per[c];
    const long long r0 = rb.rstart[c] + (long long)(blockIdx.x - rb.bstart[c]) * R;
    const long long rend = rb.rstart[c] + rb.rcount[c];
    const long long nn = (long long)nao * nao;
    for (int idx = threadIdx.x; idx < R * E; idx += blockDim.x) {
        const long long i = r0 + idx / E;
        df v{0.f, 0.f};
        int row, col;
        if (i < rend) {
            const PairDev pr = pairs[i];
            if (entry_ao(G[pr.ga], G[pr.gb], mem, idx % E, row, col)) {
                v = split_double(__ldg(D0n + ((long long)d * nk + pr.cell) * nn + (long long)row * nao + col));
                if (pr.weight == 2)
                    v = df_add(v, split_double(__ldg(D0n + ((long long)d * nk + pr.mcell) * nn +
                                                     (long long)col * nao + row)));
            }
        }
        stage[idx] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    const int r = threadIdx.x / NT, t = threadIdx.x % NT;
    const long long i = r0 + r;
    if (r >= R || i >= rend) return;
    const PairDev pr = pairs[i];
    const int ne = entries_of(G[pr.ga], G[pr.gb], mem);
    const float2* M = maps + moff[i] + t;
    const float2* v = stage + r * E;
    df acc{0.f, 0.f};
    for (int e = 0; e < ne; ++e) {
        const float2 m = __ldg(M + (long long)e * NT);
        const float2 x = v[e];
        acc = df_add(acc, df_mul_u(df{m.x, m.y}, df{x.x, x.y}));
    }
    const long long off = dst.pos ? (long long)d * dst.total + dst.base[c] + (long long)t * dst.stride[c] + dst.pos[i]
                                  : (long long)d * lay.total + lay.base[c] + (i - lay.start[c]) +
                                        (long long)t * (lay.start[c + 1] - lay.start[c]);
    Dp[off] = make_float2(acc.hi, acc.lo);
}

__global__ void __launch_bounds__(256) k_jtransform_map_df(const PairDev* __restrict__ pairs,
                                                           const GroupDev* __restrict__ G,
                                                           const MemberDev* __restrict__ mem,
                                                           const long long* __restrict__ moff,
                                                           const float2* __restrict__ maps,
                                                           const double* __restrict__ Jp, int nchunks, int nao,
                                                           int nk, MapLayout lay, RecBlocks rb,
                                                           double* __restrict__ J0n) {
    extern __shared__ float2 stage[];
    const int d = blockIdx.y;
    const int c = block_class(rb);
    const int NT = nterms(c), E = rb.width[c], R = rb.per[c];
    const long long r0 = rb.rstart[c] + (long long)(blockIdx.x - rb.bstart[c]) * R;
    const long long rend = rb.rstart[c] + rb.rcount[c];
    const long long cnt = lay.start[c + 1] - lay.start[c];
    for (int idx = threadIdx.x; idx < R * NT; idx += blockDim.x) {
        const long long i = r0 + idx / NT;
        const int t = idx % NT;
        df s{0.f, 0.f};
        if (i < rend) {
            const long long loc = i - lay.start[c];
            for (int ch = 0; ch < nchunks; ++ch)
                s = df_add(s, split_double(__ldg(Jp + ((long long)d * nchunks + ch) * lay.total + lay.base[c] +
                                                 (long long)t * cnt + loc)));
        }
        stage[idx] = make_float2(s.hi, s.lo);
    }
    __syncthreads();
    const int r = threadIdx.x / E, e = threadIdx.x % E;
    const long long i = r0 + r;
    if (r >= R || i >= rend) return;
    const PairDev pr = pairs[i];
    int row, col;
    if (!entry_ao(G[pr.ga], G[pr.gb], mem, e, row, col)) return;
    const float2* M = maps + moff[i] + (long long)e * NT;
    const float2* jt = stage + r * NT;
    df s{0.f, 0.f};
    for (int t = 0; t < NT; ++t) {
        const float2 m = __ldg(M + t);
        const float2 x = jt[t];
        s = df_add(s, df_mul_u(df{m.x, m.y}, df{x.x, x.y}));
    }
    const double v = join_df(s);
    const long long nn = (long long)nao * nao;
    atomicAdd(J0n + ((long long)d * nk + pr.cell) * nn + (long long)row * nao + col, v);
    if (pr.weight == 2) atomicAdd(J0n + ((long long)d * nk + pr.mcell) * nn + (long long)col * nao + row, v);
}

// Per-record G cutoff (Sec. 2.5, Eq. "AFT screening obj"): the radius beyond
// which 8 pi eta G (4 pi / G^2) e^{-G^2/4w^2} B(G) stays below eps, with
// eta = (1/p + 1/w^2)^{-1} and B(G) = e^{-G^2/4p} max_{fq} sum_term |M_fq,term|
// (G a_max / 2 pi)^deg(term), an upper bound of every component of the
// record's exact pair transform at |G| = G in any direction (the map M holds
// the normalisation, contraction, E coefficients, K and (pi/p)^{3/2}; the
// relative coordinates obey |n_i| <= G |a_i| / 2 pi).  Searched in the log
// domain in FP32 (a screening estimate): a 64-point scan down from the
// sphere's radius, then 16 bisections of the bracket; the upper end is kept.
__global__ void k_pair_gcut(const PairDev* __restrict__ pairs, const GroupDev* __restrict__ G,
                            const MemberDev* __restrict__ mem, const long long* __restrict__ moff,
                            const double* __restrict__ maps, long long npairs, float gmax, float amax_2pi,
                            float omega, float log_eps, float* __restrict__ gcut) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    const PairDev pr = pairs[i];
    const int L = pr.cls, NT = nterms(L);
    const int ne = entries_of(G[pr.ga], G[pr.gb], mem);
    const double* M = maps + moff[i];
    float c[kLpair + 1];
    for (int l = 0; l <= kLpair; ++l) c[l] = 0.f;
    for (int e = 0; e < ne; ++e) {
        int t = 0;
        for (int lam = 0; lam <= L; ++lam) {
            float s = 0.f;
            for (int b = 0; b < nmono(lam); ++b, ++t) s += (float)fabs(M[(long long)e * NT + t]);
            c[lam] = fmaxf(c[lam], s);
        }
    }
    const float p = (float)pr.p;
    const float eta = 1.f / (1.f / p + 1.f / (omega * omega));
    const float decay = 0.25f / (omega * omega) + 0.25f / p;
    const float lpref = logf(32.f * 9.8696044f * eta);
    auto logf_at = [&](float g) {
        float poly = 0.f, x = 1.f;
        for (int lam = 0; lam <= L; ++lam) {
            poly += c[lam] * x;
            x *= g * amax_2pi;
        }
        return poly > 0.f ? lpref - logf(g) - g * g * decay + logf(poly) : -INFINITY;
    };
    constexpr int kScan = 64;
    const float dg = gmax / kScan;
    float cut = dg;
    if (logf_at(gmax) >= log_eps) {
        cut = gmax;
    } else {
        for (int k = kScan - 1; k >= 1; --k) {
            const float g = k * dg;
            if (logf_at(g) >= log_eps) {
                float lo = g, hi = g + dg;
                for (int it = 0; it < 16; ++it) {
                    const float mid = 0.5f * (lo + hi);
                    if (logf_at(mid) >= log_eps) lo = mid;
                    else hi = mid;
                }
                cut = hi;
                break;
            }
        }
    }
    gcut[i] = fminf(cut * 1.000001f, gmax * 1.000001f);
}

// the geometry-only maps, rewritten in place as double-float
__global__ void k_maps_to_df(double* __restrict__ maps, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df v = split_double(maps[i]);
    reinterpret_cast<float2*>(maps)[i] = make_float2(v.hi, v.lo);
}

RecBlocks make_rec_blocks(const ftcj_plan* P, const long long* width, const long long* stage, int bdim) {
    RecBlocks rb;
    rb.bstart[0] = 0;
    for (int c = 0; c < kNclass; ++c) {
        rb.rstart[c] = P->class_start[c];
        rb.rcount[c] = P->class_start[c + 1] - P->class_start[c];
        rb.width[c] = (int)std::max<long long>(width[c], 1);
        rb.stage[c] = (int)std::max<long long>(stage[c], 1);
        rb.per[c] = std::max(1, bdim / rb.width[c]);
        const long long nb = rb.rcount[c] > 0 ? (rb.rcount[c] + rb.per[c] - 1) / rb.per[c] : 0;
        rb.bstart[c + 1] = rb.bstart[c] + (int)nb;
    }
    return rb;
}

size_t rec_blocks_smem(const RecBlocks& rb) {
    size_t m = 0;
    for (int c = 0; c < kNclass; ++c)
        if (rb.rcount[c] > 0) m = std::max(m, sizeof(float2) * (size_t)rb.per[c] * rb.stage[c]);
    return m;
}

// the tensor-core plans take the Hermite terms in their own K order
TermDest term_dest(const ftcj_plan* P) {
    TermDest t;
    t.pos = P->tc ? P->d_tc_pos : nullptr;
    for (int c = 0; c < kNclass; ++c) {
        t.base[c] = P->tc_dp_base[c];
        t.stride[c] = P->tc_dp_stride[c];
    }
    t.total = P->tc_dp_total;
    return t;
}

MapLayout make_map_layout(const ftcj_plan* P) {
    MapLayout l;
    for (int c = 0; c <= kNclass; ++c) l.start[c] = P->class_start[c];
    for (int c = 0; c < kNclass; ++c) l.base[c] = P->term_base[c];
    l.total = P->total_terms;
    return l;
}

}  // namespace

int build_maps(ftcj_plan* P) {
    if (P->npairs == 0) return FTCJ_OK;
    // sizes from the host copies of the records and members
    std::vector<PairDev> h((size_t)P->npairs);
    FTCJ_CUDA(cudaMemcpy(h.data(), P->d_pairs, sizeof(PairDev) * h.size(), cudaMemcpyDeviceToHost));
    std::vector<long long> off(h.size() + 1, 0);
    auto nf = [](const MemberDev& m) { return m.sph ? 2 * m.l + 1 : (m.l + 1) * (m.l + 2) / 2; };
    for (size_t i = 0; i < h.size(); ++i) {
        const GroupDev& A = P->groups[h[i].ga];
        const GroupDev& B = P->groups[h[i].gb];
        long long s = 0;
        for (int a = A.mem0; a < A.mem1; ++a)
            for (int b = B.mem0; b < B.mem1; ++b) s += (long long)nterms(h[i].cls) * nf(P->members[a]) * nf(P->members[b]);
        off[i + 1] = off[i] + s;
    }
    P->map_doubles = off.back();
    // thread ranges: a3 uses nterms(L) threads per record, a7 the largest
    // output count (sum of nf_a nf_b over member pairs) of the class
    long long maxout[kNclass] = {0, 0, 0, 0, 0};
    for (size_t i = 0; i < h.size(); ++i) {
        const GroupDev& A = P->groups[h[i].ga];
        const GroupDev& B = P->groups[h[i].gb];
        long long o = 0;
        for (int a = A.mem0; a < A.mem1; ++a)
            for (int b = B.mem0; b < B.mem1; ++b) o += (long long)nf(P->members[a]) * nf(P->members[b]);
        maxout[h[i].cls] = std::max(maxout[h[i].cls], o);
    }
    P->mt_terms.tstart[0] = P->mt_outs.tstart[0] = 0;
    for (int c = 0; c < kNclass; ++c) {
        const long long cnt = P->class_start[c + 1] - P->class_start[c];
        P->mt_terms.rstart[c] = P->mt_outs.rstart[c] = P->class_start[c];
        P->mt_terms.slots[c] = cnt > 0 ? nterms(c) : 0;
        P->mt_outs.slots[c] = cnt > 0 ? (int)maxout[c] : 0;
        P->mt_terms.tstart[c + 1] = P->mt_terms.tstart[c] + cnt * P->mt_terms.slots[c];
        P->mt_outs.tstart[c + 1] = P->mt_outs.tstart[c] + cnt * P->mt_outs.slots[c];
    }
    FTCJ_CUDA(cudaMalloc(&P->d_map_off, sizeof(long long) * off.size()));
    P->device_bytes += sizeof(long long) * off.size();
    FTCJ_CUDA(cudaMemcpy(P->d_map_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaMalloc(&P->d_maps, sizeof(double) * (size_t)std::max<long long>(P->map_doubles, 1)));
    P->device_bytes += sizeof(double) * (size_t)std::max<long long>(P->map_doubles, 1);
    // host copies of the cell-independent tables for the build kernel
    std::vector<double> Ut;
    std::vector<int> cart, Toff;
    host_hermite_tables(P, Ut, cart, Toff);
    double* dU = nullptr;
    int *dC = nullptr, *dT = nullptr;
    FTCJ_CUDA(cudaMalloc(&dU, sizeof(double) * Ut.size()));
    FTCJ_CUDA(cudaMalloc(&dC, sizeof(int) * cart.size()));
    FTCJ_CUDA(cudaMalloc(&dT, sizeof(int) * Toff.size()));
    FTCJ_CUDA(cudaMemcpy(dU, Ut.data(), sizeof(double) * Ut.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaMemcpy(dC, cart.data(), sizeof(int) * cart.size(), cudaMemcpyHostToDevice));
    FTCJ_CUDA(cudaMemcpy(dT, Toff.data(), sizeof(int) * Toff.size(), cudaMemcpyHostToDevice));
    k_map_build<<<(unsigned)((P->npairs + 127) / 128), 128>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off,
                                                              P->npairs, P->d_Tmat, dT, dU, dC, P->d_maps, P->cc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dU);
    cudaFree(dC);
    cudaFree(dT);
    if (e != cudaSuccess) return cuda_fail(e, "k_map_build");
    // split form: double-float maps and record-major blocks, when every record's
    // outputs fit one block
    if (P->params.pair_gcut_eps > 0.0) {
        int rc = launch_pair_gcut(P);
        if (rc) return rc;
    }
    P->maps_df = false;
    if (P->precision == FTCJ_PREC_SPLIT) {
        long long nt[kNclass];
        for (int c = 0; c < kNclass; ++c) nt[c] = nterms(c);
        bool fits = true;
        for (int c = 0; c < kNclass; ++c) fits = fits && maxout[c] <= 256;
        if (fits) {
            P->rb_terms = make_rec_blocks(P, nt, maxout, 256);
            P->rb_outs = make_rec_blocks(P, maxout, nt, 256);
            P->rb_terms_smem = rec_blocks_smem(P->rb_terms);
            P->rb_outs_smem = rec_blocks_smem(P->rb_outs);
            int rc = allow_dynamic_smem((const void*)k_hermite_map_df, P->rb_terms_smem);
            if (!rc) rc = allow_dynamic_smem((const void*)k_jtransform_map_df, P->rb_outs_smem);
            if (rc) return rc;
            k_maps_to_df<<<(unsigned)((P->map_doubles + 255) / 256), 256>>>(P->d_maps, P->map_doubles);
            FTCJ_CUDA(cudaGetLastError());
            FTCJ_CUDA(cudaDeviceSynchronize());
            P->maps_df = true;
        }
    }
    return FTCJ_OK;
}

int launch_pair_gcut(ftcj_plan* P) {
    if (P->npairs == 0) return FTCJ_OK;
    FTCJ_CUDA(cudaMalloc(&P->d_rec_gcut, sizeof(float) * (size_t)P->npairs));
    P->device_bytes += sizeof(float) * (size_t)P->npairs;
    double amax = 0.0;
    for (int r = 0; r < 3; ++r)
        amax = std::max(amax, std::sqrt(P->A[3 * r] * P->A[3 * r] + P->A[3 * r + 1] * P->A[3 * r + 1] +
                                        P->A[3 * r + 2] * P->A[3 * r + 2]));
    k_pair_gcut<<<(unsigned)((P->npairs + 127) / 128), 128>>>(
        P->d_pairs, P->d_groups, P->d_members, P->d_map_off, P->d_maps, P->npairs, (float)P->gcut,
        (float)(amax / (2.0 * M_PI)), (float)P->params.omega, (float)std::log(P->params.pair_gcut_eps), P->d_rec_gcut);
    FTCJ_CUDA(cudaGetLastError());
    FTCJ_CUDA(cudaDeviceSynchronize());
    return FTCJ_OK;
}

int launch_hermite_map(ftcj_plan* P, int ndens, const double* D0n, cudaStream_t s) {
    if (P->npairs == 0) return FTCJ_OK;
    if (P->maps_df) {
        dim3 g((unsigned)P->rb_terms.bstart[kNclass], ndens);
        k_hermite_map_df<<<g, 256, P->rb_terms_smem, s>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off,
                                                          reinterpret_cast<const float2*>(P->d_maps), D0n, P->nao,
                                                          P->nk, make_map_layout(P), P->rb_terms, term_dest(P),
                                                          reinterpret_cast<float2*>(P->d_Dp));
        FTCJ_CUDA(cudaGetLastError());
        return FTCJ_OK;
    }
    const long long n = P->mt_terms.tstart[kNclass];
    dim3 g((unsigned)((n + 255) / 256), ndens);
    if (P->precision == FTCJ_PREC_SPLIT)
        k_hermite_map<true><<<g, 256, 0, s>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off, P->d_maps, D0n,
                                              P->nao, P->nk, make_map_layout(P), P->mt_terms, P->d_Dp);
    else
        k_hermite_map<false><<<g, 256, 0, s>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off, P->d_maps, D0n,
                                               P->nao, P->nk, make_map_layout(P), P->mt_terms, P->d_Dp);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

int launch_jtransform_map(ftcj_plan* P, int ndens, double* J0n, cudaStream_t s, bool zero) {
    const size_t bytes = sizeof(double) * (size_t)ndens * P->nk * P->nao * P->nao;
    if (zero) FTCJ_CUDA(cudaMemsetAsync(J0n, 0, bytes, s));
    if (P->npairs == 0) return FTCJ_OK;
    if (P->maps_df) {
        dim3 g((unsigned)P->rb_outs.bstart[kNclass], ndens);
        k_jtransform_map_df<<<g, 256, P->rb_outs_smem, s>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off,
                                                            reinterpret_cast<const float2*>(P->d_maps), P->d_Jp,
                                                            jp_chunks(P), P->nao, P->nk,
                                                            make_map_layout(P), P->rb_outs, J0n);
        FTCJ_CUDA(cudaGetLastError());
        return FTCJ_OK;
    }
    const long long n = P->mt_outs.tstart[kNclass];
    dim3 g((unsigned)((n + 255) / 256), ndens);
    k_jtransform_map<<<g, 256, 0, s>>>(P->d_pairs, P->d_groups, P->d_members, P->d_map_off, P->d_maps, P->d_Jp,
                                       jp_chunks(P), P->nao, P->nk, make_map_layout(P), P->mt_outs, J0n);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

}  // namespace ftcj
