// Steps a3 and a7: the per-pair density transformation of Alg. 2 and its
// mirror for J (Alg. S2).
//
// a3: for a pair record (groups a, b; cell L) the BvK density block is taken to
// Cartesian components, then through the McMurchie-Davidson expansion of the
// Gaussian product (x-A)^i (x-B)^j e^{-p x_P^2} = sum_t E^{ij}_t (d/dP_x)^t
// e^{-p x_P^2} (equivalent to Eq. "Gaussian product of angular prefactor"
// followed by Eq. "FT of cart Gaussians") into Hermite densities h_tuv, so that
//   rho_pair(G) = K e^{-G^2/4p} e^{-iG.P} sum_tuv h_tuv (-iG_x)^t (-iG_y)^u (-iG_z)^v.
// The Cartesian powers of G are then re-expanded in the integer coordinates
// n of G = sum_i n_i b_i (Eq. "transform cart angular factor to relative
// angular factor"), giving D'_ijk with
//   rho_pair(G) = e^{-G^2/4p} e^{-iG.P} sum_ijk (-i)^{i+j+k} D'_ijk n1^i n2^j n3^k.
// a7 applies the transpose of every step to J'_ijk and scatters the AO block
// into J^{0[L]} (and its mirror into J^{0[-L]}).
#include <cmath>
#include <mutex>
#include <vector>

#include "ftcj_internal.h"

namespace ftcj {
namespace {

constexpr int kLgrad = kLpair + 1;                        // degree of the gradient sums
constexpr int kTmatSize = 1 + 9 + 36 + 100 + 225 + 441;  // sum over lambda <= 5 of nmono^2

__constant__ double c_U[kLmax + 1][2][kNcartMax][kNcartMax];  // [l][sph][function][cart]
__constant__ int c_cart[kLmax + 1][kNcartMax][3];
__constant__ int c_Toff[kLgrad + 1];

struct Layout {
    long long start[kNclass + 1];
    long long base[kNclass];
    long long total;
};

__device__ __forceinline__ int nfunc(int l, int sph) { return sph ? 2 * l + 1 : (l + 1) * (l + 2) / 2; }

// E^{ij}_t for i <= la1 <= 3, j <= lb1 <= 3 (MD recurrences), for the gradient
__device__ void ecoef_g(double PA, double PB, double a2p, int la1, int lb1, double E[4][4][7]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int t = 0; t < 7; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 1; i <= la1; ++i)
        for (int t = 0; t <= i; ++t)
            E[i][0][t] = (t > 0 ? a2p * E[i - 1][0][t - 1] : 0.0) + PA * E[i - 1][0][t] +
                         (t + 1) * E[i - 1][0][t + 1];
    for (int i = 0; i <= la1; ++i)
        for (int j = 1; j <= lb1; ++j)
            for (int t = 0; t <= i + j && t < 7; ++t)
                E[i][j][t] = (t > 0 ? a2p * E[i][j - 1][t - 1] : 0.0) + PB * E[i][j - 1][t] +
                             (t + 1 < 7 ? (t + 1) * E[i][j - 1][t + 1] : 0.0);
}

// sum_tuv E^x_t(a0,b0) E^y_u(a1,b1) E^z_v(a2,b2) J_tuv for Cartesian exponent triples a, b
__device__ __forceinline__ double cart_contract(const double (*Ex)[4][7], const double (*Ey)[4][7],
                                                const double (*Ez)[4][7], const int* a, const int* b,
                                                const double* jt) {
    double s = 0.0;
    for (int t = 0; t <= a[0] + b[0]; ++t)
        for (int u = 0; u <= a[1] + b[1]; ++u) {
            const double exy = Ex[a[0]][b[0]][t] * Ey[a[1]][b[1]][u];
            for (int v = 0; v <= a[2] + b[2]; ++v) {
                const int lam = t + u + v;
                s += exy * Ez[a[2]][b[2]][v] * jt[lam_offset(lam) + mono_index(lam, t, u)];
            }
        }
    return s;
}

// Nuclear gradient of E_J, one pair record per thread:
//   dE/dA_x = sum_{ca,cb} Dcart[ca][cb] (2 alpha S(ca + x, cb) - ca_x S(ca - x, cb)),
//   dE/dB_x = sum_{ca,cb} Dcart[ca][cb] (2 beta  S(ca, cb + x) - cb_x S(ca, cb - x)),
// from d/dA [(x-A)^i e^{-alpha (x-A)^2}] = 2 alpha (x-A)^{i+1} e^{..} - i (x-A)^{i-1} e^{..},
// with S(a, b) the Cartesian contraction of the degree-(L+1) sums J_tuv
// (= K Re sum_half W g ph (-iG)^tuv).  Dcart is the combined density of the
// record and its mirror, as in the Hermite-density step, so the mirror's derivative is included.
__global__ void __launch_bounds__(128) k_grad_assemble(const PairDev* __restrict__ pairs,
                                                       const GroupDev* __restrict__ G,
                                                       const MemberDev* __restrict__ mem,
                                                       const double* __restrict__ D0n,
                                                       const double* __restrict__ Jg, int nchunks, int nao, int nk,
                                                       Layout lay, double* __restrict__ grad, int ncentre,
                                                       const double* __restrict__ Tm, CellConst cc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (i >= lay.start[kNclass]) return;
    const PairDev pr = pairs[i];
    const int L = pr.cls, Lg = L + 1;
    const long long cnt = lay.start[L + 1] - lay.start[L];
    const long long loc = i - lay.start[L];
    double jp[nterms(kLgrad)];
    const int NT = nterms(Lg);
    for (int t = 0; t < NT; ++t) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c)
            s += Jg[((long long)d * nchunks + c) * lay.total + lay.base[L] + (long long)t * cnt + loc];
        jp[t] = s;
    }
    double jt[nterms(kLgrad)];
    for (int lam = 0; lam <= Lg; ++lam) {
        const int nm = nmono(lam), o = lam_offset(lam);
        const double* T = Tm + c_Toff[lam];
        for (int a = 0; a < nm; ++a) {
            double s = 0.0;
            for (int b = 0; b < nm; ++b) s += T[a * nm + b] * jp[o + b];
            jt[o + a] = pr.K * s;
        }
    }
    const GroupDev A = G[pr.ga];
    const GroupDev B = G[pr.gb];
    double E[3][4][4][7];
    {
        const double Av[3] = {A.x, A.y, A.z};
        const double Bv[3] = {B.x, B.y, B.z};
        const double a2p = 0.5 / pr.p;
        for (int x = 0; x < 3; ++x) {
            const double Bs = Bv[x] + pr.L[0] * cc.A[x] + pr.L[1] * cc.A[3 + x] + pr.L[2] * cc.A[6 + x];
            ecoef_g(pr.P[x] - Av[x], pr.P[x] - Bs, a2p, A.lmax + 1, B.lmax + 1, E[x]);
        }
    }
    double gA[3] = {0.0, 0.0, 0.0}, gB[3] = {0.0, 0.0, 0.0};
    const long long nn = (long long)nao * nao;
    const double* Dc = D0n + ((long long)d * nk + pr.cell) * nn;
    const double* Dm = D0n + ((long long)d * nk + pr.mcell) * nn;
    for (int ia = A.mem0; ia < A.mem1; ++ia) {
        const MemberDev ma = mem[ia];
        const int nfa = nfunc(ma.l, ma.sph), nca = (ma.l + 1) * (ma.l + 2) / 2;
        for (int ib = B.mem0; ib < B.mem1; ++ib) {
            const MemberDev mb = mem[ib];
            const int nfb = nfunc(mb.l, mb.sph), ncb = (mb.l + 1) * (mb.l + 2) / 2;
            double tmp[kNcartMax][kNcartMax];
            for (int f = 0; f < nfa; ++f)
                for (int cb = 0; cb < ncb; ++cb) {
                    double s = 0.0;
                    for (int q = 0; q < nfb; ++q) {
                        const double u = c_U[mb.l][mb.sph][q][cb];
                        if (u == 0.0) continue;
                        double dv = Dc[(long long)(ma.ao + f) * nao + mb.ao + q];
                        if (pr.weight == 2) dv += Dm[(long long)(mb.ao + q) * nao + ma.ao + f];
                        s += u * dv;
                    }
                    tmp[f][cb] = s;
                }
            const double coef = ma.coef * mb.coef;
            for (int ca = 0; ca < nca; ++ca) {
                const int* xa = c_cart[ma.l][ca];
                for (int cb = 0; cb < ncb; ++cb) {
                    double dcart = 0.0;
                    for (int f = 0; f < nfa; ++f) dcart += c_U[ma.l][ma.sph][f][ca] * tmp[f][cb];
                    dcart *= coef;
                    if (dcart == 0.0) continue;
                    const int* xb = c_cart[mb.l][cb];
                    for (int x = 0; x < 3; ++x) {
                        int a2[3] = {xa[0], xa[1], xa[2]};
                        int b2[3] = {xb[0], xb[1], xb[2]};
                        a2[x] += 1;
                        double s = 2.0 * A.alpha * cart_contract(E[0], E[1], E[2], a2, xb, jt);
                        if (xa[x] > 0) {
                            a2[x] -= 2;
                            s -= xa[x] * cart_contract(E[0], E[1], E[2], a2, xb, jt);
                        }
                        gA[x] += dcart * s;
                        b2[x] += 1;
                        double t = 2.0 * B.alpha * cart_contract(E[0], E[1], E[2], xa, b2, jt);
                        if (xb[x] > 0) {
                            b2[x] -= 2;
                            t -= xb[x] * cart_contract(E[0], E[1], E[2], xa, b2, jt);
                        }
                        gB[x] += dcart * t;
                    }
                }
            }
        }
    }
    for (int x = 0; x < 3; ++x) {
        atomicAdd(grad + ((long long)d * ncentre + A.centre) * 3 + x, gA[x]);
        atomicAdd(grad + ((long long)d * ncentre + B.centre) * 3 + x, gB[x]);
    }
}

Layout make_layout(const ftcj_plan* P) {
    Layout l;
    for (int c = 0; c <= kNclass; ++c) l.start[c] = P->class_start[c];
    for (int c = 0; c < kNclass; ++c) l.base[c] = P->term_base[c];
    l.total = P->total_terms;
    return l;
}

}  // namespace

// Host tables: Cartesian component order, the AO -> Cartesian matrices of the
// unit-normalised functions (radial part (2a/pi)^{3/4} (4a)^{l/2} is in the
// member coefficient), and the per-lambda expansion of G_x^t G_y^u G_z^v in
// n1^i n2^j n3^k for G = sum_i n_i b_i.
static std::mutex g_table_mutex;
static bool g_tables_on_device[64] = {};

// Cartesian exponents [l][c][3], AO -> Cartesian matrices [l][sph][f][c] (kNcartMax
// strides) and the per-lambda offsets of the relative-coordinate transforms.
void host_hermite_tables(const ftcj_plan* P, std::vector<double>& Uv, std::vector<int>& cartv, std::vector<int>& Toffv) {
    (void)P;
    cartv.assign((kLmax + 1) * kNcartMax * 3, 0);
    for (int l = 0; l <= kLmax; ++l) {
        int n = 0;
        for (int lx = l; lx >= 0; --lx)
            for (int ly = l - lx; ly >= 0; --ly) {
                cartv[(l * kNcartMax + n) * 3 + 0] = lx;
                cartv[(l * kNcartMax + n) * 3 + 1] = ly;
                cartv[(l * kNcartMax + n) * 3 + 2] = l - lx - ly;
                ++n;
            }
    }
    Uv.assign((kLmax + 1) * 2 * kNcartMax * kNcartMax, 0.0);
    auto U = [&](int l, int sph, int f, int c) -> double& { return Uv[((l * 2 + sph) * kNcartMax + f) * kNcartMax + c]; };
    auto dfact = [](int n) {
        double r = 1.0;
        for (int k = n; k > 1; k -= 2) r *= k;
        return r;
    };
    for (int l = 0; l <= kLmax; ++l) {
        const int nc = (l + 1) * (l + 2) / 2;
        for (int c = 0; c < nc; ++c) {
            const int* x = &cartv[(l * kNcartMax + c) * 3];
            U(l, 0, c, c) = 1.0 / std::sqrt(dfact(2 * x[0] - 1) * dfact(2 * x[1] - 1) * dfact(2 * x[2] - 1));
        }
    }
    U(0, 1, 0, 0) = 1.0;
    U(1, 1, 0, 0) = 1.0;  // x
    U(1, 1, 1, 1) = 1.0;  // y
    U(1, 1, 2, 2) = 1.0;  // z
    {
        // d: Cartesian order xx, xy, xz, yy, yz, zz; functions m = -2..2 = xy, yz, z2, xz, x2-y2
        const double r3 = 1.0 / std::sqrt(3.0);
        U(2, 1, 0, 1) = 1.0;        // xy
        U(2, 1, 1, 4) = 1.0;        // yz
        U(2, 1, 2, 0) = -0.5 * r3;  // z2 = (2zz - xx - yy)/2, over sqrt(3)
        U(2, 1, 2, 3) = -0.5 * r3;
        U(2, 1, 2, 5) = r3;
        U(2, 1, 3, 2) = 1.0;  // xz
        U(2, 1, 4, 0) = 0.5;  // (xx - yy) sqrt(3)/2, over sqrt(3)
        U(2, 1, 4, 3) = -0.5;
    }
    Toffv.assign(kLgrad + 1, 0);
    int off = 0;
    for (int lam = 0; lam <= kLgrad; ++lam) {
        Toffv[lam] = off;
        off += nmono(lam) * nmono(lam);
    }
}

int upload_hermite_tables(ftcj_plan* P) {
    int dev = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_table_mutex);
    const bool need_const = dev < 0 || dev >= 64 || !g_tables_on_device[dev];
    std::vector<double> Uh;
    std::vector<int> carth, Toffh;
    host_hermite_tables(P, Uh, carth, Toffh);
    int cart[kLmax + 1][kNcartMax][3] = {};
    std::copy(carth.begin(), carth.end(), &cart[0][0][0]);
    if (need_const) FTCJ_CUDA(cudaMemcpyToSymbol(c_cart, cart, sizeof(cart)));
    double U[kLmax + 1][2][kNcartMax][kNcartMax] = {};
    std::copy(Uh.begin(), Uh.end(), &U[0][0][0][0]);
    if (need_const) FTCJ_CUDA(cudaMemcpyToSymbol(c_U, U, sizeof(U)));
    // G_x^t G_y^u G_z^v with G_x = sum_i n_i B[i][x]: expand as polynomials in (n1, n2, n3)
    std::vector<double> T(kTmatSize, 0.0);
    int Toff[kLgrad + 1];
    int off = 0;
    for (int lam = 0; lam <= kLgrad; ++lam) {
        Toff[lam] = off;
        int nm = nmono(lam);
        for (int t = lam; t >= 0; --t)
            for (int u = lam - t; u >= 0; --u) {
                int v = lam - t - u;
                int a = mono_index(lam, t, u);
                // polynomial in n as a dense map (i, j) -> coefficient with k = deg - i - j
                std::vector<double> poly(1, 1.0);  // degree-0 polynomial
                int deg = 0;
                auto mul_linear = [&](int axis) {
                    // multiply by (B[0][axis] n1 + B[1][axis] n2 + B[2][axis] n3)
                    int nd = deg + 1;
                    std::vector<double> np(nmono(nd), 0.0);
                    for (int i = deg; i >= 0; --i)
                        for (int j = deg - i; j >= 0; --j) {
                            double cval = poly[mono_index(deg, i, j)];
                            if (cval == 0.0) continue;
                            np[mono_index(nd, i + 1, j)] += cval * P->B[0 * 3 + axis];
                            np[mono_index(nd, i, j + 1)] += cval * P->B[1 * 3 + axis];
                            np[mono_index(nd, i, j)] += cval * P->B[2 * 3 + axis];
                        }
                    poly.swap(np);
                    deg = nd;
                };
                for (int q = 0; q < t; ++q) mul_linear(0);
                for (int q = 0; q < u; ++q) mul_linear(1);
                for (int q = 0; q < v; ++q) mul_linear(2);
                for (int b = 0; b < nm; ++b) T[off + a * nm + b] = poly[b];
            }
        off += nm * nm;
    }
    FTCJ_CUDA(cudaMalloc(&P->d_Tmat, sizeof(double) * kTmatSize));
    P->device_bytes += sizeof(double) * kTmatSize;
    FTCJ_CUDA(cudaMemcpy(P->d_Tmat, T.data(), sizeof(double) * kTmatSize, cudaMemcpyHostToDevice));
    if (need_const) {
        FTCJ_CUDA(cudaMemcpyToSymbol(c_Toff, Toff, sizeof(Toff)));
        if (dev >= 0 && dev < 64) g_tables_on_device[dev] = true;
    }
    return FTCJ_OK;
}

int launch_grad_assemble(ftcj_plan* P, int ndens, const double* D0n, double* grad, cudaStream_t s) {
    FTCJ_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)ndens * P->ncentre * 3, s));
    if (P->npairs == 0) return FTCJ_OK;
    Layout lg = make_layout(P);
    for (int c = 0; c < kNclass; ++c) lg.base[c] = P->term_base_g[c];
    lg.total = P->total_terms_g;
    dim3 g((unsigned)((P->npairs + 127) / 128), ndens);
    k_grad_assemble<<<g, 128, 0, s>>>(P->d_pairs, P->d_groups, P->d_members, D0n, P->d_Jg, (int)P->chunks.size(),
                                      P->nao, P->nk, lg, grad, P->ncentre, P->d_Tmat, P->cc);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}

}  // namespace ftcj
