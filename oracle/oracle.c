/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the long-range (G != 0)
 * planewave density-fitting Coulomb build of
 *   "Efficient All-Electron Periodic Fourier-Transformed Coulomb Method"
 *   (arXiv 2509.16460).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path never calls it, and this file shares no code, header, table or
 * constant generator with that path.
 *
 * What it computes (the plain definitions, no factorisation tricks):
 *   1. D^{0n} = (1/Nk) sum_k exp(-i k.R_n) D^k over the BvK cells n
 *      (Sec. 2.2, Eq. "FT for D", read with the 1/Nk and the minus sign so
 *      that it inverts Eq. "FT of J").
 *   2. Screened ordered primitive pairs (a in the home cell, b in cell L,
 *      L in Z^3): (2 sqrt(a b)/p)^{3/2} exp(-a b/p |A-B-R_L|^2) > thresh.
 *   3. Pair transform (mu0 nuL|G) = int phi_mu(r) phi_nu(r-R_L) e^{-iG.r} dr
 *      (Sec. 2.4, Eq. "AFT for pair density"), evaluated per axis by the
 *      binomial expansion about the Gaussian product centre (Eq. "Gaussian
 *      product of angular prefactor", Eqs. GPT) and the Hermite-polynomial
 *      transform of a centred Cartesian Gaussian (Eq. "FT of cart
 *      Gaussians", read with (-i/(2 sqrt p))^l so that it matches the
 *      e^{-iG.r} transform), Hermite polynomials from their recurrence
 *      (Appendix A).
 *   4. rho(G) = sum_{mu nu L} D^{0[L]}_{mu nu} (mu0 nuL|G) for every
 *      G = sum n_i b_i != 0 with |G|^2 < Gcut^2 (long-range step 1).
 *   5. J^{0L}_{mu nu} = sum_G v(G) (mu0 nuL|G) rho(-G),
 *      v(G) = 4 pi exp(-G^2/4w^2) / (Omega G^2) (Eq. "Ewald J", second
 *      term; long-range steps 2-3), rho(-G) taken from its own explicit sum.
 *   6. J^k = sum_L exp(+i k.R_L) J^{0L} (Eq. "FT of J").
 *   7. E_J = 1/2 sum_G v(G) rho(G) rho(-G).
 *   8. With the densities classified (Sec. 2.6): pair densities whose two
 *      primitives both have exponents below alpha_cut are DD; an integral
 *      between two compact pair densities keeps v(G), every other one takes
 *      the full-range 4 pi / (Omega G^2) (orc_lrj_classified).
 *   9. The DD density on a uniform real-space grid of the cell, summed over
 *      lattice images from the basis functions themselves (App. E,
 *      orc_gpw_density); its discrete Fourier transform is the GPW route to
 *      rho_D(G).
 *
 * Normalisation: every primitive is scaled to unit self-overlap, computed
 * here from 1D Gaussian moments.  Spherical shells use real solid harmonics
 * in Racah normalisation from the closed form in Helgaker, Jorgensen, Olsen,
 * "Molecular Electronic-Structure Theory", Eqs. 6.4.48-6.4.50; order
 * m = -l..l, except p which is (x, y, z).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 4
#define ORC_MAXC 15 /* Cartesian components for l = 4 */

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

static double ipow(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

/* Cartesian component list of angular momentum l: lx = l..0, ly = l-lx..0 */
static int cart_list(int l, int c[][3])
{
    int n = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            c[n][0] = lx;
            c[n][1] = ly;
            c[n][2] = l - lx - ly;
            ++n;
        }
    return n;
}

static int cart_index(int l, int lx, int ly)
{
    /* position of (lx, ly, l-lx-ly) in cart_list order */
    int idx = 0;
    for (int x = l; x > lx; --x) idx += l - x + 1;
    return idx + (l - lx - ly);
}

/* Real solid harmonic S_lm (Racah normalisation) as coefficients over the
 * Cartesian monomials of degree l (HJO Eqs. 6.4.48-6.4.50). */
static void solid_harmonic(int l, int m, double* coef /* [ncart(l)] */)
{
    int ncart = (l + 1) * (l + 2) / 2;
    for (int i = 0; i < ncart; ++i) coef[i] = 0.0;
    int am = m < 0 ? -m : m;
    double vm = (m < 0) ? 0.5 : 0.0;
    double nlm = sqrt(2.0 * factorial(l + am) * factorial(l - am) / (m == 0 ? 2.0 : 1.0)) /
                 (ipow(2.0, am) * factorial(l));
    for (int t = 0; t <= (l - am) / 2; ++t)
        for (int u = 0; u <= t; ++u) {
            /* v runs over vm, vm+1, ..., floor(am/2 - vm) + vm */
            int nv = (int)floor(am / 2.0 - vm) + 1;
            for (int iv = 0; iv < nv; ++iv) {
                double v = vm + iv;
                int twov = (int)lround(2.0 * v);
                double sgn = (((int)lround(t + v - vm)) % 2 == 0) ? 1.0 : -1.0;
                double c = sgn * ipow(0.25, t) * binom(l, t) * binom(l - t, am + t) * binom(t, u) *
                           binom(am, twov);
                int px = 2 * t + am - 2 * u - twov;
                int py = 2 * u + twov;
                int pz = l - 2 * t - am;
                if (px < 0 || py < 0 || pz < 0) continue;
                coef[cart_index(l, px, py)] += nlm * c;
            }
        }
}

/* int_{-inf}^{inf} x^n exp(-a x^2) dx */
static double moment1d(int n, double a)
{
    if (n % 2) return 0.0;
    return tgamma(0.5 * (n + 1)) / pow(a, 0.5 * (n + 1));
}

/* ------------------------------------------------------------------------ */
/* basis                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int cen, l, sph, nf, nc, ao0, np;
    const double* ex;
    const double* co;
    int cx[ORC_MAXC][3];
    double U[2 * ORC_LMAX + 1][ORC_MAXC]; /* function f = sum_c U[f][c] monomial_c */
    double* nrm;                          /* [np][nf] unit self-overlap scale */
} OShell;

typedef struct {
    double A[3][3];   /* rows a_i */
    double B[3][3];   /* rows b_i, a_i . b_j = 2 pi delta_ij */
    double M[3][3];   /* metric b_i . b_j */
    double vol;
    int ncen;
    const double* xyz;
    int nsh, nao;
    OShell* sh;
} OSys;

static int build_system(OSys* S, const double* A, int ncen, const double* xyz, int nsh, const int* sh_cen,
                        const int* sh_l, const int* sh_sph, const int* sh_np, const int* sh_off,
                        const double* exps, const double* coefs)
{
    memset(S, 0, sizeof(*S));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S->A[i][j] = A[3 * i + j];
    double (*a)[3] = S->A;
    double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                 a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                 a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    if (fabs(det) < 1e-12) return -1;
    S->vol = fabs(det);
    /* b_i = 2 pi (a_j x a_k) / det */
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        double cx = a[j][1] * a[k][2] - a[j][2] * a[k][1];
        double cy = a[j][2] * a[k][0] - a[j][0] * a[k][2];
        double cz = a[j][0] * a[k][1] - a[j][1] * a[k][0];
        S->B[i][0] = 2.0 * M_PI * cx / det;
        S->B[i][1] = 2.0 * M_PI * cy / det;
        S->B[i][2] = 2.0 * M_PI * cz / det;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S->M[i][j] = S->B[i][0] * S->B[j][0] + S->B[i][1] * S->B[j][1] + S->B[i][2] * S->B[j][2];
    S->ncen = ncen;
    S->xyz = xyz;
    S->nsh = nsh;
    S->sh = (OShell*)calloc((size_t)(nsh > 0 ? nsh : 1), sizeof(OShell));
    int ao = 0;
    for (int s = 0; s < nsh; ++s) {
        OShell* h = &S->sh[s];
        h->cen = sh_cen[s];
        h->l = sh_l[s];
        h->sph = sh_sph[s];
        if (h->l < 0 || h->l > ORC_LMAX || h->cen < 0 || h->cen >= ncen || sh_np[s] < 1) return -2;
        h->nc = cart_list(h->l, h->cx);
        h->nf = h->sph ? 2 * h->l + 1 : h->nc;
        h->ao0 = ao;
        ao += h->nf;
        h->np = sh_np[s];
        h->ex = exps + sh_off[s];
        h->co = coefs + sh_off[s];
        memset(h->U, 0, sizeof(h->U));
        if (!h->sph) {
            for (int c = 0; c < h->nc; ++c) h->U[c][c] = 1.0;
        } else if (h->l == 1) {
            /* p as (x, y, z): S_{1,1}=x, S_{1,-1}=y, S_{1,0}=z */
            int order[3] = {1, -1, 0};
            for (int f = 0; f < 3; ++f) solid_harmonic(1, order[f], h->U[f]);
        } else {
            for (int f = 0; f < h->nf; ++f) solid_harmonic(h->l, f - h->l, h->U[f]);
        }
        h->nrm = (double*)malloc(sizeof(double) * (size_t)(h->np * h->nf));
        for (int k = 0; k < h->np; ++k) {
            double al = h->ex[k];
            if (!(al > 0.0)) return -3;
            for (int f = 0; f < h->nf; ++f) {
                /* self overlap of sum_c U[f][c] x^c e^{-al r^2} from 1D moments */
                double ov = 0.0;
                for (int c1 = 0; c1 < h->nc; ++c1)
                    for (int c2 = 0; c2 < h->nc; ++c2) {
                        double u = h->U[f][c1] * h->U[f][c2];
                        if (u == 0.0) continue;
                        ov += u * moment1d(h->cx[c1][0] + h->cx[c2][0], 2.0 * al) *
                              moment1d(h->cx[c1][1] + h->cx[c2][1], 2.0 * al) *
                              moment1d(h->cx[c1][2] + h->cx[c2][2], 2.0 * al);
                    }
                h->nrm[k * h->nf + f] = 1.0 / sqrt(ov);
            }
        }
    }
    S->nao = ao;
    return 0;
}

static void free_system(OSys* S)
{
    if (!S->sh) return;
    for (int s = 0; s < S->nsh; ++s) free(S->sh[s].nrm);
    free(S->sh);
    S->sh = NULL;
}

/* ------------------------------------------------------------------------ */
/* pair transform                                                            */
/* ------------------------------------------------------------------------ */

/* physicists' Hermite polynomials H_0..H_n at x (Appendix A recurrence) */
static void hermite(int n, double x, double* H)
{
    H[0] = 1.0;
    if (n >= 1) H[1] = 2.0 * x;
    for (int k = 2; k <= n; ++k) H[k] = 2.0 * x * H[k - 1] - 2.0 * (k - 1) * H[k - 2];
}

/* 1D factors F[i][j] = int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) exp(-i g x) dx
 * for i <= la, j <= lb, by the binomial expansion about P and the Hermite
 * transform of (x-P)^k exp(-p (x-P)^2). */
static void factors1d(int la, int lb, double a, double Ax, double b, double Bx, double g,
                      cplx F[ORC_LMAX + 1][ORC_LMAX + 1])
{
    double p = a + b;
    double mu = a * b / p;
    double Px = (a * Ax + b * Bx) / p;
    double PA = Px - Ax, PB = Px - Bx;
    double H[2 * ORC_LMAX + 2];
    int n = la + lb;
    double sp = sqrt(p);
    hermite(n, g / (2.0 * sp), H);
    cplx base = exp(-mu * (Ax - Bx) * (Ax - Bx)) * sqrt(M_PI / p) * exp(-g * g / (4.0 * p)) *
                cexp(-I * g * Px);
    cplx T[2 * ORC_LMAX + 2];
    cplx fac = 1.0;
    for (int k = 0; k <= n; ++k) {
        T[k] = base * fac * H[k];
        fac *= -I / (2.0 * sp);
    }
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            cplx s = 0.0;
            for (int r = 0; r <= i; ++r)
                for (int t = 0; t <= j; ++t)
                    s += binom(i, r) * binom(j, t) * ipow(PA, i - r) * ipow(PB, j - t) * T[r + t];
            F[i][j] = s;
        }
}

/* d/dA of the 1D factors: d/dA [(x-A)^i e^{-a(x-A)^2}] = 2a (x-A)^{i+1} e^{..} - i (x-A)^{i-1} e^{..},
 * so dF[i][j]/dA = 2a F[i+1][j] - i F[i-1][j] (same for B with b and j). */
static void factors1d_deriv(int la, int lb, double a, double Ax, double b, double Bx, double g,
                            cplx dA[ORC_LMAX + 1][ORC_LMAX + 1], cplx dB[ORC_LMAX + 1][ORC_LMAX + 1])
{
    cplx F[ORC_LMAX + 2][ORC_LMAX + 2]; /* factors up to one extra power on either side */
    {
        double p = a + b;
        double mu = a * b / p;
        double Px = (a * Ax + b * Bx) / p;
        double PA = Px - Ax, PB = Px - Bx;
        double H[2 * ORC_LMAX + 4];
        int n = la + lb + 2;
        double sp = sqrt(p);
        hermite(n, g / (2.0 * sp), H);
        cplx base = exp(-mu * (Ax - Bx) * (Ax - Bx)) * sqrt(M_PI / p) * exp(-g * g / (4.0 * p)) * cexp(-I * g * Px);
        cplx Tk[2 * ORC_LMAX + 4];
        cplx fac = 1.0;
        for (int k = 0; k <= n; ++k) {
            Tk[k] = base * fac * H[k];
            fac *= -I / (2.0 * sp);
        }
        for (int i = 0; i <= la + 1; ++i)
            for (int j = 0; j <= lb + 1; ++j) {
                cplx s = 0.0;
                for (int r = 0; r <= i; ++r)
                    for (int t = 0; t <= j; ++t)
                        s += binom(i, r) * binom(j, t) * ipow(PA, i - r) * ipow(PB, j - t) * Tk[r + t];
                F[i][j] = s;
            }
    }
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            dA[i][j] = 2.0 * a * F[i + 1][j] - (i > 0 ? i * F[i - 1][j] : 0.0);
            dB[i][j] = 2.0 * b * F[i][j + 1] - (j > 0 ? j * F[i][j - 1] : 0.0);
        }
}

/* d/dA_x and d/dB'_x (x = 0,1,2) of one primitive pair's transform block:
 * outA/outB [3][nfa*nfb]. */
static void prim_pair_ft_grad(const OShell* sa, int ka, const double* A, const OShell* sb, int kb, const double* Bs,
                              const double G[3], cplx* outA, cplx* outB, int nfab)
{
    double a = sa->ex[ka], b = sb->ex[kb];
    cplx F[3][ORC_LMAX + 1][ORC_LMAX + 1], dA[3][ORC_LMAX + 1][ORC_LMAX + 1], dB[3][ORC_LMAX + 1][ORC_LMAX + 1];
    for (int x = 0; x < 3; ++x) {
        factors1d(sa->l, sb->l, a, A[x], b, Bs[x], G[x], F[x]);
        factors1d_deriv(sa->l, sb->l, a, A[x], b, Bs[x], G[x], dA[x], dB[x]);
    }
    double dd = sa->co[ka] * sb->co[kb];
    for (int dir = 0; dir < 3; ++dir)
        for (int side = 0; side < 2; ++side) {
            cplx C[ORC_MAXC][ORC_MAXC];
            for (int ca = 0; ca < sa->nc; ++ca)
                for (int cb = 0; cb < sb->nc; ++cb) {
                    cplx v = 1.0;
                    for (int x = 0; x < 3; ++x) {
                        int i = sa->cx[ca][x], j = sb->cx[cb][x];
                        v *= (x == dir) ? (side == 0 ? dA[x][i][j] : dB[x][i][j]) : F[x][i][j];
                    }
                    C[ca][cb] = v;
                }
            cplx* out = (side == 0 ? outA : outB) + (size_t)dir * nfab;
            for (int fa = 0; fa < sa->nf; ++fa)
                for (int fb = 0; fb < sb->nf; ++fb) {
                    cplx sum = 0.0;
                    for (int ca = 0; ca < sa->nc; ++ca) {
                        if (sa->U[fa][ca] == 0.0) continue;
                        for (int cb = 0; cb < sb->nc; ++cb)
                            if (sb->U[fb][cb] != 0.0) sum += sa->U[fa][ca] * sb->U[fb][cb] * C[ca][cb];
                    }
                    out[fa * sb->nf + fb] += dd * sa->nrm[ka * sa->nf + fa] * sb->nrm[kb * sb->nf + fb] * sum;
                }
        }
}

/* transform of one primitive pair: out[fa*nfb + fb] += d_a d_b N N int ... */
static void prim_pair_ft(const OShell* sa, int ka, const double* A, const OShell* sb, int kb, const double* Bs,
                         const double G[3], cplx* out /* [nfa][nfb] */)
{
    double a = sa->ex[ka], b = sb->ex[kb];
    cplx F[3][ORC_LMAX + 1][ORC_LMAX + 1];
    for (int x = 0; x < 3; ++x) factors1d(sa->l, sb->l, a, A[x], b, Bs[x], G[x], F[x]);
    cplx C[ORC_MAXC][ORC_MAXC];
    for (int ca = 0; ca < sa->nc; ++ca)
        for (int cb = 0; cb < sb->nc; ++cb)
            C[ca][cb] = F[0][sa->cx[ca][0]][sb->cx[cb][0]] * F[1][sa->cx[ca][1]][sb->cx[cb][1]] *
                        F[2][sa->cx[ca][2]][sb->cx[cb][2]];
    /* two-stage transform to the shell functions */
    cplx T1[2 * ORC_LMAX + 1][ORC_MAXC];
    for (int fa = 0; fa < sa->nf; ++fa)
        for (int cb = 0; cb < sb->nc; ++cb) {
            cplx s = 0.0;
            for (int ca = 0; ca < sa->nc; ++ca)
                if (sa->U[fa][ca] != 0.0) s += sa->U[fa][ca] * C[ca][cb];
            T1[fa][cb] = s;
        }
    double dd = sa->co[ka] * sb->co[kb];
    for (int fa = 0; fa < sa->nf; ++fa)
        for (int fb = 0; fb < sb->nf; ++fb) {
            cplx s = 0.0;
            for (int cb = 0; cb < sb->nc; ++cb)
                if (sb->U[fb][cb] != 0.0) s += sb->U[fb][cb] * T1[fa][cb];
            out[fa * sb->nf + fb] += dd * sa->nrm[ka * sa->nf + fa] * sb->nrm[kb * sb->nf + fb] * s;
        }
}

/* ------------------------------------------------------------------------ */
/* pair list and G sphere                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int sa, ka, sb, kb, L[3];
} OPair;

static double prim_overlap_screen(double a, double b, double r2)
{
    double p = a + b;
    return pow(2.0 * sqrt(a * b) / p, 1.5) * exp(-a * b / p * r2);
}

static long enumerate_pairs(const OSys* S, double thresh, OPair** out)
{
    long cap = 1024, n = 0;
    OPair* P = (OPair*)malloc(sizeof(OPair) * (size_t)cap);
    double bn[3];
    for (int i = 0; i < 3; ++i) bn[i] = sqrt(S->M[i][i]);
    for (int sa = 0; sa < S->nsh; ++sa)
        for (int sb = 0; sb < S->nsh; ++sb) {
            const OShell* ha = &S->sh[sa];
            const OShell* hb = &S->sh[sb];
            const double* A = S->xyz + 3 * ha->cen;
            const double* B = S->xyz + 3 * hb->cen;
            double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
            double dab = sqrt(AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2]);
            for (int ka = 0; ka < ha->np; ++ka)
                for (int kb = 0; kb < hb->np; ++kb) {
                    double a = ha->ex[ka], b = hb->ex[kb];
                    double p = a + b, mu = a * b / p;
                    double s0 = pow(2.0 * sqrt(a * b) / p, 1.5);
                    if (!(s0 > thresh)) continue;
                    double rmax = sqrt(log(s0 / thresh) / mu);
                    int lim[3];
                    for (int i = 0; i < 3; ++i) lim[i] = (int)ceil((dab + rmax) * bn[i] / (2.0 * M_PI)) + 1;
                    for (int L1 = -lim[0]; L1 <= lim[0]; ++L1)
                        for (int L2 = -lim[1]; L2 <= lim[1]; ++L2)
                            for (int L3 = -lim[2]; L3 <= lim[2]; ++L3) {
                                double R[3];
                                for (int x = 0; x < 3; ++x)
                                    R[x] = AB[x] - (L1 * S->A[0][x] + L2 * S->A[1][x] + L3 * S->A[2][x]);
                                double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
                                if (!(prim_overlap_screen(a, b, r2) > thresh)) continue;
                                if (n == cap) {
                                    cap *= 2;
                                    P = (OPair*)realloc(P, sizeof(OPair) * (size_t)cap);
                                }
                                P[n].sa = sa;
                                P[n].ka = ka;
                                P[n].sb = sb;
                                P[n].kb = kb;
                                P[n].L[0] = L1;
                                P[n].L[1] = L2;
                                P[n].L[2] = L3;
                                ++n;
                            }
                }
        }
    *out = P;
    return n;
}

static double gnorm2(const OSys* S, const int n[3])
{
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += n[i] * S->M[i][j] * n[j];
    return s;
}

static long enumerate_g(const OSys* S, double gcut, int** out)
{
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        double an = sqrt(S->A[i][0] * S->A[i][0] + S->A[i][1] * S->A[i][1] + S->A[i][2] * S->A[i][2]);
        lim[i] = (int)floor(gcut * an / (2.0 * M_PI)) + 1;
    }
    long cap = 1024, n = 0;
    int* g = (int*)malloc(sizeof(int) * 3 * (size_t)cap);
    double gc2 = gcut * gcut;
    for (int n1 = -lim[0]; n1 <= lim[0]; ++n1)
        for (int n2 = -lim[1]; n2 <= lim[1]; ++n2)
            for (int n3 = -lim[2]; n3 <= lim[2]; ++n3) {
                if (n1 == 0 && n2 == 0 && n3 == 0) continue;
                int v[3] = {n1, n2, n3};
                if (!(gnorm2(S, v) < gc2)) continue;
                if (n == cap) {
                    cap *= 2;
                    g = (int*)realloc(g, sizeof(int) * 3 * (size_t)cap);
                }
                g[3 * n] = n1;
                g[3 * n + 1] = n2;
                g[3 * n + 2] = n3;
                ++n;
            }
    *out = g;
    return n;
}

static void gvec(const OSys* S, const int n[3], double G[3])
{
    for (int x = 0; x < 3; ++x) G[x] = n[0] * S->B[0][x] + n[1] * S->B[1][x] + n[2] * S->B[2][x];
}

static int wrap(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* exported entry points                                                     */
/* ------------------------------------------------------------------------ */

#define ORC_BASIS_ARGS                                                                                     \
    const double *A, int ncen, const double *xyz, int nsh, const int *sh_cen, const int *sh_l,             \
        const int *sh_sph, const int *sh_np, const int *sh_off, const double *exps, const double *coefs
#define ORC_BASIS_PASS A, ncen, xyz, nsh, sh_cen, sh_l, sh_sph, sh_np, sh_off, exps, coefs

int orc_nao(ORC_BASIS_ARGS)
{
    OSys S;
    int rc = build_system(&S, ORC_BASIS_PASS);
    int nao = S.nao;
    free_system(&S);
    return rc ? rc : nao;
}

/* reciprocal lattice (rows) and volume */
int orc_reciprocal(const double* A, double* B_out, double* vol_out)
{
    OSys S;
    int rc = build_system(&S, A, 0, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    if (rc) return rc;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B_out[3 * i + j] = S.B[i][j];
    *vol_out = S.vol;
    free_system(&S);
    return 0;
}

/* Full G sphere (n != 0, |G|^2 < gcut^2).  Returns the count; writes at most
 * cap triples into n_out (may be NULL to query the count). */
long orc_gsphere(const double* A, double gcut, long cap, int* n_out)
{
    OSys S;
    if (build_system(&S, A, 0, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL)) return -1;
    int* g = NULL;
    long n = enumerate_g(&S, gcut, &g);
    if (n_out) memcpy(n_out, g, sizeof(int) * 3 * (size_t)(n < cap ? n : cap));
    free(g);
    free_system(&S);
    return n;
}

/* Screened ordered primitive-shell pairs as 7-tuples (sa, ka, sb, kb, L1, L2, L3). */
long orc_pairs(ORC_BASIS_ARGS, double thresh, long cap, int* out7)
{
    OSys S;
    if (build_system(&S, ORC_BASIS_PASS)) return -1;
    OPair* P = NULL;
    long n = enumerate_pairs(&S, thresh, &P);
    if (out7)
        for (long i = 0; i < n && i < cap; ++i) {
            out7[7 * i + 0] = P[i].sa;
            out7[7 * i + 1] = P[i].ka;
            out7[7 * i + 2] = P[i].sb;
            out7[7 * i + 3] = P[i].kb;
            out7[7 * i + 4] = P[i].L[0];
            out7[7 * i + 5] = P[i].L[1];
            out7[7 * i + 6] = P[i].L[2];
        }
    free(P);
    free_system(&S);
    return n;
}

/* (mu0 nuL|G) for every function pair of shells sa, sb at one Cartesian G,
 * summed over the primitive pairs passing thresh (thresh <= 0: all).
 * out: complex interleaved [nf(sa)][nf(sb)]. */
int orc_pair_ft(ORC_BASIS_ARGS, int sa, int sb, const int* L, const double* G, double thresh, double* out)
{
    OSys S;
    if (build_system(&S, ORC_BASIS_PASS)) return -1;
    const OShell* ha = &S.sh[sa];
    const OShell* hb = &S.sh[sb];
    const double* Ac = xyz + 3 * ha->cen;
    double Bs[3];
    for (int x = 0; x < 3; ++x)
        Bs[x] = xyz[3 * hb->cen + x] + L[0] * S.A[0][x] + L[1] * S.A[1][x] + L[2] * S.A[2][x];
    cplx blk[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC];
    memset(blk, 0, sizeof(blk));
    double r2 = 0.0;
    for (int x = 0; x < 3; ++x) r2 += (Ac[x] - Bs[x]) * (Ac[x] - Bs[x]);
    for (int ka = 0; ka < ha->np; ++ka)
        for (int kb = 0; kb < hb->np; ++kb) {
            if (thresh > 0 && !(prim_overlap_screen(ha->ex[ka], hb->ex[kb], r2) > thresh)) continue;
            prim_pair_ft(ha, ka, Ac, hb, kb, Bs, G, blk);
        }
    for (int i = 0; i < ha->nf * hb->nf; ++i) {
        out[2 * i] = creal(blk[i]);
        out[2 * i + 1] = cimag(blk[i]);
    }
    free_system(&S);
    return 0;
}

/* D^{0n} = (1/Nk) sum_k exp(-i k.R_n) D^k, complex interleaved in/out,
 * [ndens][Nk][nao][nao] -> [ndens][Ncell][nao][nao]. */
static void fold_density(int ndens, const int km[3], int nao, const cplx* Dk, cplx* D0n)
{
    int nk = km[0] * km[1] * km[2];
    size_t nn = (size_t)nao * nao;
    for (int d = 0; d < ndens; ++d)
        for (int c = 0; c < nk; ++c) {
            int n1 = c / (km[1] * km[2]), n2 = (c / km[2]) % km[1], n3 = c % km[2];
            cplx* out = D0n + ((size_t)d * nk + c) * nn;
            for (size_t e = 0; e < nn; ++e) out[e] = 0.0;
            for (int k = 0; k < nk; ++k) {
                int m1 = k / (km[1] * km[2]), m2 = (k / km[2]) % km[1], m3 = k % km[2];
                double th = 2.0 * M_PI *
                            ((double)m1 * n1 / km[0] + (double)m2 * n2 / km[1] + (double)m3 * n3 / km[2]);
                cplx ph = cexp(-I * th) / nk;
                const cplx* in = Dk + ((size_t)d * nk + k) * nn;
                for (size_t e = 0; e < nn; ++e) out[e] += ph * in[e];
            }
        }
}

int orc_fold_density(int ndens, const int* kmesh, int nao, const double* Dk, double* D0n)
{
    fold_density(ndens, kmesh, nao, (const cplx*)Dk, (cplx*)D0n);
    return 0;
}

/* A primitive is diffuse when its exponent lies below alpha_cut (Sec. 2.6,
 * Eq. "cd cutoff": alpha_cut = w^2/2 by default); a primitive pair density is
 * DD when both of its primitives are diffuse and compact (CC or CD) otherwise.
 * alpha_cut <= 0 makes every pair compact. */
static int pair_is_dd(const OShell* ha, int ka, const OShell* hb, int kb, double alpha_cut)
{
    return ha->ex[ka] < alpha_cut && hb->ex[kb] < alpha_cut;
}

/* The build with classified pair densities (Sec. 2.6).  An integral between
 * two compact pair densities takes the long-range kernel of the Ewald split,
 * v_LR(G) = 4 pi e^{-G^2/4w^2} / (Omega G^2); every integral with a DD
 * density on either side is taken entirely in reciprocal space with the
 * full-range kernel v_FR(G) = 4 pi / (Omega G^2), the G = 0 term removed.
 * With rho_C and rho_D the sums over the compact and the DD pairs:
 *   J^{0L}_{mu nu} (compact pair) = sum_G (mu0 nuL|G) [v_LR rho_C(-G) + v_FR rho_D(-G)]
 *   J^{0L}_{mu nu} (DD pair)      = sum_G (mu0 nuL|G) v_FR [rho_C(-G) + rho_D(-G)]
 *   E_J = 1/2 sum_G [v_LR rho_C rho_C(-G) + v_FR (rho_C rho_D(-G) + rho_D rho_C(-G) + rho_D rho_D(-G))]
 * (a contracted shell whose primitives straddle alpha_cut is split into its
 * compact and diffuse parts, which the per-primitive-pair sums do by
 * themselves).  alpha_cut <= 0 is the plain long-range build.  rho_out gets
 * rho_C, rhoD_out (may be NULL) rho_D. */
static int lrj_core(ORC_BASIS_ARGS, const int* kmesh, double omega, double gcut, double pair_thresh,
                    double alpha_cut, int ndens, const double* Dk_in, double* Jk_out, double* EJ_out,
                    double* rho_out, double* rhoD_out, long g_cap, int* G_out, double* J0n_out, int pair_stride,
                    int nthreads, double* stats)
{
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    OSys S;
    int rc = build_system(&S, ORC_BASIS_PASS);
    if (rc) return rc;
    if (!(omega > 0.0) || !(gcut > 0.0) || pair_stride < 1) {
        free_system(&S);
        return -4;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int nao = S.nao;
    int nk = kmesh[0] * kmesh[1] * kmesh[2];
    size_t nn = (size_t)nao * nao;

    cplx* D0n = (cplx*)malloc(sizeof(cplx) * (size_t)ndens * nk * nn);
    fold_density(ndens, kmesh, nao, (const cplx*)Dk_in, D0n);

    int* gl = NULL;
    long nG = enumerate_g(&S, gcut, &gl);
    if (G_out) memcpy(G_out, gl, sizeof(int) * 3 * (size_t)(nG < g_cap ? nG : g_cap));
    double* Gc = (double*)malloc(sizeof(double) * 3 * (size_t)(nG > 0 ? nG : 1));
    double* vG = (double*)malloc(sizeof(double) * (size_t)(nG > 0 ? nG : 1));
    double* vF = (double*)malloc(sizeof(double) * (size_t)(nG > 0 ? nG : 1));
    long* neg = (long*)malloc(sizeof(long) * (size_t)(nG > 0 ? nG : 1));
    for (long g = 0; g < nG; ++g) {
        gvec(&S, gl + 3 * g, Gc + 3 * g);
        double g2 = gnorm2(&S, gl + 3 * g);
        vG[g] = 4.0 * M_PI * exp(-g2 / (4.0 * omega * omega)) / (S.vol * g2);
        vF[g] = 4.0 * M_PI / (S.vol * g2);
        neg[g] = -1;
    }
    /* index of -G (searched plainly) */
    for (long g = 0; g < nG; ++g)
        for (long h = 0; h < nG; ++h)
            if (gl[3 * h] == -gl[3 * g] && gl[3 * h + 1] == -gl[3 * g + 1] && gl[3 * h + 2] == -gl[3 * g + 2]) {
                neg[g] = h;
                break;
            }

    OPair* P = NULL;
    long np_all = enumerate_pairs(&S, pair_thresh, &P);
    long npr = (np_all + pair_stride - 1) / pair_stride;

    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    /* per thread: rho_C in the first ndens * nG entries, rho_D in the next */
    cplx* rho_t = (cplx*)calloc((size_t)nthr * 2 * ndens * (size_t)(nG > 0 ? nG : 1), sizeof(cplx));

    /* --- step 1: rho_C(G) and rho_D(G) ------------------------------------- */
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        cplx blk[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC];
#pragma omp for schedule(static)
        for (long ip = 0; ip < npr; ++ip) {
            const OPair* q = &P[ip * pair_stride];
            const OShell* ha = &S.sh[q->sa];
            const OShell* hb = &S.sh[q->sb];
            const int dd = pair_is_dd(ha, q->ka, hb, q->kb, alpha_cut);
            cplx* my = rho_t + ((size_t)tid * 2 + (size_t)dd) * ndens * nG;
            const double* Ac = xyz + 3 * ha->cen;
            double Bs[3];
            for (int x = 0; x < 3; ++x)
                Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
            int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] +
                       wrap(q->L[2], kmesh[2]);
            for (long g = 0; g < nG; ++g) {
                memset(blk, 0, sizeof(cplx) * (size_t)(ha->nf * hb->nf));
                prim_pair_ft(ha, q->ka, Ac, hb, q->kb, Bs, Gc + 3 * g, blk);
                for (int d = 0; d < ndens; ++d) {
                    const cplx* Dc = D0n + ((size_t)d * nk + cell) * nn;
                    cplx s = 0.0;
                    for (int fa = 0; fa < ha->nf; ++fa)
                        for (int fb = 0; fb < hb->nf; ++fb)
                            s += Dc[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb] * blk[fa * hb->nf + fb];
                    my[(size_t)d * nG + g] += s;
                }
            }
        }
    }
    cplx* rho = (cplx*)calloc((size_t)ndens * (size_t)(nG > 0 ? nG : 1), sizeof(cplx));
    cplx* rhoD = (cplx*)calloc((size_t)ndens * (size_t)(nG > 0 ? nG : 1), sizeof(cplx));
    for (int t = 0; t < nthr; ++t)
        for (size_t e = 0; e < (size_t)ndens * nG; ++e) {
            rho[e] += rho_t[((size_t)t * 2) * ndens * nG + e];
            rhoD[e] += rho_t[((size_t)t * 2 + 1) * ndens * nG + e];
        }
    free(rho_t);

    /* --- step 2-3: J^{0L} per pair, then J^k and the folded J^{0n} ---------- */
    int maxf = 2 * ORC_LMAX + 1 > ORC_MAXC ? 2 * ORC_LMAX + 1 : ORC_MAXC;
    size_t bsz = (size_t)maxf * maxf;
    cplx* Jp = (cplx*)calloc((size_t)(npr > 0 ? npr : 1) * ndens * bsz, sizeof(cplx));
#pragma omp parallel
    {
        cplx blk[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC];
#pragma omp for schedule(static)
        for (long ip = 0; ip < npr; ++ip) {
            const OPair* q = &P[ip * pair_stride];
            const OShell* ha = &S.sh[q->sa];
            const OShell* hb = &S.sh[q->sb];
            const double* Ac = xyz + 3 * ha->cen;
            double Bs[3];
            for (int x = 0; x < 3; ++x)
                Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
            int nfab = ha->nf * hb->nf;
            const int dd = pair_is_dd(ha, q->ka, hb, q->kb, alpha_cut);
            for (long g = 0; g < nG; ++g) {
                memset(blk, 0, sizeof(cplx) * (size_t)nfab);
                prim_pair_ft(ha, q->ka, Ac, hb, q->kb, Bs, Gc + 3 * g, blk);
                for (int d = 0; d < ndens; ++d) {
                    const cplx rc = rho[(size_t)d * nG + neg[g]], rd = rhoD[(size_t)d * nG + neg[g]];
                    cplx w = dd ? vF[g] * (rc + rd) : vG[g] * rc + vF[g] * rd;
                    cplx* out = Jp + ((size_t)ip * ndens + d) * bsz;
                    for (int e = 0; e < nfab; ++e) out[e] += w * blk[e];
                }
            }
        }
    }
    cplx* Jk = (cplx*)Jk_out;
    memset(Jk, 0, sizeof(cplx) * (size_t)ndens * nk * nn);
    cplx* J0n = (cplx*)J0n_out;
    if (J0n) memset(J0n, 0, sizeof(cplx) * (size_t)ndens * nk * nn);
    for (long ip = 0; ip < npr; ++ip) {
        const OPair* q = &P[ip * pair_stride];
        const OShell* ha = &S.sh[q->sa];
        const OShell* hb = &S.sh[q->sb];
        int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] +
                   wrap(q->L[2], kmesh[2]);
        for (int d = 0; d < ndens; ++d) {
            const cplx* blk = Jp + ((size_t)ip * ndens + d) * bsz;
            for (int k = 0; k < nk; ++k) {
                int m1 = k / (kmesh[1] * kmesh[2]), m2 = (k / kmesh[2]) % kmesh[1], m3 = k % kmesh[2];
                double th = 2.0 * M_PI *
                            ((double)m1 * q->L[0] / kmesh[0] + (double)m2 * q->L[1] / kmesh[1] +
                             (double)m3 * q->L[2] / kmesh[2]);
                cplx ph = cexp(I * th);
                cplx* out = Jk + ((size_t)d * nk + k) * nn;
                for (int fa = 0; fa < ha->nf; ++fa)
                    for (int fb = 0; fb < hb->nf; ++fb)
                        out[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb] += ph * blk[fa * hb->nf + fb];
            }
            if (J0n) {
                cplx* out = J0n + ((size_t)d * nk + cell) * nn;
                for (int fa = 0; fa < ha->nf; ++fa)
                    for (int fb = 0; fb < hb->nf; ++fb)
                        out[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb] += blk[fa * hb->nf + fb];
            }
        }
    }
    free(Jp);

    /* --- energy ----------------------------------------------------------- */
    for (int d = 0; d < ndens; ++d) {
        cplx e = 0.0;
        for (long g = 0; g < nG; ++g) {
            const cplx c = rho[(size_t)d * nG + g], cm = rho[(size_t)d * nG + neg[g]];
            const cplx q = rhoD[(size_t)d * nG + g], qm = rhoD[(size_t)d * nG + neg[g]];
            e += vG[g] * c * cm + vF[g] * (c * qm + q * cm + q * qm);
        }
        EJ_out[d] = 0.5 * creal(e);
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(cplx) * (size_t)ndens * nG);
    if (rhoD_out) memcpy(rhoD_out, rhoD, sizeof(cplx) * (size_t)ndens * nG);

    clock_gettime(CLOCK_MONOTONIC, &t1);
    if (stats) {
        stats[0] = (double)npr;
        stats[1] = (double)nG;
        stats[2] = (double)npr * (double)nG;
        stats[3] = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    }
    free(rho);
    free(rhoD);
    free(P);
    free(neg);
    free(vF);
    free(vG);
    free(Gc);
    free(gl);
    free(D0n);
    free_system(&S);
    return 0;
}

/* The whole long-range build.  Outputs (any may be NULL except Jk/EJ):
 *   Jk     complex [ndens][Nk][nao][nao]
 *   EJ     [ndens]
 *   rho    complex [ndens][nG] in the order of G_out
 *   G_out  int [nG][3]
 *   J0n    complex [ndens][Ncell][nao][nao] (J^{0L} folded into the BvK cells)
 * pair_stride > 1 processes every pair_stride-th pair only (timing samples;
 * the results are then not the build).  stats[0..3] = npairs (ordered
 * primitive-shell pairs used), nG, pair*G units per pass, wall seconds. */
int orc_lrj(ORC_BASIS_ARGS, const int* kmesh, double omega, double gcut, double pair_thresh, int ndens,
            const double* Dk_in, double* Jk_out, double* EJ_out, double* rho_out, long g_cap, int* G_out,
            double* J0n_out, int pair_stride, int nthreads, double* stats)
{
    return lrj_core(ORC_BASIS_PASS, kmesh, omega, gcut, pair_thresh, 0.0, ndens, Dk_in, Jk_out, EJ_out, rho_out,
                    NULL, g_cap, G_out, J0n_out, pair_stride, nthreads, stats);
}

/* The classified build (see lrj_core): rhoC_out and rhoD_out complex
 * [ndens][nG] in the order of G_out. */
int orc_lrj_classified(ORC_BASIS_ARGS, const int* kmesh, double omega, double gcut, double pair_thresh,
                       double alpha_cut, int ndens, const double* Dk_in, double* Jk_out, double* EJ_out,
                       double* rhoC_out, double* rhoD_out, long g_cap, int* G_out, double* J0n_out, int nthreads)
{
    return lrj_core(ORC_BASIS_PASS, kmesh, omega, gcut, pair_thresh, alpha_cut, ndens, Dk_in, Jk_out, EJ_out,
                    rhoC_out, rhoD_out, g_cap, G_out, J0n_out, 1, nthreads, NULL);
}

/* rho at listed reciprocal vectors (n triples), full pair loop; used to check
 * large systems at sampled G.  rho_out: complex [ndens][nGs]. */
int orc_rho_at(ORC_BASIS_ARGS, const int* kmesh, double pair_thresh, int ndens, const double* Dk_in, int nGs,
               const int* n_list, double* rho_out, int nthreads)
{
    OSys S;
    int rc = build_system(&S, ORC_BASIS_PASS);
    if (rc) return rc;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int nao = S.nao;
    int nk = kmesh[0] * kmesh[1] * kmesh[2];
    size_t nn = (size_t)nao * nao;
    cplx* D0n = (cplx*)malloc(sizeof(cplx) * (size_t)ndens * nk * nn);
    fold_density(ndens, kmesh, nao, (const cplx*)Dk_in, D0n);
    OPair* P = NULL;
    long np_all = enumerate_pairs(&S, pair_thresh, &P);
    cplx* rho = (cplx*)rho_out;
    memset(rho, 0, sizeof(cplx) * (size_t)ndens * nGs);
    for (int g = 0; g < nGs; ++g) {
        double G[3];
        gvec(&S, n_list + 3 * g, G);
        double accr[64] = {0}, acci[64] = {0};
        int nd = ndens < 64 ? ndens : 64;
#pragma omp parallel for schedule(static) reduction(+ : accr[:64], acci[:64])
        for (long ip = 0; ip < np_all; ++ip) {
            const OPair* q = &P[ip];
            const OShell* ha = &S.sh[q->sa];
            const OShell* hb = &S.sh[q->sb];
            const double* Ac = xyz + 3 * ha->cen;
            double Bs[3];
            for (int x = 0; x < 3; ++x)
                Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
            int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] +
                       wrap(q->L[2], kmesh[2]);
            cplx blk[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC];
            memset(blk, 0, sizeof(cplx) * (size_t)(ha->nf * hb->nf));
            prim_pair_ft(ha, q->ka, Ac, hb, q->kb, Bs, G, blk);
            for (int d = 0; d < nd; ++d) {
                const cplx* Dc = D0n + ((size_t)d * nk + cell) * nn;
                cplx s = 0.0;
                for (int fa = 0; fa < ha->nf; ++fa)
                    for (int fb = 0; fb < hb->nf; ++fb)
                        s += Dc[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb] * blk[fa * hb->nf + fb];
                accr[d] += creal(s);
                acci[d] += cimag(s);
            }
        }
        for (int d = 0; d < nd; ++d) rho[(size_t)d * nGs + g] = accr[d] + I * acci[d];
    }
    free(P);
    free(D0n);
    free_system(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* GPW: the DD density on a real-space grid (Sec. 2.6, App. E)               */
/* ------------------------------------------------------------------------ */

/* Functions of shell h built on its primitive k (contraction coefficient and
 * unit-self-overlap scale included) at the displacement u = r - centre. */
static void shell_values(const OShell* h, int k, const double u[3], double* out /* [nf] */)
{
    double e = exp(-h->ex[k] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    for (int f = 0; f < h->nf; ++f) {
        double s = 0.0;
        for (int c = 0; c < h->nc; ++c)
            if (h->U[f][c] != 0.0)
                s += h->U[f][c] * ipow(u[0], h->cx[c][0]) * ipow(u[1], h->cx[c][1]) * ipow(u[2], h->cx[c][2]);
        out[f] = h->co[k] * h->nrm[k * h->nf + f] * s * e;
    }
}

/* The density of the DD pairs on the grid r_m = sum_i (m_i / N_i) a_i,
 * m_i = 0..N_i-1 (App. E, Eq. "rho_shellpair"):
 *   rho_D(r) = sum_{DD pairs (a in mu, b in nu, L)} Re D^{0[L]}_{mu nu}
 *              sum_T chi_a(r - A - T) chi_b(r - B - R_L - T),
 * the ordered DD pairs of the screened list, T over the lattice translations
 * whose product Gaussian e^{-p |r - P - T|^2} exceeds e^{-50}.  D^{0n} is real
 * for time-reversal symmetric input; its imaginary part is not used.
 * out: double [ndens][N1][N2][N3]. */
int orc_gpw_density(ORC_BASIS_ARGS, const int* kmesh, double pair_thresh, double alpha_cut, int ndens,
                    const double* Dk_in, const int* grid, double* out, int nthreads)
{
    OSys S;
    int rc = build_system(&S, ORC_BASIS_PASS);
    if (rc) return rc;
    if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1) {
        free_system(&S);
        return -4;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    const int nao = S.nao;
    const int nk = kmesh[0] * kmesh[1] * kmesh[2];
    const size_t nn = (size_t)nao * nao;
    cplx* D0n = (cplx*)malloc(sizeof(cplx) * (size_t)ndens * nk * nn);
    fold_density(ndens, kmesh, nao, (const cplx*)Dk_in, D0n);
    OPair* P = NULL;
    long np_all = enumerate_pairs(&S, pair_thresh, &P);
    long ndd = 0;
    for (long i = 0; i < np_all; ++i)
        if (pair_is_dd(&S.sh[P[i].sa], P[i].ka, &S.sh[P[i].sb], P[i].kb, alpha_cut)) P[ndd++] = P[i];
    const long npts = (long)grid[0] * grid[1] * grid[2];
    memset(out, 0, sizeof(double) * (size_t)ndens * npts);
#pragma omp parallel for schedule(dynamic, 16)
    for (long m = 0; m < npts; ++m) {
        const int m1 = (int)(m / ((long)grid[1] * grid[2])), m2 = (int)((m / grid[2]) % grid[1]),
                  m3 = (int)(m % grid[2]);
        double r[3];
        for (int x = 0; x < 3; ++x)
            r[x] = (double)m1 / grid[0] * S.A[0][x] + (double)m2 / grid[1] * S.A[1][x] +
                   (double)m3 / grid[2] * S.A[2][x];
        double va[2 * ORC_LMAX + 1], vb[2 * ORC_LMAX + 1];
        for (long ip = 0; ip < ndd; ++ip) {
            const OPair* q = &P[ip];
            const OShell* ha = &S.sh[q->sa];
            const OShell* hb = &S.sh[q->sb];
            const double a = ha->ex[q->ka], b = hb->ex[q->kb], p = a + b;
            const double* Ac = xyz + 3 * ha->cen;
            double Bs[3], Pc[3];
            for (int x = 0; x < 3; ++x) {
                Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
                Pc[x] = (a * Ac[x] + b * Bs[x]) / p;
            }
            const int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] +
                             wrap(q->L[2], kmesh[2]);
            const double rs = sqrt(50.0 / p);
            int tlo[3], thi[3];
            for (int i = 0; i < 3; ++i) {
                /* fractional coordinate of r - P along a_i, and the reach of the radius rs */
                double phi = 0.0;
                for (int x = 0; x < 3; ++x) phi += S.B[i][x] * (r[x] - Pc[x]);
                phi /= 2.0 * M_PI;
                double reach = rs * sqrt(S.M[i][i]) / (2.0 * M_PI);
                tlo[i] = (int)ceil(phi - reach);
                thi[i] = (int)floor(phi + reach);
            }
            for (int t1 = tlo[0]; t1 <= thi[0]; ++t1)
                for (int t2 = tlo[1]; t2 <= thi[1]; ++t2)
                    for (int t3 = tlo[2]; t3 <= thi[2]; ++t3) {
                        double T[3], ua[3], ub[3], up2 = 0.0;
                        for (int x = 0; x < 3; ++x) {
                            T[x] = t1 * S.A[0][x] + t2 * S.A[1][x] + t3 * S.A[2][x];
                            ua[x] = r[x] - Ac[x] - T[x];
                            ub[x] = r[x] - Bs[x] - T[x];
                            double up = r[x] - Pc[x] - T[x];
                            up2 += up * up;
                        }
                        if (p * up2 > 50.0) continue;
                        shell_values(ha, q->ka, ua, va);
                        shell_values(hb, q->kb, ub, vb);
                        for (int d = 0; d < ndens; ++d) {
                            const cplx* Dc = D0n + ((size_t)d * nk + cell) * nn;
                            double s = 0.0;
                            for (int fa = 0; fa < ha->nf; ++fa)
                                for (int fb = 0; fb < hb->nf; ++fb)
                                    s += creal(Dc[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb]) * va[fa] * vb[fb];
                            out[(size_t)d * npts + m] += s;
                        }
                    }
        }
    }
    free(P);
    free(D0n);
    free_system(&S);
    return 0;
}

/* Solid-harmonic coefficients over Cartesian monomials, for the tests. */
int orc_solid_harmonic(int l, int m, double* coef)
{
    if (l < 0 || l > ORC_LMAX || m < -l || m > l) return -1;
    solid_harmonic(l, m, coef);
    return 0;
}

/* Per-function normalisation factor of one primitive of one shell, for the tests. */
int orc_norms(ORC_BASIS_ARGS, int s, int k, double* out)
{
    OSys S;
    if (build_system(&S, ORC_BASIS_PASS)) return -1;
    for (int f = 0; f < S.sh[s].nf; ++f) out[f] = S.sh[s].nrm[k * S.sh[s].nf + f];
    free_system(&S);
    return 0;
}

/* Nuclear gradient of the long-range energy, dE_J/dR_C for every centre C
 * (D^k fixed):  E_J = 1/2 sum_G v(G) rho(G) rho(-G), so
 *   dE_J/dR = 1/2 sum_G v(G) [drho(G)/dR rho(-G) + rho(G) drho(-G)/dR],
 * with drho/dR from the derivatives of the pair transforms with respect to
 * their two centres (the b centre sits at R_B + R_L).  grad_out: [ndens][ncen][3]. */
int orc_grad(ORC_BASIS_ARGS, const int* kmesh, double omega, double gcut, double pair_thresh, int ndens,
             const double* Dk_in, double* grad_out, int nthreads)
{
    OSys S;
    int rc = build_system(&S, ORC_BASIS_PASS);
    if (rc) return rc;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int nao = S.nao;
    int nk = kmesh[0] * kmesh[1] * kmesh[2];
    size_t nn = (size_t)nao * nao;
    cplx* D0n = (cplx*)malloc(sizeof(cplx) * (size_t)ndens * nk * nn);
    fold_density(ndens, kmesh, nao, (const cplx*)Dk_in, D0n);
    int* gl = NULL;
    long nG = enumerate_g(&S, gcut, &gl);
    double* Gc = (double*)malloc(sizeof(double) * 3 * (size_t)(nG > 0 ? nG : 1));
    double* vG = (double*)malloc(sizeof(double) * (size_t)(nG > 0 ? nG : 1));
    long* neg = (long*)malloc(sizeof(long) * (size_t)(nG > 0 ? nG : 1));
    for (long g = 0; g < nG; ++g) {
        gvec(&S, gl + 3 * g, Gc + 3 * g);
        double g2 = gnorm2(&S, gl + 3 * g);
        vG[g] = 4.0 * M_PI * exp(-g2 / (4.0 * omega * omega)) / (S.vol * g2);
        neg[g] = -1;
        for (long h = 0; h < nG; ++h)
            if (gl[3 * h] == -gl[3 * g] && gl[3 * h + 1] == -gl[3 * g + 1] && gl[3 * h + 2] == -gl[3 * g + 2]) {
                neg[g] = h;
                break;
            }
    }
    OPair* P = NULL;
    long np_all = enumerate_pairs(&S, pair_thresh, &P);
    /* rho(G) first (plain pair loop, as in orc_lrj) */
    cplx* rho = (cplx*)calloc((size_t)ndens * (size_t)(nG > 0 ? nG : 1), sizeof(cplx));
    for (long ip = 0; ip < np_all; ++ip) {
        const OPair* q = &P[ip];
        const OShell* ha = &S.sh[q->sa];
        const OShell* hb = &S.sh[q->sb];
        const double* Ac = xyz + 3 * ha->cen;
        double Bs[3];
        for (int x = 0; x < 3; ++x)
            Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
        int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] + wrap(q->L[2], kmesh[2]);
        cplx blk[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC];
        for (long g = 0; g < nG; ++g) {
            memset(blk, 0, sizeof(cplx) * (size_t)(ha->nf * hb->nf));
            prim_pair_ft(ha, q->ka, Ac, hb, q->kb, Bs, Gc + 3 * g, blk);
            for (int d = 0; d < ndens; ++d) {
                const cplx* Dc = D0n + ((size_t)d * nk + cell) * nn;
                cplx s = 0.0;
                for (int fa = 0; fa < ha->nf; ++fa)
                    for (int fb = 0; fb < hb->nf; ++fb)
                        s += Dc[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb] * blk[fa * hb->nf + fb];
                rho[(size_t)d * nG + g] += s;
            }
        }
    }
    int ncent = S.ncen;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double* gt = (double*)calloc((size_t)nthr * ndens * ncent * 3, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* my = gt + (size_t)tid * ndens * ncent * 3;
        cplx dA[3 * ((2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC)];
        cplx dB[3 * ((2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC)];
#pragma omp for schedule(static)
        for (long ip = 0; ip < np_all; ++ip) {
            const OPair* q = &P[ip];
            const OShell* ha = &S.sh[q->sa];
            const OShell* hb = &S.sh[q->sb];
            const double* Ac = xyz + 3 * ha->cen;
            double Bs[3];
            for (int x = 0; x < 3; ++x)
                Bs[x] = xyz[3 * hb->cen + x] + q->L[0] * S.A[0][x] + q->L[1] * S.A[1][x] + q->L[2] * S.A[2][x];
            int cell = (wrap(q->L[0], kmesh[0]) * kmesh[1] + wrap(q->L[1], kmesh[1])) * kmesh[2] +
                       wrap(q->L[2], kmesh[2]);
            int nfab = ha->nf * hb->nf;
            for (long g = 0; g < nG; ++g) {
                memset(dA, 0, sizeof(cplx) * 3 * (size_t)nfab);
                memset(dB, 0, sizeof(cplx) * 3 * (size_t)nfab);
                prim_pair_ft_grad(ha, q->ka, Ac, hb, q->kb, Bs, Gc + 3 * g, dA, dB, nfab);
                /* the same derivatives at -G are the complex conjugates only for real functions;
                   evaluate -G explicitly */
                double Gm[3] = {-Gc[3 * g], -Gc[3 * g + 1], -Gc[3 * g + 2]};
                cplx eA[3 * ((2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC)];
                cplx eB[3 * ((2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) + ORC_MAXC * ORC_MAXC)];
                memset(eA, 0, sizeof(cplx) * 3 * (size_t)nfab);
                memset(eB, 0, sizeof(cplx) * 3 * (size_t)nfab);
                prim_pair_ft_grad(ha, q->ka, Ac, hb, q->kb, Bs, Gm, eA, eB, nfab);
                for (int d = 0; d < ndens; ++d) {
                    const cplx* Dc = D0n + ((size_t)d * nk + cell) * nn;
                    cplx rp = rho[(size_t)d * nG + g], rm = rho[(size_t)d * nG + neg[g]];
                    for (int dir = 0; dir < 3; ++dir) {
                        cplx sa_ = 0.0, sb_ = 0.0, ta = 0.0, tb = 0.0;
                        for (int fa = 0; fa < ha->nf; ++fa)
                            for (int fb = 0; fb < hb->nf; ++fb) {
                                cplx Dv = Dc[(size_t)(ha->ao0 + fa) * nao + hb->ao0 + fb];
                                int e = dir * nfab + fa * hb->nf + fb;
                                sa_ += Dv * dA[e];
                                sb_ += Dv * dB[e];
                                ta += Dv * eA[e];
                                tb += Dv * eB[e];
                            }
                        /* 1/2 v [drho(G) rho(-G) + rho(G) drho(-G)] */
                        my[((size_t)d * ncent + ha->cen) * 3 + dir] += 0.5 * vG[g] * creal(sa_ * rm + rp * ta);
                        my[((size_t)d * ncent + hb->cen) * 3 + dir] += 0.5 * vG[g] * creal(sb_ * rm + rp * tb);
                    }
                }
            }
        }
    }
    memset(grad_out, 0, sizeof(double) * (size_t)ndens * ncent * 3);
    for (int t = 0; t < nthr; ++t)
        for (size_t e = 0; e < (size_t)ndens * ncent * 3; ++e) grad_out[e] += gt[(size_t)t * ndens * ncent * 3 + e];
    free(gt);
    free(rho);
    free(P);
    free(neg);
    free(vG);
    free(Gc);
    free(gl);
    free(D0n);
    free_system(&S);
    return 0;
}
