"""Pins that tie the FP64 CPU oracle to the paper and to mathematics.

Each test checks the oracle against something other than itself: closed
forms, Gauss-Hermite / grid quadrature, brute-force lattice sums, library
FFTs, and invariants the definitions imply.  A plausible slip in the oracle
(a sign of i, a dropped binomial term, a transposed operand, a wrong 1/Nk or
phase sign, a wrong solid-harmonic coefficient) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W
from tests import numerics as N


def one_shell_system(specs, A=None, spherical=True):
    """specs: list of (centre_xyz, l, alpha)."""
    cen = [s[0] for s in specs]
    shell_spec = [(i, s[1], [s[2]]) for i, s in enumerate(specs)]
    return W.tiny(A=A if A is not None else np.eye(3) * 30.0, centres=cen, shell_spec=shell_spec,
                  spherical=spherical)


# ---------------------------------------------------------------------------
# closed forms for the pair transform (Eq. "AFT for pair density")
# ---------------------------------------------------------------------------

def test_ss_closed_form(orc):
    """s-s: N_a N_b (pi/p)^{3/2} e^{-mu R^2} e^{-G^2/4p} e^{-iG.P}."""
    A = np.array([0.3, -0.2, 0.1])
    B = np.array([1.1, 0.4, -0.7])
    a, b = 1.3, 0.55
    w = one_shell_system([(A, 0, a), (B, 0, b)])
    p = a + b
    mu = a * b / p
    P = (a * A + b * B) / p
    Na = (2 * a / math.pi) ** 0.75
    Nb = (2 * b / math.pi) ** 0.75
    for G in [np.zeros(3), np.array([0.7, -0.3, 1.1]), np.array([-2.0, 1.5, 0.4])]:
        ref = Na * Nb * (math.pi / p) ** 1.5 * math.exp(-mu * np.sum((A - B) ** 2)) * \
            math.exp(-G @ G / (4 * p)) * np.exp(-1j * (G @ P))
        got = orc.pair_ft(w, 0, 1, [0, 0, 0], G, thresh=0.0)[0, 0]
        assert abs(got - ref) < 1e-14 * max(1.0, abs(ref))


def test_sp_closed_form_pins_sign_of_i(orc):
    """s-p_x: the s-s value times N_p/N_s-ratio times ((P_x-B_x) - i G_x/(2p)).

    This fixes the sign of i in the transform of a Cartesian Gaussian: the
    factor printed with +i in Eq. "FT of cart Gaussians" must be read as -i
    for the e^{-iG.r} transform of Eq. "AFT for pair density"."""
    A = np.array([0.0, 0.1, 0.0])
    B = np.array([0.9, -0.3, 0.4])
    a, b = 0.8, 1.7
    w = one_shell_system([(A, 0, a), (B, 1, b)], spherical=False)
    p = a + b
    mu = a * b / p
    P = (a * A + b * B) / p
    Na = (2 * a / math.pi) ** 0.75
    Nb = (2 * b / math.pi) ** 0.75 * math.sqrt(4 * b)
    G = np.array([0.9, -0.4, 0.6])
    base = Na * Nb * (math.pi / p) ** 1.5 * math.exp(-mu * np.sum((A - B) ** 2)) * \
        math.exp(-G @ G / (4 * p)) * np.exp(-1j * (G @ P))
    got = orc.pair_ft(w, 0, 1, [0, 0, 0], G, thresh=0.0)[0]
    for x in range(3):
        ref = base * ((P[x] - B[x]) - 1j * G[x] / (2 * p))
        assert abs(got[x] - ref) < 1e-14
    # the opposite sign of i is detectably wrong
    wrong = base * ((P[0] - B[0]) + 1j * G[0] / (2 * p))
    assert abs(got[0] - wrong) > 1e-3


# ---------------------------------------------------------------------------
# G -> 0 limit and quadrature
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("spherical", [True, False])
def test_g0_limit_is_overlap(orc, spherical):
    """(mu0 nuL|G=0) equals the overlap S_{mu nu}; functions unit-normalised.
    Overlaps by Gauss-Hermite quadrature; spherical functions from the
    textbook l<=2 forms."""
    rng = np.random.default_rng(5)
    for la, lb in itertools.product(range(3), range(3)):
        A = rng.normal(size=3) * 0.6
        B = rng.normal(size=3) * 0.6
        a, b = rng.uniform(0.3, 2.5, 2)
        w = one_shell_system([(A, la, a), (B, lb, b)], spherical=spherical)
        got = orc.pair_ft(w, 0, 1, [0, 0, 0], np.zeros(3), thresh=0.0)
        ref = N.shell_overlap(w.shells[0], A, w.shells[1], B)
        np.testing.assert_allclose(got.real, ref, atol=1e-13, rtol=0)
        assert np.abs(got.imag).max() < 1e-15
        # unit self-overlap
        s_aa = orc.pair_ft(w, 0, 0, [0, 0, 0], np.zeros(3), thresh=0.0)
        np.testing.assert_allclose(np.diag(s_aa.real), 1.0, atol=1e-13)


@pytest.mark.parametrize("la,lb", [(0, 1), (1, 1), (2, 0), (1, 2), (2, 2)])
def test_grid_fourier_transform(orc, la, lb):
    """Pair transform against a 3D grid sum of phi_a phi_b e^{-iG.r}."""
    rng = np.random.default_rng(10 * la + lb)
    A = rng.normal(size=3) * 0.5
    B = rng.normal(size=3) * 0.5
    a, b = rng.uniform(0.6, 1.6, 2)
    w = one_shell_system([(A, la, a), (B, lb, b)], spherical=True)
    for G in [np.array([0.8, -0.5, 0.3]), np.array([-1.7, 0.9, 2.1])]:
        got = orc.pair_ft(w, 0, 1, [0, 0, 0], G, thresh=0.0)
        ref = N.grid_ft(w.shells[0], A, w.shells[1], B, G, box=16.0, h=0.16)
        np.testing.assert_allclose(got, ref, atol=2e-11, rtol=0)


def test_lattice_translation_of_b(orc):
    """(mu0 nuL|G) is the transform of phi_mu(r) phi_nu(r - R_L)."""
    Acell = np.array([[6.0, 0.0, 0.0], [1.0, 5.5, 0.0], [0.5, 0.7, 6.5]])
    A = np.array([0.2, 0.1, -0.3])
    B = np.array([0.7, 0.9, 0.2])
    w = one_shell_system([(A, 1, 0.9), (B, 2, 0.7)], A=Acell)
    L = np.array([1, -1, 0])
    Bs = B + L @ Acell
    w2 = one_shell_system([(A, 1, 0.9), (Bs, 2, 0.7)], A=np.eye(3) * 40.0)
    G = np.array([0.4, -0.8, 0.5])
    got = orc.pair_ft(w, 0, 1, L, G, thresh=0.0)
    ref = orc.pair_ft(w2, 0, 1, [0, 0, 0], G, thresh=0.0)
    np.testing.assert_allclose(got, ref, atol=1e-15, rtol=1e-13)


# ---------------------------------------------------------------------------
# solid harmonics and normalisation
# ---------------------------------------------------------------------------

def test_solid_harmonics_textbook_l_le_2(orc):
    order = {0: [0], 1: [1, -1, 0], 2: [-2, -1, 0, 1, 2]}
    for l in range(3):
        for f, m in enumerate(order[l]):
            np.testing.assert_allclose(orc.solid_harmonic(l, m), N.TEXTBOOK_SPH[l][f], atol=1e-15)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_solid_harmonics_harmonic_and_orthogonal(orc, l):
    """Every S_lm is harmonic (Laplacian 0) and the set is orthogonal on the
    sphere with equal norms (Racah normalisation)."""
    carts = N.cart_list(l)

    rows = [orc.solid_harmonic(l, m) for m in range(-l, l + 1)]
    for coef in rows:
        lap = {}
        for c, v in zip(carts, coef):
            for ax in range(3):
                if c[ax] >= 2:
                    d = list(c)
                    d[ax] -= 2
                    lap[tuple(d)] = lap.get(tuple(d), 0.0) + v * c[ax] * (c[ax] - 1)
        assert max(abs(x) for x in lap.values()) < 1e-12 if lap else True
    # Gram matrix of the Gaussian-weighted functions at one exponent
    S = np.zeros((len(carts), len(carts)))
    for i, ci in enumerate(carts):
        for j, cj in enumerate(carts):
            S[i, j] = N.monomial_overlap(ci, 0.7, np.zeros(3), cj, 0.7, np.zeros(3))
    U = np.array(rows)
    Gm = U @ S @ U.T
    d = np.diag(Gm)
    np.testing.assert_allclose(Gm - np.diag(d), 0.0, atol=1e-12 * d.max())
    np.testing.assert_allclose(d, d[0], rtol=1e-12)



def test_norms_match_quadrature(orc):
    w = one_shell_system([(np.zeros(3), 2, 0.9)], spherical=False)
    nrm = orc.norms(w, 0)
    carts = N.cart_list(2)
    ref = [1.0 / math.sqrt(N.monomial_overlap(c, 0.9, np.zeros(3), c, 0.9, np.zeros(3))) for c in carts]
    np.testing.assert_allclose(nrm, ref, rtol=1e-13)


# ---------------------------------------------------------------------------
# G sphere, pair list, k <-> BvK transform
# ---------------------------------------------------------------------------

def test_gsphere_brute_force(orc):
    A = np.array([[6.0, 0.0, 0.0], [2.0, 5.0, 0.0], [-1.0, 1.5, 7.0]])
    gc = 2.9
    got = orc.gsphere(A, gc)
    B = 2 * np.pi * np.linalg.inv(A).T
    ref = []
    for n in itertools.product(range(-15, 16), repeat=3):
        if n == (0, 0, 0):
            continue
        G = np.array(n) @ B
        if G @ G < gc * gc:
            ref.append(n)
    assert sorted(map(tuple, got.tolist())) == sorted(ref)
    Bo, vol = orc.reciprocal(A)
    np.testing.assert_allclose(Bo @ A.T, 2 * np.pi * np.eye(3), atol=1e-13)
    assert abs(vol - abs(np.linalg.det(A))) < 1e-12


def test_pair_list_brute_force(orc):
    w = W.tiny(seed=3, A=np.array([[4.5, 0, 0], [0.8, 4.0, 0], [0.3, -0.6, 5.0]]),
               centres=[[0.0, 0.0, 0.0], [1.5, 1.2, 0.8]],
               shell_spec=[(0, 0, [0.25, 3.0]), (1, 1, [0.4]), (1, 0, [0.15])])
    got = sorted(map(tuple, orc.pairs(w).tolist()))
    ref = []
    for sa, ha in enumerate(w.shells):
        for sb, hb in enumerate(w.shells):
            a, b = ha.exps[0], hb.exps[0]
            p = a + b
            for L in itertools.product(range(-12, 13), repeat=3):
                R = w.xyz[ha.centre] - w.xyz[hb.centre] - np.array(L) @ w.A
                s = (2 * math.sqrt(a * b) / p) ** 1.5 * math.exp(-a * b / p * (R @ R))
                if s > w.pair_thresh:
                    ref.append((sa, 0, sb, 0) + L)
    assert got == sorted(ref)


def test_fold_density_matches_fft(orc):
    w = W.tiny(seed=4, kmesh=(2, 3, 2))
    got = orc.fold_density(w)
    Dk = w.Dk.reshape(w.ndens, 2, 3, 2, w.nao, w.nao)
    ref = np.fft.fftn(Dk, axes=(1, 2, 3)).reshape(w.ndens, 12, w.nao, w.nao) / 12.0
    np.testing.assert_allclose(got, ref, atol=1e-14)
    assert np.abs(got.imag).max() < 1e-14   # time-reversal symmetric input -> real D^{0n}


# ---------------------------------------------------------------------------
# whole-build pins
# ---------------------------------------------------------------------------

def test_erf_lattice_sum_brute_force(orc):
    """E_J of a neutral, dipole-free density of same-centre s Gaussians equals
    the brute-force real-space erf(omega r)/r lattice sum (the G=0 term is
    zero for such a density; Eq. "Ewald J", long-range term)."""
    A = np.array([[7.0, 0.0, 0.0], [1.2, 7.5, 0.0], [-0.8, 0.9, 8.0]])
    cen = [[0.3, 0.2, 0.1], [3.1, 4.2, 2.6]]
    spec = [(0, 0, [2.5, 1.2]), (1, 0, [1.6, 3.0])]
    w = W.tiny(seed=1, A=A, centres=cen, shell_spec=spec, omega=0.4, eps_g=1e-17, pair_thresh=1e-12)
    q = np.array([1.0, -1.0, 0.7, -0.7])
    D = np.diag(q).astype(np.complex128)[None, None]
    pl = orc.pairs(w)
    # only same-cell pairs survive between the charged functions
    for sa, _, sb, _, l1, l2, l3 in pl:
        if sa == sb:
            assert (l1, l2, l3) == (0, 0, 0)
    r = orc.lrj(w, Dk=D)
    charges = [(q[i], 2 * w.shells[i].exps[0], w.xyz[w.shells[i].centre]) for i in range(4)]
    ref = N.erf_lattice_energy(A, charges, 0.4, rmax=45.0)
    assert abs(r["EJ"][0] - ref) < 1e-12


def test_parseval_hermitian_and_trace(orc):
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    r = orc.lrj(w)
    Jk = r["Jk"]
    assert np.abs(Jk - np.conj(np.transpose(Jk, (0, 1, 3, 2)))).max() < 1e-13 * np.abs(Jk).max()
    for d in range(2):
        tr = sum(np.trace(w.Dk[d, k] @ Jk[d, k]) for k in range(w.nk)) / (2 * w.nk)
        assert abs(tr.imag) < 1e-13
        assert abs(tr.real - r["EJ"][d]) < 1e-12 * max(1.0, abs(r["EJ"][d]))
    # D^{0n} and J^{0n} are real for time-reversal symmetric input
    assert np.abs(r["J0n"].imag).max() < 1e-13


def test_linearity_and_bilinear_symmetry(orc):
    w = W.tiny(seed=8, kmesh=(1, 2, 1))
    w2 = W.tiny(seed=9, kmesh=(1, 2, 1))
    D1, D2 = w.Dk, w2.Dk
    J1 = orc.lrj(w, Dk=D1)["Jk"]
    J2 = orc.lrj(w, Dk=D2)["Jk"]
    J12 = orc.lrj(w, Dk=0.3 * D1 - 1.7 * D2)["Jk"]
    np.testing.assert_allclose(J12, 0.3 * J1 - 1.7 * J2, atol=1e-12 * np.abs(J12).max())
    t12 = sum(np.trace(D1[0, k] @ J2[0, k]) for k in range(w.nk))
    t21 = sum(np.trace(D2[0, k] @ J1[0, k]) for k in range(w.nk))
    assert abs(t12 - t21) < 1e-12 * abs(t12)


def test_rigid_translation_invariance(orc):
    w = W.tiny(seed=12, kmesh=(2, 1, 1))
    r0 = orc.lrj(w)
    w.xyz = w.xyz + np.array([0.37, -1.21, 2.05])
    r1 = orc.lrj(w)
    assert abs(r0["EJ"][0] - r1["EJ"][0]) < 1e-12
    np.testing.assert_allclose(r1["Jk"], r0["Jk"], atol=1e-12)


def test_supercell_folding_pins_k_conventions(orc):
    """N_k E_J(k-mesh, cell) = E_J(Gamma, BvK supercell whose density is built
    from D^{0n}); J of the supercell reproduces J^{0n}.  This fixes the sign
    and the 1/N_k of the k <-> BvK transforms (Eqs. "FT of J", "FT for D")."""
    km = (2, 1, 2)
    w = W.tiny(seed=13, kmesh=km, A=np.diag([4.2, 4.8, 4.4]), centres=[[0.1, 0.2, 0.3], [1.6, 1.9, 1.2]],
               shell_spec=[(0, 0, [1.4, 0.35]), (0, 1, [0.7]), (1, 0, [0.9]), (1, 1, [0.5])])
    r = orc.lrj(w)
    D0n = orc.fold_density(w)[0].real
    nk = w.nk
    cells = [(i, j, k) for i in range(km[0]) for j in range(km[1]) for k in range(km[2])]
    Asc = np.diag(km) @ w.A
    xyz_sc = np.vstack([w.xyz + np.array(c) @ w.A for c in cells])
    shells_sc = []
    for ci, _ in enumerate(cells):
        for s in w.shells:
            shells_sc.append(W.Shell(s.centre + ci * len(w.xyz), s.l, s.spherical, s.exps, s.coefs))
    nao = w.nao
    Dsc = np.zeros((nk * nao, nk * nao))
    for ci, c in enumerate(cells):
        for cj, cc in enumerate(cells):
            n = tuple((np.array(cc) - np.array(c)) % np.array(km))
            Dsc[ci * nao:(ci + 1) * nao, cj * nao:(cj + 1) * nao] = D0n[cells.index(n)]
    wsc = W.Workload("sc", Asc, xyz_sc, shells_sc, (1, 1, 1), w.omega, Dsc[None, None].astype(complex),
                     eps_g=w.eps_g, pair_thresh=w.pair_thresh)
    rsc = orc.lrj(wsc)
    assert abs(rsc["EJ"][0] - nk * r["EJ"][0]) < 1e-11 * max(1.0, abs(rsc["EJ"][0]))
    Jsc = rsc["Jk"][0, 0].real
    J0n = r["J0n"][0].real
    for ci, c in enumerate(cells):
        n = cells.index(tuple((np.array(c)) % np.array(km)))
        np.testing.assert_allclose(Jsc[0:nao, ci * nao:(ci + 1) * nao], J0n[n], atol=1e-11)


def test_gcut_convergence(orc):
    w = W.tiny(seed=14, kmesh=(1, 1, 2))
    e14 = orc.lrj(w)["EJ"][0]
    w.eps_g = 1e-18
    e18 = orc.lrj(w)["EJ"][0]
    assert abs(e14 - e18) < 1e-12 * max(1.0, abs(e14))


def test_cfg1_counts(orc):
    """Sizes of the Gamma-point 2-centre workload: 340 G-vectors, 1118 ordered pairs."""
    w = W.cfg1()
    assert len(orc.gsphere(w.A, orc.gcut_of(w))) == 340
    assert len(orc.pairs(w)) == 1118


def test_rho_at_matches_full_build(orc):
    """The sampled-rho entry used for large cells reproduces the pinned full build."""
    w = W.tiny(seed=15, kmesh=(2, 1, 1), ndens=2)
    r = orc.lrj(w)
    sel = [0, 5, 17, len(r["G"]) - 1]
    got = orc.rho_at(w, r["G"][sel])
    np.testing.assert_allclose(got, r["rho"][:, sel], atol=1e-13, rtol=0)


def test_oracle_gradient_matches_central_differences(orc):
    """dE_J/dR_C of the oracle against central finite differences (h = 1e-4 bohr)
    of the pinned oracle energy; the screened pair list is unchanged by the
    displacements here."""
    A = np.array([[5.0, 0.0, 0.0], [0.9, 5.3, 0.0], [-0.4, 0.6, 5.6]])
    w = W.tiny(seed=61, A=A, kmesh=(2, 1, 1), centres=[[0.1, 0.2, 0.3], [1.5, 0.7, -0.5]])
    g = orc.grad(w)
    h = 1e-4
    x0 = w.xyz.copy()
    for c in range(2):
        for d in range(3):
            w.xyz = x0.copy()
            w.xyz[c, d] += h
            ep = orc.lrj(w, want_rho=False, want_j0n=False)["EJ"][0]
            w.xyz = x0.copy()
            w.xyz[c, d] -= h
            em = orc.lrj(w, want_rho=False, want_j0n=False)["EJ"][0]
            fd = (ep - em) / (2 * h)
            assert abs(fd - g[0, c, d]) < 1e-7 * max(1.0, abs(fd)), (c, d, fd, g[0, c, d])
    w.xyz = x0
    # translational invariance: the gradients sum to zero
    assert np.abs(g.sum(axis=1)).max() < 1e-10


# ---------------------------------------------------------------------------
# density classification and the GPW route (Sec. 2.6, App. E)
# ---------------------------------------------------------------------------

def dense_gpw_grid(w, pmax, margin=2):
    """Grid points per axis that keep every alias of a DD transform (exponent
    at most pmax) beyond e^{-46} on the sphere: N_i |b_i| >= Gcut + sqrt(4 pmax 46)."""
    reach = orc_gcut(w) + math.sqrt(4.0 * pmax * 46.0)
    return [int(math.ceil(reach * np.linalg.norm(w.A[i]) / (2 * math.pi))) + margin for i in range(3)]


def orc_gcut(w):
    from oracle import gcut_of
    return gcut_of(w)


def test_classified_build_without_diffuse_pairs_is_the_plain_build(orc):
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    r0 = orc.lrj(w)
    r1 = orc.lrj_classified(w, alpha_cut=0.0)
    assert np.array_equal(r0["Jk"], r1["Jk"])
    assert np.array_equal(r0["EJ"], r1["EJ"])
    assert np.abs(r1["rhoD"]).max() == 0.0


@pytest.mark.parametrize("triclinic", [False, True])
def test_gpw_grid_transform_is_the_pair_transform(orc, triclinic):
    """rho_D(G) from the DD density sampled on a dense real-space grid (App. E)
    and a library FFT equals the direct pair transforms summed over the DD pairs
    (Eq. "AFT for pair density"): pins the collocation's images, normalisation
    and sign conventions.  alpha_cut = 0.9 makes s, p and d primitives diffuse,
    so DD pairs of classes 0..4 take part."""
    A = np.array([[6.0, 0.0, 0.0], [1.1, 6.4, 0.0], [-0.7, 0.8, 6.9]]) if triclinic else None
    w = W.tiny(seed=7, A=A, kmesh=(2, 1, 2), ndens=2)
    acut = 0.9
    r = orc.lrj_classified(w, alpha_cut=acut)
    grid = dense_gpw_grid(w, pmax=1.6)
    rho_r = orc.gpw_density(w, grid, alpha_cut=acut)
    rg = orc.grid_transform(w.A, rho_r, r["G"])
    scale = np.abs(r["rhoD"]).max()
    assert scale > 0.1
    assert np.abs(rg - r["rhoD"]).max() < 1e-13 * scale


def test_classified_all_diffuse_is_the_full_range_limit(orc):
    """With every primitive diffuse, the classified build is the long-range
    build in the limit w -> infinity (v_LR -> 4 pi / (Omega G^2))."""
    w = W.tiny(seed=5, kmesh=(1, 2, 1))
    r = orc.lrj_classified(w, alpha_cut=1e9)
    assert np.abs(r["rhoC"]).max() == 0.0
    gc = orc_gcut(w)
    w.gcut = gc
    w.omega = 1e8
    r_inf = orc.lrj(w)
    assert abs(r["EJ"][0] - r_inf["EJ"][0]) < 1e-13 * abs(r_inf["EJ"][0])
    assert np.abs(r["Jk"] - r_inf["Jk"]).max() < 1e-13 * np.abs(r_inf["Jk"]).max()


def test_classified_parseval_hermitian_and_bilinear_symmetry(orc):
    """E_J = (1/2Nk) sum_k Tr(D^k J^k) and Tr(D1 J[D2]) = Tr(D2 J[D1]) with
    mixed classes: an integral class given the wrong kernel on one side only
    breaks both."""
    acut = 0.9
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    r = orc.lrj_classified(w, alpha_cut=acut)
    Jk = r["Jk"]
    assert np.abs(r["rhoC"]).max() > 0.1 and np.abs(r["rhoD"]).max() > 0.1
    assert np.abs(Jk - np.conj(np.transpose(Jk, (0, 1, 3, 2)))).max() < 1e-13 * np.abs(Jk).max()
    for d in range(2):
        tr = sum(np.trace(w.Dk[d, k] @ Jk[d, k]) for k in range(w.nk)) / (2 * w.nk)
        assert abs(tr.imag) < 1e-13
        assert abs(tr.real - r["EJ"][d]) < 1e-12 * abs(r["EJ"][d])
    D1, D2 = w.Dk[:1], w.Dk[1:]
    J1 = orc.lrj_classified(w, alpha_cut=acut, Dk=D1)["Jk"]
    J2 = orc.lrj_classified(w, alpha_cut=acut, Dk=D2)["Jk"]
    t12 = sum(np.trace(D1[0, k] @ J2[0, k]) for k in range(w.nk))
    t21 = sum(np.trace(D2[0, k] @ J1[0, k]) for k in range(w.nk))
    assert abs(t12 - t21) < 1e-12 * abs(t12)


def test_classified_energy_terms_match_erf_lattice_sums(orc):
    """Neutral, dipole-free clouds of same-centre s Gaussians: compact charges
    (exponents 2.5, 1.2) on one centre, diffuse ones (0.09, 0.15) on another.
    Their compact-compact energy is the long-range erf(w r)/r lattice sum, the
    diffuse-diffuse one and the cross term the full-range sums (Sec. 2.6: only
    integrals between two compact densities keep the Ewald split).  The cell is
    large enough that no diffuse function overlaps its own images."""
    A = np.array([[26.0, 0.0, 0.0], [1.5, 27.0, 0.0], [-1.0, 1.2, 28.0]])
    cen = [[0.3, 0.2, 0.1], [1.1, -0.4, 0.7]]
    spec = [(0, 0, [2.5, 1.2]), (1, 0, [0.09, 0.15])]
    w = W.tiny(seed=1, A=A, centres=cen, shell_spec=spec, omega=0.4, eps_g=1e-17, pair_thresh=1e-12)
    for sa, _, sb, _, l1, l2, l3 in orc.pairs(w):
        if sa == sb:
            assert (l1, l2, l3) == (0, 0, 0)
    acut = 0.5
    q = np.array([1.0, -1.0, 0.7, -0.7])
    qc = q * np.array([1, 1, 0, 0])
    qd = q * np.array([0, 0, 1, 1])
    E = {}
    for name, qq in (("all", q), ("c", qc), ("d", qd)):
        D = np.diag(qq).astype(np.complex128)[None, None]
        E[name] = orc.lrj_classified(w, alpha_cut=acut, Dk=D)["EJ"][0]
    charges = [(q[i], 2 * w.shells[i].exps[0], w.xyz[w.shells[i].centre]) for i in range(4)]
    cc, dc = charges[:2], charges[2:]
    e_cc = N.erf_lattice_energy(A, cc, 0.4, rmax=60.0)
    e_dd = N.erf_lattice_energy(A, dc, math.inf, rmax=60.0)
    e_x_full = N.erf_lattice_energy(A, charges, math.inf, rmax=60.0) - \
        N.erf_lattice_energy(A, cc, math.inf, rmax=60.0) - e_dd
    e_x_lr = N.erf_lattice_energy(A, charges, 0.4, rmax=60.0) - e_cc - N.erf_lattice_energy(A, dc, 0.4, rmax=60.0)
    assert abs(E["c"] - e_cc) < 1e-12
    assert abs(E["d"] - e_dd) < 1e-12
    e_x = E["all"] - E["c"] - E["d"]
    assert abs(e_x - e_x_full) < 1e-12
    assert abs(e_x_full - e_x_lr) > 1e-4  # the two kernels are told apart


def test_gpw_grid_rule_without_margin_is_alias_free(orc):
    """At the smallest grid the alias rule allows (N_i |b_i| >= Gcut + sqrt(184 p_max),
    N_i > 2 max|n_i|, no extra points) the grid transform of the DD density still
    equals the pair transforms to 1e-12 of max|rho_D|; at a third of those points per
    axis it does not (the rule is what keeps the aliases out)."""
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=1)
    acut = 0.9
    r = orc.lrj_classified(w, alpha_cut=acut)
    nmax = np.abs(r["G"]).max(axis=0)
    grid = [max(int(2 * nmax[i] + 1), g) for i, g in enumerate(dense_gpw_grid(w, pmax=1.6, margin=0))]
    scale = np.abs(r["rhoD"]).max()
    rg = orc.grid_transform(w.A, orc.gpw_density(w, grid, alpha_cut=acut), r["G"])
    assert np.abs(rg - r["rhoD"]).max() < 1e-12 * scale
    coarse = [max(int(2 * nmax[i] + 1), g // 3) for i, g in enumerate(grid)]
    rc = orc.grid_transform(w.A, orc.gpw_density(w, coarse, alpha_cut=acut), r["G"])
    assert np.abs(rc - r["rhoD"]).max() > 1e-6 * scale
