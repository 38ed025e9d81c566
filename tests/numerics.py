"""Independent numerical references used to pin the oracle (numpy/scipy only).

Nothing here imports the oracle's arithmetic or the CUDA path: these are
quadratures, brute-force lattice sums and closed forms written out for the
tests.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def cart_list(l):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


# Real solid harmonics (Racah normalisation) written out for l <= 2, in the
# library's order m = -l..l (p as x, y, z); coefficients over cart_list(l).
TEXTBOOK_SPH = {
    0: [[1.0]],
    1: [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    2: [
        [0, math.sqrt(3), 0, 0, 0, 0],          # xy
        [0, 0, 0, 0, math.sqrt(3), 0],          # yz
        [-0.5, 0, 0, -0.5, 0, 1.0],             # z^2 - (x^2+y^2)/2
        [0, 0, math.sqrt(3), 0, 0, 0],          # xz
        [math.sqrt(3) / 2, 0, 0, -math.sqrt(3) / 2, 0, 0],  # (x^2-y^2) sqrt3/2
    ],
}


def ao_values(shell, centre, pts, sph_table=TEXTBOOK_SPH):
    """Values of the (unit-normalised by quadrature later) shell functions at
    pts [N,3]; returns [nf, N] UNNORMALISED per primitive (single primitive)."""
    l = shell.l
    r = pts - centre[None, :]
    r2 = np.sum(r * r, axis=1)
    carts = cart_list(l)
    mono = np.stack([r[:, 0] ** a * r[:, 1] ** b * r[:, 2] ** c for (a, b, c) in carts])
    if shell.spherical:
        U = np.array(sph_table[l], float)
        ang = U @ mono
    else:
        ang = mono
    return ang * np.exp(-shell.exps[0] * r2)[None, :]


def gh_overlap_1d(i, j, a, A, b, B, n=40):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx by Gauss-Hermite quadrature."""
    x, w = np.polynomial.hermite.hermgauss(n)
    p = a + b
    P = (a * A + b * B) / p
    pref = math.exp(-a * b / p * (A - B) ** 2)
    xs = P + x / math.sqrt(p)
    return pref / math.sqrt(p) * np.sum(w * (xs - A) ** i * (xs - B) ** j)


def monomial_overlap(ca, a, A, cb, b, B):
    return np.prod([gh_overlap_1d(ca[k], cb[k], a, A[k], b, B[k]) for k in range(3)])


def shell_overlap(sa, A, sb, B, sph_table=TEXTBOOK_SPH):
    """Overlap matrix of two single-primitive shells, each function unit-normalised
    by its own quadrature self-overlap."""
    def U(s):
        if s.spherical:
            return np.array(sph_table[s.l], float)
        return np.eye(len(cart_list(s.l)))
    Ua, Ub = U(sa), U(sb)
    la, lb = cart_list(sa.l), cart_list(sb.l)
    a, b = sa.exps[0], sb.exps[0]
    Sab = np.array([[monomial_overlap(x, a, A, y, b, B) for y in lb] for x in la])
    Saa = np.array([[monomial_overlap(x, a, A, y, a, A) for y in la] for x in la])
    Sbb = np.array([[monomial_overlap(x, b, B, y, b, B) for y in lb] for x in lb])
    na = 1.0 / np.sqrt(np.einsum("fc,cd,fd->f", Ua, Saa, Ua))
    nb = 1.0 / np.sqrt(np.einsum("fc,cd,fd->f", Ub, Sbb, Ub))
    return (na[:, None] * (Ua @ Sab @ Ub.T) * nb[None, :]) * sa.coefs[0] * sb.coefs[0]


def grid_ft(sa, A, sb, B, G, box=18.0, h=0.12, sph_table=TEXTBOOK_SPH):
    """int phi_a(r) phi_b(r) exp(-i G.r) dr by a 3D Riemann sum on a uniform
    grid (spectrally accurate for Gaussians); functions normalised on the
    same grid."""
    c = 0.5 * (np.asarray(A) + np.asarray(B))
    n = int(round(box / h))
    ax = (np.arange(n) - n / 2) * h
    X, Y, Z = np.meshgrid(ax + c[0], ax + c[1], ax + c[2], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    fa = ao_values(sa, np.asarray(A, float), pts, sph_table)
    fb = ao_values(sb, np.asarray(B, float), pts, sph_table)
    dv = h ** 3
    na = 1.0 / np.sqrt(np.sum(fa * fa, axis=1) * dv)
    nb = 1.0 / np.sqrt(np.sum(fb * fb, axis=1) * dv)
    ph = np.exp(-1j * (pts @ np.asarray(G, float)))
    out = np.einsum("fn,gn,n->fg", fa, fb, ph) * dv
    return out * na[:, None] * nb[None, :] * sa.coefs[0] * sb.coefs[0]


def erf_lattice_energy(A, charges, omega, rmax=40.0):
    """Brute-force real-space energy 1/2 sum_T sum_ij q_i q_j erf(g_ij|R_ij+T|)/|R_ij+T|
    of Gaussian charges (q, exponent p, centre) under erf(omega r)/r, with
    g_ij^-2 = omega^-2 + 1/p_i + 1/p_j, T over the lattice within rmax; the
    T=0, R=0 terms take the limit 2 g/sqrt(pi).  Valid (absolutely
    convergent) for a neutral, dipole-free cell."""
    A = np.asarray(A, float)
    q = np.array([c[0] for c in charges])
    p = np.array([c[1] for c in charges])
    R = np.array([c[2] for c in charges], float)
    Binv = np.linalg.inv(A)
    lim = [int(math.ceil(rmax * np.linalg.norm(Binv[:, i]))) + 1 for i in range(3)]
    Ts = np.array([[i, j, k] for i in range(-lim[0], lim[0] + 1) for j in range(-lim[1], lim[1] + 1)
                   for k in range(-lim[2], lim[2] + 1)], float) @ A
    E = 0.0
    for i in range(len(q)):
        for j in range(len(q)):
            g = 1.0 / math.sqrt(1.0 / omega ** 2 + 1.0 / p[i] + 1.0 / p[j])
            d = R[i] - R[j] + Ts
            r = np.linalg.norm(d, axis=1)
            small = r < 1e-12
            val = np.where(small, 2.0 * g / math.sqrt(math.pi), erf(g * np.where(small, 1.0, r)) /
                           np.where(small, 1.0, r))
            val = np.where(r <= rmax, val, 0.0)
            E += 0.5 * q[i] * q[j] * np.sum(val)
    return E
