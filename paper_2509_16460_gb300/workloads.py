"""Seeded synthetic inputs for the long-range planewave density-fitting Coulomb build.

This module only draws inputs: lattice, centres, uncontracted Gaussian shells,
k-mesh and Bloch density matrices D^k.  It holds none of the method's
arithmetic (no overlaps, no transforms, no Fourier sums), so both the CPU
oracle and the CUDA path can be fed from it.

The systems are stand-ins shaped like the paper's workloads (diamond-like
solid, molecular crystal, surface slab with adsorbate; Sec. 3 of the paper),
with exponent sets drawn as geometric sequences chosen here.  No published
basis-set data is reproduced.

Conventions (shared with the C-ABI):
  * lattice ``A`` is 3x3 with ROW i = lattice vector a_i, bohr;
  * k-mesh is Gamma-centred: k_m = sum_i (m_i / N_i) b_i, m_i in [0, N_i),
    flattened as m = (m1 * N2 + m2) * N3 + m3;
  * AO order is shell order; inside a Cartesian shell the components run
    lx = l..0, ly = l-lx..0 (xx, xy, xz, yy, yz, zz for d); inside a
    spherical shell m = -l..l, except p which is (x, y, z);
  * ``coefs`` multiply unit-normalised primitives;
  * D^k is complex128 [ndens][Nk][nao][nao], Hermitian per k, and
    time-reversal symmetric: D^{-k} = conj(D^k).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

DEFAULT_EPS_G = 1e-14
DEFAULT_PAIR_THRESH = 1e-12


@dataclasses.dataclass
class Shell:
    centre: int
    l: int
    spherical: bool
    exps: np.ndarray
    coefs: np.ndarray

    @property
    def nfunc(self) -> int:
        return 2 * self.l + 1 if self.spherical else (self.l + 1) * (self.l + 2) // 2


@dataclasses.dataclass
class Workload:
    name: str
    A: np.ndarray                 # [3,3] rows = lattice vectors (bohr)
    xyz: np.ndarray               # [ncentre,3] Cartesian bohr
    shells: List[Shell]
    kmesh: tuple
    omega: float
    Dk: np.ndarray                # complex128 [ndens][Nk][nao][nao]
    eps_g: float = DEFAULT_EPS_G
    gcut: float = 0.0             # <= 0: derived from eps_g
    pair_thresh: float = DEFAULT_PAIR_THRESH
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nao(self) -> int:
        return sum(s.nfunc for s in self.shells)

    @property
    def nk(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def ndens(self) -> int:
        return int(self.Dk.shape[0])

    def flat_basis(self):
        """Flat arrays describing the basis (the layout both sides parse)."""
        sh_cen = np.array([s.centre for s in self.shells], dtype=np.int32)
        sh_l = np.array([s.l for s in self.shells], dtype=np.int32)
        sh_sph = np.array([1 if s.spherical else 0 for s in self.shells], dtype=np.int32)
        sh_np = np.array([len(s.exps) for s in self.shells], dtype=np.int32)
        sh_off = np.zeros(len(self.shells), dtype=np.int32)
        if len(self.shells):
            sh_off[1:] = np.cumsum(sh_np)[:-1]
        exps = np.concatenate([np.asarray(s.exps, float) for s in self.shells]) if self.shells else np.zeros(0)
        coefs = np.concatenate([np.asarray(s.coefs, float) for s in self.shells]) if self.shells else np.zeros(0)
        return dict(sh_cen=sh_cen, sh_l=sh_l, sh_sph=sh_sph, sh_np=sh_np, sh_off=sh_off,
                    exps=np.ascontiguousarray(exps), coefs=np.ascontiguousarray(coefs))


# ----------------------------------------------------------------------------
# basic helpers (geometry and random matrices only)
# ----------------------------------------------------------------------------

def geometric(lo: float, hi: float, n: int) -> List[float]:
    if n == 1:
        return [float(lo)]
    r = (hi / lo) ** (1.0 / (n - 1))
    return [float(lo * r ** i) for i in range(n)]


def uncontracted(centre: int, l: int, exps: Sequence[float], spherical: bool) -> List[Shell]:
    return [Shell(centre, l, spherical, np.array([e], float), np.array([1.0])) for e in exps]


def kmesh_partner(kmesh) -> np.ndarray:
    """Index of -k for every k of a Gamma-centred mesh (pure index arithmetic)."""
    n1, n2, n3 = kmesh
    out = np.zeros(n1 * n2 * n3, dtype=np.int64)
    for m1 in range(n1):
        for m2 in range(n2):
            for m3 in range(n3):
                p = (((-m1) % n1) * n2 + ((-m2) % n2)) * n3 + ((-m3) % n3)
                out[(m1 * n2 + m2) * n3 + m3] = p
    return out


def random_bloch_density(rng: np.random.Generator, nao: int, kmesh, nocc: int,
                         sigma: float = 0.5) -> np.ndarray:
    """D^k = C^k C^k^dagger from random orbitals, with C^{-k} = conj(C^k).

    At self-conjugate k the orbitals are real.  Entries are N(0, sigma^2)
    (split evenly between real and imaginary parts for complex C)."""
    nk = int(np.prod(kmesh))
    partner = kmesh_partner(kmesh)
    C = np.zeros((nk, nao, nocc), dtype=np.complex128)
    for k in range(nk):
        pk = partner[k]
        if pk == k:
            C[k] = rng.normal(0.0, sigma, size=(nao, nocc))
        elif k < pk:
            re = rng.normal(0.0, sigma / math.sqrt(2.0), size=(nao, nocc))
            im = rng.normal(0.0, sigma / math.sqrt(2.0), size=(nao, nocc))
            C[k] = re + 1j * im
            C[pk] = np.conj(C[k])
    D = np.einsum("kmi,kni->kmn", C, np.conj(C))
    # exact Hermiticity and time-reversal symmetry at the bit level
    D = 0.5 * (D + np.conj(np.transpose(D, (0, 2, 1))))
    for k in range(nk):
        pk = partner[k]
        if pk == k:
            D[k] = D[k].real
        elif k < pk:
            D[pk] = np.conj(D[k])
    return D


def rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def min_image_distance(A: np.ndarray, f1: np.ndarray, f2: np.ndarray, reach: int = 2) -> float:
    """Shortest distance between two sites given in fractional coordinates,
    over the lattice translations with |T_i| <= reach (enough for the cells
    drawn here, whose angles stay within 60-120 degrees)."""
    d = np.asarray(f1, float) - np.asarray(f2, float)
    d -= np.round(d)
    r = np.arange(-reach, reach + 1)
    T = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return float(np.min(np.linalg.norm((d[None, :] + T) @ A, axis=1)))


# ----------------------------------------------------------------------------
# element templates (synthetic, geometric exponent sequences)
# ----------------------------------------------------------------------------

def _template(kind: str):
    if kind == "C2":      # carbon-like for the diamond-like solid: s8 p4 d2 = 30 AOs
        return [(0, geometric(0.1, 1.0e4, 8)), (1, geometric(0.15, 10.0, 4)), (2, [0.3, 1.2])]
    if kind == "C":       # carbon-like for molecular crystal / adsorbate: 30 AOs
        return [(0, geometric(0.1, 8.0e3, 8)), (1, geometric(0.15, 10.0, 4)), (2, [0.3, 1.2])]
    if kind == "H":       # hydrogen-like: s5 p3 = 14 AOs
        return [(0, geometric(0.1, 80.0, 5)), (1, geometric(0.2, 1.8, 3))]
    if kind == "O":       # oxygen-like: s8 p4 d2 = 30 AOs
        return [(0, geometric(0.15, 1.5e4, 8)), (1, geometric(0.2, 30.0, 4)), (2, [0.4, 1.6])]
    if kind == "Mg":      # magnesium-like: s8 p4 d1 = 25 AOs
        return [(0, geometric(0.08, 2.0e4, 8)), (1, geometric(0.1, 50.0, 4)), (2, [0.5])]
    raise ValueError(kind)


_Z_KIND = {1: "H", 6: "C", 8: "O", 12: "Mg"}


def shells_for(centre: int, kind: str, spherical: bool = True) -> List[Shell]:
    out: List[Shell] = []
    for l, exps in _template(kind):
        out += uncontracted(centre, l, exps, spherical)
    return out


# ----------------------------------------------------------------------------
# the five workload shapes
# ----------------------------------------------------------------------------

def cfg1(seed: int = 1) -> Workload:
    """Gamma point, cubic 8 bohr, 2 centres, Cartesian s(10,1,0.2)+p(1,0.3), 18 AOs, omega 0.3."""
    A = np.eye(3) * 8.0
    xyz = np.array([[0.0, 0.0, 0.0], [1.4, 0.0, 0.0]])
    shells: List[Shell] = []
    for c in range(2):
        shells += uncontracted(c, 0, [10.0, 1.0, 0.2], False)
        shells += uncontracted(c, 1, [1.0, 0.3], False)
    rng = np.random.default_rng(seed)
    nao = sum(s.nfunc for s in shells)
    C = rng.normal(0.0, 0.5, size=(nao, 2))
    D = (C @ C.T)[None, None].astype(np.complex128)
    return Workload("cfg1-gamma-2centre-18ao", A, xyz, shells, (1, 1, 1), 0.3, D,
                    meta=dict(seed=seed, nocc=2, sigma=0.5))


def cfg2(seed: int = 2, kmesh=(4, 4, 4)) -> Workload:
    """Diamond-like cubic cell a=6.74, 8 C-like centres, spherical s8p4d2 (240 AOs), k 4x4x4, omega 0.4."""
    a = 6.74
    A = np.eye(3) * a
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    frac = np.vstack([fcc, fcc + 0.25])
    xyz = frac @ A
    shells: List[Shell] = []
    for c in range(8):
        shells += shells_for(c, "C2")
    rng = np.random.default_rng(seed)
    nao = sum(s.nfunc for s in shells)
    Dk = random_bloch_density(rng, nao, kmesh, 16)[None]
    return Workload("cfg2-diamond-240ao-k444", A, xyz, shells, tuple(kmesh), 0.4, Dk,
                    meta=dict(seed=seed, nocc=16, sigma=0.5))


def benzene_ring(rng: np.random.Generator):
    """6 C at radius 2.64 (C-C 2.64 bohr) and 6 H 2.05 bohr further out, random orientation."""
    ang = np.arange(6) * (np.pi / 3.0)
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], axis=1)
    c = ring * 2.64
    h = ring * (2.64 + 2.05)
    R = rotation(rng)
    return c @ R.T, h @ R.T


def cfg3(seed: int = 3, kmesh=(2, 2, 2), nspin: int = 2) -> Workload:
    """Orthorhombic 14.0x17.8x12.9, 4 benzene-like rings (24 C + 24 H, 1056 AOs), k 2x2x2, 2 spins, omega 0.5."""
    A = np.diag([14.0, 17.8, 12.9])
    sites = np.array([[0, 0, 0], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]]) @ A
    rng = np.random.default_rng(seed)
    cs, hs = [], []
    for s in sites:
        c, h = benzene_ring(rng)
        cs.append(c + s)
        hs.append(h + s)
    xyz = np.vstack(cs + hs)
    shells: List[Shell] = []
    for i in range(24):
        shells += shells_for(i, "C")
    for i in range(24, 48):
        shells += shells_for(i, "H")
    nao = sum(s.nfunc for s in shells)
    Dk = np.stack([random_bloch_density(rng, nao, kmesh, 84) for _ in range(nspin)])
    return Workload("cfg3-benzene-crystal-1056ao-k222-2spin", A, xyz, shells, tuple(kmesh), 0.5, Dk,
                    meta=dict(seed=seed, nocc=84, sigma=0.5, nspin=nspin))


def triclinic_cell(rng: np.random.Generator, lo=6.0, hi=16.0) -> np.ndarray:
    while True:
        a, b, c = rng.uniform(lo, hi, 3)
        al, be, ga = np.radians(rng.uniform(60.0, 120.0, 3))
        cx = math.cos(be)
        cy = (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
        cz2 = 1.0 - cx * cx - cy * cy
        if cz2 < 0.1:
            continue
        A = np.array([[a, 0, 0],
                      [b * math.cos(ga), b * math.sin(ga), 0],
                      [c * cx, c * cy, c * math.sqrt(cz2)]])
        return A


def cfg4_cell(rng: np.random.Generator, index: int) -> Workload:
    A = triclinic_cell(rng)
    ncen = int(rng.integers(2, 25))
    zs = rng.choice([1, 6, 8, 12], size=ncen)
    frac: List[np.ndarray] = []
    while len(frac) < ncen:
        f = rng.uniform(0, 1, 3)
        ok = True
        for g in frac:
            d = f - g
            d -= np.round(d)
            if np.linalg.norm(d @ A) < 1.5:
                ok = False
                break
        if ok:
            frac.append(f)
    xyz = np.array(frac) @ A
    shells: List[Shell] = []
    for i, z in enumerate(zs):
        shells += shells_for(i, _Z_KIND[int(z)])
    kmesh = tuple(int(x) for x in rng.integers(1, 4, 3))
    omega = float(rng.uniform(0.3, 0.5))
    nao = sum(s.nfunc for s in shells)
    Dk = random_bloch_density(rng, nao, kmesh, max(1, nao // 10))[None]
    return Workload(f"cfg4-triclinic-{index}", A, xyz, shells, kmesh, omega, Dk,
                    meta=dict(index=index, ncentre=ncen, z=[int(z) for z in zs]))


def cfg4(seed: int = 4, ncell: int = 64) -> List[Workload]:
    """64 random triclinic cells (edges 6-16 bohr, 2-24 centres, Z in {1,6,8,12})."""
    rng = np.random.default_rng(seed)
    return [cfg4_cell(rng, i) for i in range(ncell)]


def cfg5(seed: int = 5, kmesh=(3, 3, 1)) -> Workload:
    """Rock-salt (001) 2x2 slab, 4 layers (16 Mg-like + 16 O-like) + CO adsorbate, 20 bohr vacuum, k 3x3x1."""
    d = 3.98
    side = 2.0 * math.sqrt(2.0) * d            # 11.26 bohr
    c = 3.0 * d + 20.0
    A = np.diag([side, side, c])
    u = np.array([1.0, 1.0, 0.0]) * (d / math.sqrt(2.0))
    v = np.array([-1.0, 1.0, 0.0]) * (d / math.sqrt(2.0))
    xyz: List[np.ndarray] = []
    kinds: List[str] = []
    for layer in range(4):
        fr: List[np.ndarray] = []
        for i in range(4):
            for j in range(-2, 2):
                p = i * u + j * v
                f = np.linalg.solve(A.T, p)
                # wrap into [0, 1) with a tolerance, so that a site on the cell
                # boundary (f = 1 - eps) lands on 0 and is seen as an image
                f = np.mod(np.round(f, 10), 1.0)
                if any(min_image_distance(A, f, g) < 1e-6 for g in fr):
                    continue
                fr.append(f)
                xyz.append(f @ A + np.array([0, 0, layer * d]))
                kinds.append("Mg" if (i + j + layer) % 2 == 0 else "O")
        # the square cell of side 2 sqrt(2) d holds 8 sites of a rock-salt (001) layer
        if len(fr) != 8:
            raise AssertionError(f"slab layer {layer}: {len(fr)} sites, expected 8")
    top = max(p[2] for p in xyz)
    mg_top = [p for p, k in zip(xyz, kinds) if k == "Mg" and abs(p[2] - top) < 1e-6][0]
    xyz.append(mg_top + np.array([0, 0, 4.3]))
    kinds.append("C")
    xyz.append(mg_top + np.array([0, 0, 4.3 + 2.13]))
    kinds.append("O")
    shells: List[Shell] = []
    for i, k in enumerate(kinds):
        shells += shells_for(i, k)
    rng = np.random.default_rng(seed)
    nao = sum(s.nfunc for s in shells)
    Dk = random_bloch_density(rng, nao, kmesh, 40)[None]
    return Workload("cfg5-mgo001-slab-co", A, np.array(xyz), shells, tuple(kmesh), 0.4, Dk,
                    meta=dict(seed=seed, kinds=kinds))


# ----------------------------------------------------------------------------
# tiny systems for tests
# ----------------------------------------------------------------------------

def tiny(seed: int = 11, A=None, centres=None, shell_spec=None, kmesh=(1, 1, 1), omega=0.35,
         nocc: int = 2, spherical: bool = True, ndens: int = 1, sigma: float = 0.5,
         pair_thresh: float = DEFAULT_PAIR_THRESH, eps_g: float = DEFAULT_EPS_G) -> Workload:
    """A small seeded system; ``shell_spec`` is a list of (centre, l, [exps])."""
    if A is None:
        A = np.diag([5.0, 5.5, 6.0])
    A = np.asarray(A, float)
    if centres is None:
        centres = [[0.1, 0.2, 0.3], [1.3, 0.9, -0.4]]
    xyz = np.asarray(centres, float)
    if shell_spec is None:
        shell_spec = [(0, 0, [2.0, 0.4]), (0, 1, [0.8]), (1, 0, [1.1]), (1, 2, [0.6])]
    shells: List[Shell] = []
    for c, l, exps in shell_spec:
        shells += uncontracted(c, l, exps, spherical)
    rng = np.random.default_rng(seed)
    nao = sum(s.nfunc for s in shells)
    Dk = np.stack([random_bloch_density(rng, nao, kmesh, nocc, sigma) for _ in range(ndens)])
    return Workload(f"tiny-{seed}", A, xyz, shells, tuple(kmesh), omega, Dk,
                    pair_thresh=pair_thresh, eps_g=eps_g, meta=dict(seed=seed))


def by_name(name: str) -> Workload:
    return {"cfg1": cfg1, "cfg2": cfg2, "cfg3": cfg3, "cfg5": cfg5}[name]()
