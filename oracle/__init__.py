"""Python access to the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA product path never
imports this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    basis = [_dp, ctypes.c_int, _dp, ctypes.c_int, _ip, _ip, _ip, _ip, _ip, _dp, _dp]
    L.orc_nao.argtypes = basis
    L.orc_nao.restype = ctypes.c_int
    L.orc_reciprocal.argtypes = [_dp, _dp, _dp]
    L.orc_reciprocal.restype = ctypes.c_int
    L.orc_gsphere.argtypes = [_dp, ctypes.c_double, ctypes.c_long, _ip]
    L.orc_gsphere.restype = ctypes.c_long
    L.orc_pairs.argtypes = basis + [ctypes.c_double, ctypes.c_long, _ip]
    L.orc_pairs.restype = ctypes.c_long
    L.orc_pair_ft.argtypes = basis + [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_double, _dp]
    L.orc_pair_ft.restype = ctypes.c_int
    L.orc_fold_density.argtypes = [ctypes.c_int, _ip, ctypes.c_int, _dp, _dp]
    L.orc_fold_density.restype = ctypes.c_int
    L.orc_lrj.argtypes = basis + [_ip, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  _dp, _dp, _dp, _dp, ctypes.c_long, _ip, _dp, ctypes.c_int, ctypes.c_int, _dp]
    L.orc_lrj.restype = ctypes.c_int
    L.orc_lrj_classified.argtypes = basis + [_ip, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_long,
                                             _ip, _dp, ctypes.c_int]
    L.orc_lrj_classified.restype = ctypes.c_int
    L.orc_gpw_density.argtypes = basis + [_ip, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _ip, _dp,
                                          ctypes.c_int]
    L.orc_gpw_density.restype = ctypes.c_int
    L.orc_rho_at.argtypes = basis + [_ip, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp,
                                     ctypes.c_int]
    L.orc_rho_at.restype = ctypes.c_int
    L.orc_grad.argtypes = basis + [_ip, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                   ctypes.c_int]
    L.orc_grad.restype = ctypes.c_int
    L.orc_solid_harmonic.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
    L.orc_solid_harmonic.restype = ctypes.c_int
    L.orc_norms.argtypes = basis + [ctypes.c_int, ctypes.c_int, _dp]
    L.orc_norms.restype = ctypes.c_int


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


class _Basis:
    """Keeps the flat arrays alive while the C call runs."""

    def __init__(self, A, xyz, fb):
        self.A = np.ascontiguousarray(A, dtype=np.float64)
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.fb = {k: np.ascontiguousarray(v) for k, v in fb.items()}

    def args(self):
        f = self.fb
        return [_d(self.A), int(self.xyz.shape[0]), _d(self.xyz), int(len(f["sh_l"])), _i(f["sh_cen"]),
                _i(f["sh_l"]), _i(f["sh_sph"]), _i(f["sh_np"]), _i(f["sh_off"]), _d(f["exps"]), _d(f["coefs"])]


def gcut_of(w) -> float:
    """Sphere radius: given gcut, else 2 w sqrt(ln(1/eps_g)) so that exp(-G^2/4w^2) = eps_g."""
    if w.gcut and w.gcut > 0:
        return float(w.gcut)
    return 2.0 * w.omega * float(np.sqrt(np.log(1.0 / w.eps_g)))


def reciprocal(A):
    B = np.zeros((3, 3))
    vol = np.zeros(1)
    rc = lib().orc_reciprocal(_d(np.ascontiguousarray(A, float)), _d(B), _d(vol))
    assert rc == 0
    return B, float(vol[0])


def gsphere(A, gcut):
    A = np.ascontiguousarray(A, float)
    n = lib().orc_gsphere(_d(A), float(gcut), 0, None)
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib().orc_gsphere(_d(A), float(gcut), n, _i(out))
    return out[:n]


def pairs(w):
    b = _Basis(w.A, w.xyz, w.flat_basis())
    n = lib().orc_pairs(*b.args(), float(w.pair_thresh), 0, None)
    out = np.zeros((max(n, 1), 7), dtype=np.int32)
    lib().orc_pairs(*b.args(), float(w.pair_thresh), n, _i(out))
    return out[:n]


def pair_ft(w, sa, sb, L, G, thresh=None):
    b = _Basis(w.A, w.xyz, w.flat_basis())
    nf = [s.nfunc for s in w.shells]
    out = np.zeros((nf[sa], nf[sb], 2))
    Lv = np.ascontiguousarray(L, dtype=np.int32)
    Gv = np.ascontiguousarray(G, dtype=np.float64)
    th = w.pair_thresh if thresh is None else thresh
    rc = lib().orc_pair_ft(*b.args(), int(sa), int(sb), _i(Lv), _d(Gv), float(th), _d(out))
    assert rc == 0
    return out[..., 0] + 1j * out[..., 1]


def fold_density(w):
    Dk = np.ascontiguousarray(w.Dk, dtype=np.complex128)
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    out = np.zeros((w.ndens, w.nk, w.nao, w.nao), dtype=np.complex128)
    lib().orc_fold_density(w.ndens, _i(km), w.nao, Dk.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def lrj(w, Dk=None, nthreads: int = 0, pair_stride: int = 1, want_rho: bool = True, want_j0n: bool = True):
    """Run the whole oracle build.  Returns a dict with Jk, EJ, rho, G (full
    sphere, oracle order), J0n, stats."""
    b = _Basis(w.A, w.xyz, w.flat_basis())
    Dk = np.ascontiguousarray(w.Dk if Dk is None else Dk, dtype=np.complex128)
    ndens, nk, nao = Dk.shape[0], Dk.shape[1], Dk.shape[2]
    gc = gcut_of(w)
    nG = int(lib().orc_gsphere(_d(b.A), gc, 0, None))
    Jk = np.zeros((ndens, nk, nao, nao), dtype=np.complex128)
    EJ = np.zeros(ndens)
    rho = np.zeros((ndens, max(nG, 1)), dtype=np.complex128) if want_rho else None
    G = np.zeros((max(nG, 1), 3), dtype=np.int32)
    J0n = np.zeros((ndens, nk, nao, nao), dtype=np.complex128) if want_j0n else None
    stats = np.zeros(4)
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    rc = lib().orc_lrj(*b.args(), _i(km), float(w.omega), gc, float(w.pair_thresh), int(ndens),
                       Dk.ctypes.data_as(_dp), Jk.ctypes.data_as(_dp), _d(EJ),
                       rho.ctypes.data_as(_dp) if rho is not None else None, nG, _i(G),
                       J0n.ctypes.data_as(_dp) if J0n is not None else None, int(pair_stride), int(nthreads),
                       _d(stats))
    if rc != 0:
        raise RuntimeError(f"orc_lrj failed: {rc}")
    return dict(Jk=Jk, EJ=EJ, rho=None if rho is None else rho[:, :nG], G=G[:nG], J0n=J0n,
                npairs=int(stats[0]), nG=int(stats[1]), units=float(stats[2]), seconds=float(stats[3]))


def alpha_cut_of(w, alpha_cut=None) -> float:
    """Compact/diffuse exponent boundary: given, else w^2/2 (Sec. 2.6, Eq. "cd cutoff")."""
    return 0.5 * w.omega ** 2 if alpha_cut is None else float(alpha_cut)


def lrj_classified(w, alpha_cut=None, Dk=None, nthreads: int = 0, want_j0n: bool = False):
    """The build with compact/diffuse pair classes (Sec. 2.6).  Returns a dict
    with Jk, EJ, rhoC, rhoD (full sphere, oracle order), G and optionally J0n."""
    b = _Basis(w.A, w.xyz, w.flat_basis())
    Dk = np.ascontiguousarray(w.Dk if Dk is None else Dk, dtype=np.complex128)
    ndens, nk, nao = Dk.shape[0], Dk.shape[1], Dk.shape[2]
    gc = gcut_of(w)
    nG = int(lib().orc_gsphere(_d(b.A), gc, 0, None))
    Jk = np.zeros((ndens, nk, nao, nao), dtype=np.complex128)
    EJ = np.zeros(ndens)
    rc_ = np.zeros((ndens, max(nG, 1)), dtype=np.complex128)
    rd_ = np.zeros((ndens, max(nG, 1)), dtype=np.complex128)
    G = np.zeros((max(nG, 1), 3), dtype=np.int32)
    J0n = np.zeros((ndens, nk, nao, nao), dtype=np.complex128) if want_j0n else None
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    rc = lib().orc_lrj_classified(*b.args(), _i(km), float(w.omega), gc, float(w.pair_thresh),
                                  alpha_cut_of(w, alpha_cut), int(ndens), Dk.ctypes.data_as(_dp),
                                  Jk.ctypes.data_as(_dp), _d(EJ), rc_.ctypes.data_as(_dp), rd_.ctypes.data_as(_dp),
                                  nG, _i(G), J0n.ctypes.data_as(_dp) if J0n is not None else None, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_lrj_classified failed: {rc}")
    return dict(Jk=Jk, EJ=EJ, rhoC=rc_[:, :nG], rhoD=rd_[:, :nG], G=G[:nG], J0n=J0n)


def gpw_density(w, grid, alpha_cut=None, Dk=None, nthreads: int = 0):
    """The DD density on the grid r_m = sum_i (m_i/N_i) a_i: [ndens][N1][N2][N3] (App. E)."""
    b = _Basis(w.A, w.xyz, w.flat_basis())
    Dk = np.ascontiguousarray(w.Dk if Dk is None else Dk, dtype=np.complex128)
    gr = np.ascontiguousarray(grid, dtype=np.int32)
    out = np.zeros((Dk.shape[0], int(gr[0]), int(gr[1]), int(gr[2])))
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    rc = lib().orc_gpw_density(*b.args(), _i(km), float(w.pair_thresh), alpha_cut_of(w, alpha_cut),
                               int(Dk.shape[0]), Dk.ctypes.data_as(_dp), _i(gr), _d(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_gpw_density failed: {rc}")
    return out


def grid_transform(A, values, G):
    """rho(G_n) = (Omega/N) sum_m rho(r_m) e^{-i G_n . r_m} for the listed n
    triples, by the library FFT (e^{-2 pi i n.m/N} on the grid axes)."""
    _, vol = reciprocal(A)
    shape = values.shape[-3:]
    F = np.fft.fftn(values, axes=(-3, -2, -1)) * (vol / float(np.prod(shape)))
    n = np.asarray(G, dtype=np.int64)
    return F[..., n[:, 0] % shape[0], n[:, 1] % shape[1], n[:, 2] % shape[2]]


def rho_at(w, n_list, nthreads: int = 0):
    b = _Basis(w.A, w.xyz, w.flat_basis())
    Dk = np.ascontiguousarray(w.Dk, dtype=np.complex128)
    nl = np.ascontiguousarray(n_list, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((w.ndens, nl.shape[0]), dtype=np.complex128)
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    rc = lib().orc_rho_at(*b.args(), _i(km), float(w.pair_thresh), int(w.ndens), Dk.ctypes.data_as(_dp),
                          int(nl.shape[0]), _i(nl), out.ctypes.data_as(_dp), int(nthreads))
    assert rc == 0
    return out


def solid_harmonic(l, m):
    out = np.zeros((l + 1) * (l + 2) // 2)
    assert lib().orc_solid_harmonic(int(l), int(m), _d(out)) == 0
    return out


def norms(w, s, k=0):
    b = _Basis(w.A, w.xyz, w.flat_basis())
    out = np.zeros(w.shells[s].nfunc)
    assert lib().orc_norms(*b.args(), int(s), int(k), _d(out)) == 0
    return out


def grad(w, Dk=None, nthreads: int = 0):
    """dE_J/dR_C [ndens][ncentre][3] (D^k held fixed)."""
    b = _Basis(w.A, w.xyz, w.flat_basis())
    Dk = np.ascontiguousarray(w.Dk if Dk is None else Dk, dtype=np.complex128)
    out = np.zeros((Dk.shape[0], b.xyz.shape[0], 3))
    km = np.ascontiguousarray(w.kmesh, dtype=np.int32)
    rc = lib().orc_grad(*b.args(), _i(km), float(w.omega), gcut_of(w), float(w.pair_thresh), int(Dk.shape[0]),
                        Dk.ctypes.data_as(_dp), _d(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_grad failed: {rc}")
    return out
