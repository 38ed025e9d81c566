"""Thin Python binding of libftcj.so (the C-ABI declared in include/ftcj.h).

Argument marshalling only: torch supplies device memory and streams, every
step of the build runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libftcj.so")

FTCJ_PREC_FP64 = 0
FTCJ_PREC_SPLIT = 1
FTCJ_LMAX = 2

_c_int, _c_double, _c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class Cell(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 9)]


class ShellDesc(ctypes.Structure):
    _fields_ = [("centre", _c_int), ("l", _c_int), ("spherical", _c_int), ("nprim", _c_int),
                ("exps", _dp), ("coefs", _dp)]


class BasisDesc(ctypes.Structure):
    _fields_ = [("ncentre", _c_int), ("xyz", _dp), ("nshell", _c_int), ("shells", ctypes.POINTER(ShellDesc))]


class Params(ctypes.Structure):
    _fields_ = [("omega", _c_double), ("gcut", _c_double), ("eps_g", _c_double), ("pair_thresh", _c_double),
                ("precision", _c_int), ("max_dens", _c_int), ("chunk_points", _c_int), ("rho_blocks", _c_int),
                ("pair_gcut_eps", _c_double), ("shard_count", _c_int), ("shard_index", _c_int),
                ("contraction", _c_int), ("tc_wait_log2", _c_int), ("classify", _c_int),
                ("alpha_cut", _c_double), ("gpw_grid", _c_int * 3)]


class Info(ctypes.Structure):
    _fields_ = [("nao", _c_int), ("nk", _c_int), ("nshell", _c_int), ("ngroup", _c_int),
                ("npairs", ctypes.c_int64), ("npairs_ordered", ctypes.c_int64), ("ng_half", ctypes.c_int64),
                ("ng_full", ctypes.c_int64), ("pair_g_units", ctypes.c_int64),
                ("pairs_by_class", ctypes.c_int64 * 5), ("nlines", _c_int), ("nchunks", _c_int),
                ("gcut", _c_double), ("volume", _c_double), ("device_bytes", ctypes.c_size_t),
                ("rho_blocks", _c_int), ("n1_table", _c_int), ("pair_g_units_screened", ctypes.c_int64),
                ("pair_g_units_walked", ctypes.c_int64), ("n_abs_max", _c_int), ("grad_split", _c_int),
                ("rho_walk_launches", _c_int), ("j_walk_launches", _c_int), ("contraction", _c_int),
                ("tc_mma_flops", ctypes.c_int64), ("j_contraction", _c_int), ("tc_j_mma_flops", ctypes.c_int64),
                ("tc_column_axis", _c_int), ("tc_rows", _c_int), ("tc_row_tiles", _c_int),
                ("tc_blocks_per_window", _c_int), ("tc_dens_per_launch", _c_int),
                ("dd_pairs", ctypes.c_int64), ("dd_pairs_ordered", ctypes.c_int64), ("alpha_cut", _c_double),
                ("gpw_grid", _c_int * 3), ("gpw_separable", _c_int), ("gpw_launches", _c_int),
                ("dd_pairs_by_class", ctypes.c_int64 * 5)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["pairs_by_class"] = list(self.pairs_by_class)
        d["gpw_grid"] = list(self.gpw_grid)
        d["dd_pairs_by_class"] = list(self.dd_pairs_by_class)
        return d


EXPORTED = [
    "ftcj_plan_create", "ftcj_plan_info", "ftcj_plan_destroy", "ftcj_jbuild", "ftcj_jbuild_host",
    "ftcj_fold_density", "ftcj_rho", "ftcj_potential", "ftcj_jback", "ftcj_unfold_j", "ftcj_check_density",
    "ftcj_get_gvectors", "ftcj_get_pairs", "ftcj_get_groups", "ftcj_strerror", "ftcj_last_error",
    "ftcj_profile_enable", "ftcj_profile_read", "ftcj_launches_per_batch", "ftcj_probe_fma_peak",
    "ftcj_potential_noalloc", "ftcj_batch_create", "ftcj_batch_info", "ftcj_batch_jbuild", "ftcj_batch_capture",
    "ftcj_batch_replay", "ftcj_batch_destroy", "ftcj_autotune", "ftcj_grad", "ftcj_shard_bounds",
    "ftcj_plan_status", "ftcj_batch_set_wait", "ftcj_batch_status",
]

FTCJ_CONTRACT_WALK = 0
FTCJ_CONTRACT_TC = 1

FTCJ_BATCH_AUTOTUNE = 1
FTCJ_BATCH_PERSISTENT = 2

FTCJ_NOALLOC_MAX_PARTIALS = 16384

PHASES = ["fold", "hermite", "rho_walk", "potential", "j_walk", "j_to_ao", "unfold", "gpw_rho", "gpw_j"]

_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


class FtcjError(RuntimeError):
    pass


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FtcjError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
                                "or python -m paper_2509_16460_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    P = _c_void_p
    L.ftcj_plan_create.argtypes = [ctypes.POINTER(Cell), ctypes.POINTER(BasisDesc), _ip, ctypes.POINTER(Params),
                                   ctypes.POINTER(_c_void_p)]
    L.ftcj_plan_info.argtypes = [P, ctypes.POINTER(Info)]
    L.ftcj_plan_destroy.argtypes = [P]
    L.ftcj_plan_destroy.restype = None
    for name in ("ftcj_jbuild", "ftcj_jbuild_host"):
        getattr(L, name).argtypes = [P, _c_int, P, P, P, P]
    for name in ("ftcj_fold_density", "ftcj_rho", "ftcj_jback", "ftcj_unfold_j"):
        getattr(L, name).argtypes = [P, _c_int, P, P, P]
    L.ftcj_potential.argtypes = [P, _c_int, P, P, P, P]
    L.ftcj_check_density.argtypes = [P, _c_int, P, _dp, _dp, P]
    L.ftcj_plan_status.argtypes = [P, _ip, P]
    L.ftcj_get_gvectors.argtypes = [P, _ip]
    L.ftcj_get_pairs.argtypes = [P, _ip]
    L.ftcj_get_groups.argtypes = [P, _ip, _dp, _ip, _ip]
    L.ftcj_profile_enable.argtypes = [P, _c_int]
    L.ftcj_profile_read.argtypes = [P, _dp, _ip, ctypes.POINTER(ctypes.c_int64)]
    L.ftcj_launches_per_batch.argtypes = [P, _c_int, ctypes.POINTER(ctypes.c_int64)]
    L.ftcj_probe_fma_peak.argtypes = [_c_int, _dp, P]
    L.ftcj_potential_noalloc.argtypes = [_dp, _c_double, _c_int, ctypes.c_int64, P, P, P, P, P]
    VPP = ctypes.POINTER(_c_void_p)
    L.ftcj_batch_create.argtypes = [_c_int, ctypes.POINTER(Cell), ctypes.POINTER(BasisDesc), _ip,
                                    ctypes.POINTER(Params), _c_int, ctypes.POINTER(_c_void_p)]
    L.ftcj_batch_info.argtypes = [P, _c_int, ctypes.POINTER(Info)]
    L.ftcj_batch_jbuild.argtypes = [P, _ip, VPP, VPP, VPP, P]
    L.ftcj_batch_capture.argtypes = [P, _ip, VPP, VPP, VPP, P]
    L.ftcj_batch_replay.argtypes = [P, P]
    L.ftcj_batch_set_wait.argtypes = [P, _c_int]
    L.ftcj_batch_status.argtypes = [P, _ip, P]
    L.ftcj_batch_destroy.argtypes = [P]
    L.ftcj_batch_destroy.restype = None
    L.ftcj_autotune.argtypes = [ctypes.POINTER(Cell), ctypes.POINTER(BasisDesc), _ip, ctypes.POINTER(Params),
                                ctypes.POINTER(Params), _dp]
    L.ftcj_grad.argtypes = [P, _c_int, P, P, P, P]
    L.ftcj_shard_bounds.argtypes = [ctypes.POINTER(ctypes.c_int64), _c_int, _c_int, ctypes.POINTER(ctypes.c_int64)]
    L.ftcj_strerror.argtypes = [_c_int]
    L.ftcj_strerror.restype = ctypes.c_char_p
    L.ftcj_last_error.argtypes = []
    L.ftcj_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        f = getattr(L, name)
        if name not in ("ftcj_plan_destroy", "ftcj_strerror", "ftcj_last_error", "ftcj_batch_destroy"):
            f.restype = _c_int


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        raise FtcjError(f"{what}: {L.ftcj_strerror(rc).decode()} ({rc}): {L.ftcj_last_error().decode()}")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FtcjError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise FtcjError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise FtcjError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise FtcjError(f"{name} must be contiguous")
    return _c_void_p(t.data_ptr())


def _describe(A, xyz, shells, keep):
    """ctypes descriptors of a cell and a basis; arrays are appended to keep."""
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(3, 3)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    keep += [A, xyz]
    cell = Cell()
    for i, v in enumerate(A.ravel()):
        cell.A[i] = float(v)
    sh = (ShellDesc * len(shells))()
    for i, s in enumerate(shells):
        e = np.ascontiguousarray(s.exps, dtype=np.float64)
        c = np.ascontiguousarray(s.coefs, dtype=np.float64)
        keep += [e, c]
        sh[i] = ShellDesc(int(s.centre), int(s.l), 1 if s.spherical else 0, int(len(e)),
                          e.ctypes.data_as(_dp), c.ctypes.data_as(_dp))
    keep.append(sh)
    basis = BasisDesc(int(xyz.shape[0]), xyz.ctypes.data_as(_dp), len(shells), sh)
    return cell, basis


def _params_of(w, precision=FTCJ_PREC_FP64, max_dens=None, chunk_points=0, rho_blocks=0, pair_gcut_eps=0.0,
               contraction=0):
    return Params(float(w.omega), float(w.gcut), float(w.eps_g), float(w.pair_thresh), int(precision),
                  int(max_dens or w.ndens), int(chunk_points), int(rho_blocks), float(pair_gcut_eps), 0, 0,
                  int(contraction), 0, 0, 0.0, (_c_int * 3)(0, 0, 0))


def shard_bounds(class_counts, precision, shard_count):
    """ftcj_shard_bounds: the record ranges [b[s], b[s+1]) of a sharded build
    (host only)."""
    cc = (ctypes.c_int64 * 5)(*[int(c) for c in class_counts])
    out = (ctypes.c_int64 * (int(shard_count) + 1))()
    _check(lib().ftcj_shard_bounds(cc, int(precision), int(shard_count), out), "ftcj_shard_bounds")
    return [int(v) for v in out]


def autotune(w, precision=FTCJ_PREC_FP64):
    """ftcj_autotune for one workload: (chunk_points, rho_blocks, best_ms); a 0
    stands for the plan's own default, so the pair passes straight back to Plan."""
    keep = []
    cell, basis = _describe(w.A, w.xyz, w.shells, keep)
    km = (ctypes.c_int * 3)(*[int(k) for k in w.kmesh])
    pin = _params_of(w, precision)
    pout = Params()
    ms = ctypes.c_double()
    _check(lib().ftcj_autotune(ctypes.byref(cell), ctypes.byref(basis), km, ctypes.byref(pin), ctypes.byref(pout),
                               ctypes.byref(ms)), "ftcj_autotune")
    return pout.chunk_points, pout.rho_blocks, ms.value


class Batch:
    """Independent cells built together (ftcj_batch_*), optionally autotuned,
    optionally captured into one CUDA graph and replayed."""

    def __init__(self, workloads, precision=FTCJ_PREC_FP64, autotune=False, persistent=False):
        L = lib()
        self._keep = []
        n = len(workloads)
        cells = (Cell * n)()
        bases = (BasisDesc * n)()
        prms = (Params * n)()
        km = (ctypes.c_int * (3 * n))()
        for i, w in enumerate(workloads):
            c, b = _describe(w.A, w.xyz, w.shells, self._keep)
            cells[i] = c
            bases[i] = b
            prms[i] = _params_of(w, precision)
            for j in range(3):
                km[3 * i + j] = int(w.kmesh[j])
        self._keep += [cells, bases, prms, km]
        h = _c_void_p()
        flags = (FTCJ_BATCH_AUTOTUNE if autotune else 0) | (FTCJ_BATCH_PERSISTENT if persistent else 0)
        _check(L.ftcj_batch_create(n, cells, bases, km, prms, flags, ctypes.byref(h)), "ftcj_batch_create")
        self._h = h
        self.n = n
        self.infos = []
        for i in range(n):
            inf = Info()
            _check(L.ftcj_batch_info(self._h, i, ctypes.byref(inf)), "ftcj_batch_info")
            self.infos.append(inf.as_dict())

    def _arrays(self, Dks, Jks, EJs):
        import torch
        n = self.n
        nd = (ctypes.c_int * n)()
        a = (_c_void_p * n)()
        b = (_c_void_p * n)()
        c = (_c_void_p * n)()
        for i in range(n):
            inf = self.infos[i]
            d = int(Dks[i].shape[0])
            shp = (d, inf["nk"], inf["nao"], inf["nao"])
            nd[i] = d
            a[i] = _dev_ptr(Dks[i], torch.complex128, shp, f"Dk[{i}]").value
            b[i] = _dev_ptr(Jks[i], torch.complex128, shp, f"Jk[{i}]").value
            c[i] = _dev_ptr(EJs[i], torch.float64, (d,), f"EJ[{i}]").value
        self._last = (nd, a, b, c)
        return nd, a, b, c

    def outputs_like(self, Dks):
        import torch
        Jks = [torch.empty_like(D) for D in Dks]
        EJs = [torch.empty(D.shape[0], dtype=torch.float64, device=D.device) for D in Dks]
        return Jks, EJs

    def jbuild(self, Dks, Jks=None, EJs=None, stream=None):
        if Jks is None:
            Jks, EJs = self.outputs_like(Dks)
        nd, a, b, c = self._arrays(Dks, Jks, EJs)
        _check(lib().ftcj_batch_jbuild(self._h, nd, a, b, c, _stream_ptr(stream)), "ftcj_batch_jbuild")
        return Jks, EJs

    def capture(self, Dks, Jks, EJs, stream):
        nd, a, b, c = self._arrays(Dks, Jks, EJs)
        _check(lib().ftcj_batch_capture(self._h, nd, a, b, c, _stream_ptr(stream)), "ftcj_batch_capture")

    def replay(self, stream=None):
        _check(lib().ftcj_batch_replay(self._h, _stream_ptr(stream)), "ftcj_batch_replay")

    def set_wait(self, wait_log2: int):
        """Wait budget of the persistent launch's back-contraction items (ftcj_batch_set_wait)."""
        _check(lib().ftcj_batch_set_wait(self._h, int(wait_log2)), "ftcj_batch_set_wait")

    def status(self, stream=None) -> int:
        """Error word of the last persistent launch; raises FtcjError (FTCJ_ETIMEOUT) when a wait gave up."""
        w = _c_int(0)
        _check(lib().ftcj_batch_status(self._h, ctypes.byref(w), _stream_ptr(stream)), "ftcj_batch_status")
        return int(w.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ftcj_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A plan for one cell, basis and k-mesh (ftcj_plan_create)."""

    def __init__(self, A, xyz, shells, kmesh, omega, eps_g=1e-14, gcut=0.0, pair_thresh=1e-12,
                 precision=FTCJ_PREC_FP64, max_dens=1, chunk_points=0, rho_blocks=0, pair_gcut_eps=0.0,
                 shard_count=0, shard_index=0, contraction=FTCJ_CONTRACT_WALK, tc_wait_log2=0, classify=False,
                 alpha_cut=0.0, gpw_grid=None):
        L = lib()
        self._keep = []
        cell, basis = _describe(A, xyz, shells, self._keep)
        km = (ctypes.c_int * 3)(*[int(k) for k in kmesh])
        prm = Params(float(omega), float(gcut), float(eps_g), float(pair_thresh), int(precision), int(max_dens),
                     int(chunk_points), int(rho_blocks), float(pair_gcut_eps), int(shard_count), int(shard_index),
                     int(contraction), int(tc_wait_log2), int(classify), float(alpha_cut or 0.0),
                     (_c_int * 3)(*[int(v) for v in (gpw_grid or (0, 0, 0))]))
        self.shard_count = max(1, int(shard_count))
        self.shard_index = int(shard_index)
        h = _c_void_p()
        _check(L.ftcj_plan_create(ctypes.byref(cell), ctypes.byref(basis), km, ctypes.byref(prm), ctypes.byref(h)),
               "ftcj_plan_create")
        self._h = h
        self.max_dens = int(max_dens)
        inf = Info()
        _check(L.ftcj_plan_info(self._h, ctypes.byref(inf)), "ftcj_plan_info")
        self.info = inf.as_dict()
        self.nao = inf.nao
        self.nk = inf.nk
        self.ng_half = int(inf.ng_half)
        self.ncentre = int(np.asarray(xyz).reshape(-1, 3).shape[0])
        self.xyz = np.array(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))

    @classmethod
    def from_workload(cls, w, max_dens=None, precision=FTCJ_PREC_FP64, chunk_points=0, rho_blocks=0,
                      pair_gcut_eps=0.0, shard_count=0, shard_index=0, contraction=FTCJ_CONTRACT_WALK,
                      tc_wait_log2=0, classify=False, alpha_cut=0.0, gpw_grid=None):
        return cls(w.A, w.xyz, w.shells, w.kmesh, w.omega, eps_g=w.eps_g, gcut=w.gcut, pair_thresh=w.pair_thresh,
                   precision=precision, max_dens=max_dens or w.ndens, chunk_points=chunk_points,
                   pair_gcut_eps=pair_gcut_eps, rho_blocks=rho_blocks, shard_count=shard_count,
                   shard_index=shard_index, contraction=contraction, tc_wait_log2=tc_wait_log2,
                   classify=classify, alpha_cut=alpha_cut, gpw_grid=gpw_grid)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ftcj_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- whole build ----
    def jbuild(self, Dk, Jk=None, EJ=None, stream=None):
        import torch
        nd = Dk.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        if Jk is None:
            Jk = torch.empty(shp, dtype=torch.complex128, device=Dk.device)
        if EJ is None:
            EJ = torch.empty(nd, dtype=torch.float64, device=Dk.device)
        _check(lib().ftcj_jbuild(self._h, nd, _dev_ptr(Dk, torch.complex128, shp, "Dk"),
                                 _dev_ptr(Jk, torch.complex128, shp, "Jk"), _dev_ptr(EJ, torch.float64, (nd,), "EJ"),
                                 _stream_ptr(stream)), "ftcj_jbuild")
        return Jk, EJ

    def jbuild_host(self, Dk, Jk=None, EJ=None, stream=None):
        """Host buffers in and out (numpy or CPU torch tensors; pinned ones are
        read and written by the device directly, the outputs are allocated pinned)."""
        import torch
        nd = Dk.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        if isinstance(Dk, np.ndarray):
            Dk = torch.from_numpy(np.ascontiguousarray(Dk, dtype=np.complex128))
        if Jk is None:
            Jk = torch.empty(shp, dtype=torch.complex128, pin_memory=True)
        if EJ is None:
            EJ = torch.empty(nd, dtype=torch.float64, pin_memory=True)
        for t, name, dt, s in ((Dk, "Dk", torch.complex128, shp), (Jk, "Jk", torch.complex128, shp),
                               (EJ, "EJ", torch.float64, (nd,))):
            if t.is_cuda or t.dtype != dt or tuple(t.shape) != tuple(s) or not t.is_contiguous():
                raise FtcjError(f"{name}: contiguous host tensor {dt} {s} required")
        _check(lib().ftcj_jbuild_host(self._h, nd, _c_void_p(Dk.data_ptr()), _c_void_p(Jk.data_ptr()),
                                      _c_void_p(EJ.data_ptr()), _stream_ptr(stream)), "ftcj_jbuild_host")
        return Jk, EJ

    # ---- individual steps ----
    def fold_density(self, Dk, D0n=None, stream=None):
        import torch
        nd = Dk.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        if D0n is None:
            D0n = torch.empty(shp, dtype=torch.float64, device=Dk.device)
        _check(lib().ftcj_fold_density(self._h, nd, _dev_ptr(Dk, torch.complex128, shp, "Dk"),
                                       _dev_ptr(D0n, torch.float64, shp, "D0n"), _stream_ptr(stream)),
               "ftcj_fold_density")
        return D0n

    def rho(self, D0n, rho=None, stream=None):
        import torch
        nd = D0n.shape[0]
        if rho is None:
            rho = torch.empty((nd, self.ng_half), dtype=torch.complex128, device=D0n.device)
        _check(lib().ftcj_rho(self._h, nd, _dev_ptr(D0n, torch.float64, (nd, self.nk, self.nao, self.nao), "D0n"),
                              _dev_ptr(rho, torch.complex128, (nd, self.ng_half), "rho"), _stream_ptr(stream)),
               "ftcj_rho")
        return rho

    def potential(self, rho, W=None, EJ=None, stream=None):
        import torch
        nd = rho.shape[0]
        if W is None:
            W = torch.empty((nd, self.ng_half), dtype=torch.complex128, device=rho.device)
        if EJ is None:
            EJ = torch.empty(nd, dtype=torch.float64, device=rho.device)
        _check(lib().ftcj_potential(self._h, nd, _dev_ptr(rho, torch.complex128, (nd, self.ng_half), "rho"),
                                    _dev_ptr(W, torch.complex128, (nd, self.ng_half), "W"),
                                    _dev_ptr(EJ, torch.float64, (nd,), "EJ"), _stream_ptr(stream)), "ftcj_potential")
        return W, EJ

    def jback(self, W, J0n=None, stream=None):
        import torch
        nd = W.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        if J0n is None:
            J0n = torch.empty(shp, dtype=torch.float64, device=W.device)
        _check(lib().ftcj_jback(self._h, nd, _dev_ptr(W, torch.complex128, (nd, self.ng_half), "W"),
                                _dev_ptr(J0n, torch.float64, shp, "J0n"), _stream_ptr(stream)), "ftcj_jback")
        return J0n

    def unfold_j(self, J0n, Jk=None, stream=None):
        import torch
        nd = J0n.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        if Jk is None:
            Jk = torch.empty(shp, dtype=torch.complex128, device=J0n.device)
        _check(lib().ftcj_unfold_j(self._h, nd, _dev_ptr(J0n, torch.float64, shp, "J0n"),
                                   _dev_ptr(Jk, torch.complex128, shp, "Jk"), _stream_ptr(stream)), "ftcj_unfold_j")
        return Jk

    def grad(self, Dk, EJ=None, grad=None, stream=None):
        """(E_J, dE_J/dR_C) with D^k fixed: device tensors [ndens], [ndens, ncentre, 3]."""
        import torch
        nd = Dk.shape[0]
        shp = (nd, self.nk, self.nao, self.nao)
        nc = self.ncentre
        if EJ is None:
            EJ = torch.empty(nd, dtype=torch.float64, device=Dk.device)
        if grad is None:
            grad = torch.empty((nd, nc, 3), dtype=torch.float64, device=Dk.device)
        _check(lib().ftcj_grad(self._h, nd, _dev_ptr(Dk, torch.complex128, shp, "Dk"),
                               _dev_ptr(EJ, torch.float64, (nd,), "EJ"),
                               _dev_ptr(grad, torch.float64, (nd, nc, 3), "grad"), _stream_ptr(stream)), "ftcj_grad")
        return EJ, grad

    def check_density(self, Dk, stream=None):
        import torch
        nd = Dk.shape[0]
        mi, ma = ctypes.c_double(), ctypes.c_double()
        _check(lib().ftcj_check_density(self._h, nd,
                                        _dev_ptr(Dk, torch.complex128, (nd, self.nk, self.nao, self.nao), "Dk"),
                                        ctypes.byref(mi), ctypes.byref(ma), _stream_ptr(stream)),
               "ftcj_check_density")
        return mi.value, ma.value

    # ---- measurement ----
    def profile_enable(self, max_batches: int):
        _check(lib().ftcj_profile_enable(self._h, int(max_batches)), "ftcj_profile_enable")

    def profile_read(self):
        """(ms per phase dict, batches, kernel launches) since the last read."""
        ms = (ctypes.c_double * len(PHASES))()
        nb = ctypes.c_int()
        nl = ctypes.c_int64()
        _check(lib().ftcj_profile_read(self._h, ms, ctypes.byref(nb), ctypes.byref(nl)), "ftcj_profile_read")
        return dict(zip(PHASES, list(ms))), nb.value, nl.value

    def status(self, stream=None) -> int:
        """ftcj_plan_status: the device error word of the last builds (0: every
        bounded wait completed); clears it."""
        f = ctypes.c_int()
        _check(lib().ftcj_plan_status(self._h, ctypes.byref(f), _stream_ptr(stream)), "ftcj_plan_status")
        return f.value

    def launches_per_batch(self, nd: int = 1) -> int:
        n = ctypes.c_int64()
        _check(lib().ftcj_launches_per_batch(self._h, int(nd), ctypes.byref(n)), "ftcj_launches_per_batch")
        return n.value

    # ---- exports ----
    def gvectors(self):
        out = np.zeros((max(self.ng_half, 1), 3), dtype=np.int32)
        _check(lib().ftcj_get_gvectors(self._h, out.ctypes.data_as(_ip)), "ftcj_get_gvectors")
        return out[:self.ng_half]

    def pairs(self):
        n = int(self.info["npairs"])
        out = np.zeros((max(n, 1), 6), dtype=np.int32)
        _check(lib().ftcj_get_pairs(self._h, out.ctypes.data_as(_ip)), "ftcj_get_pairs")
        return out[:n]

    def groups(self):
        ng = int(self.info["ngroup"])
        nm = ctypes.c_int()
        _check(lib().ftcj_get_groups(self._h, None, None, None, ctypes.byref(nm)), "ftcj_get_groups")
        cen = np.zeros(max(ng, 1), dtype=np.int32)
        ex = np.zeros(max(ng, 1))
        mem = np.zeros((max(nm.value, 1), 3), dtype=np.int32)
        _check(lib().ftcj_get_groups(self._h, cen.ctypes.data_as(_ip), ex.ctypes.data_as(_dp),
                                     mem.ctypes.data_as(_ip), ctypes.byref(nm)), "ftcj_get_groups")
        return cen[:ng], ex[:ng], mem[:nm.value]


def probe_fma_peak(precision: int = 0, stream=None) -> float:
    """Measured FMA throughput (flop/s) of the current GPU: 0 = FP64, 1 = FP32."""
    out = ctypes.c_double()
    _check(lib().ftcj_probe_fma_peak(int(precision), ctypes.byref(out), _stream_ptr(stream)), "ftcj_probe_fma_peak")
    return out.value


def potential_noalloc(A, omega, gvec, rho, W=None, EJ=None, stream=None):
    """ftcj_potential_noalloc: W = 2 v conj(rho) and E_J without a plan and
    without any device allocation inside the library (see include/ftcj.h).
    gvec is a CUDA int32 tensor [ng, 3]; rho a CUDA complex128 tensor
    [ndens, ng]; W and E_J are allocated here by torch when not given."""
    import torch
    nd, ng = int(rho.shape[0]), int(rho.shape[1])
    dev = rho.device
    if W is None:
        W = torch.empty((nd, ng), dtype=torch.complex128, device=dev)
    if EJ is None:
        EJ = torch.empty(nd, dtype=torch.float64, device=dev)
    # the library takes the scratch array's address and the default stream of
    # the CURRENT device: every tensor must live there, and that device is made
    # current for the call
    for name, t in (("gvec", gvec), ("W", W), ("EJ", EJ)):
        if t.device != dev:
            raise FtcjError(f"{name} is on {t.device}, rho on {dev}: all four must share one device")
    Ah = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(A, dtype=np.float64).ravel()])
    with torch.cuda.device(dev):
        _check(lib().ftcj_potential_noalloc(Ah, float(omega), nd, ng, _dev_ptr(gvec, torch.int32, (ng, 3), "gvec"),
                                            _dev_ptr(rho, torch.complex128, (nd, ng), "rho"),
                                            _dev_ptr(W, torch.complex128, (nd, ng), "W"),
                                            _dev_ptr(EJ, torch.float64, (nd,), "EJ"), _stream_ptr(stream)),
               "ftcj_potential_noalloc")
    return W, EJ


def _autograd_function():
    import torch

    class LongRangeCoulomb(torch.autograd.Function):
        """E_J(D^k, R) of a plan, differentiable in both arguments.

        forward(Dk, xyz, plan) -> E_J [ndens]; the plan must have been made for
        the centres xyz (positions are not rebuilt here).
        backward: dE/dD^k = J^k / Nk (the PyTorch gradient d/dRe + i d/dIm of
        the real energy), dE/dR from ftcj_grad (summed over densities with the
        incoming weights)."""

        @staticmethod
        def forward(ctx, Dk, xyz, plan):
            if not np.allclose(xyz.detach().cpu().numpy(), plan.xyz, rtol=0, atol=1e-12):
                raise FtcjError("xyz differs from the geometry the plan was made for")
            Jk, EJ = plan.jbuild(Dk)
            ctx.plan = plan
            ctx.xyz_device = xyz.device
            ctx.xyz_dtype = xyz.dtype
            ctx.save_for_backward(Dk, Jk)
            return EJ

        @staticmethod
        def backward(ctx, gE):
            Dk, Jk = ctx.saved_tensors
            plan = ctx.plan
            gD = gx = None
            if ctx.needs_input_grad[0]:
                gD = gE.to(Jk.dtype).view(-1, 1, 1, 1) * Jk / plan.nk
            if ctx.needs_input_grad[1]:
                _, g = plan.grad(Dk)
                gx = (gE.view(-1, 1, 1) * g).sum(0).to(device=ctx.xyz_device, dtype=ctx.xyz_dtype)
            return gD, gx, None

    return LongRangeCoulomb


_LRC = None


def sharded_jbuild(plan, Dk, group=None, all_reduce=None):
    """The build of a record-sharded plan (shard_count > 1; one plan, GPU and
    rank per share): J^k and E_J of the whole pair list on every rank.  The
    partial rho(G) and J^{0n} of the shards are summed across the ranks of
    `group` between the steps (torch.distributed all-reduce: NCCL on GPUs,
    gloo in host tests; `all_reduce(tensor)` may replace it), and the potential
    and the unfold run on the sums.  Every step is the library's."""
    import torch
    if all_reduce is None:
        import torch.distributed as dist

        def all_reduce(t):
            dist.all_reduce(t, group=group)
    nd = Dk.shape[0]
    Jk = torch.empty(Dk.shape, dtype=torch.complex128, device=Dk.device)
    EJ = torch.empty(nd, dtype=torch.float64, device=Dk.device)
    for b0 in range(0, nd, plan.max_dens):
        b1 = min(nd, b0 + plan.max_dens)
        D0n = plan.fold_density(Dk[b0:b1].contiguous())
        rho = plan.rho(D0n)
        all_reduce(torch.view_as_real(rho))
        W, E = plan.potential(rho)
        J0n = plan.jback(W)
        all_reduce(J0n)
        Jk[b0:b1] = plan.unfold_j(J0n)
        EJ[b0:b1] = E
    return Jk, EJ


def long_range_energy(Dk, xyz, plan):
    """Differentiable E_J (see LongRangeCoulomb): torch.autograd gives dE/dD^k and dE/dR."""
    global _LRC
    if _LRC is None:
        _LRC = _autograd_function()
    return _LRC.apply(Dk, xyz, plan)
