"""Plan creation refuses bad or unsupported input on the host, before any
device call: every case below fails with its own error code and message on
a machine without a GPU.  (The split form is given an explicit walk chunk,
since its default chunk is sized from the device's shared memory.)"""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W


@pytest.fixture(scope="module")
def F():
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def base():
    return W.tiny(seed=71)


def plan_of(F, w, **kw):
    kw.setdefault("chunk_points", 4096)
    return F.Plan.from_workload(w, **kw)


def _singular(w):
    w.A = np.array([[5.0, 0.0, 0.0], [5.0, 0.0, 0.0], [0.0, 0.0, 6.0]])


def _nan_lattice(w):
    w.A = w.A.copy()
    w.A[1, 2] = np.nan


def _kmesh_zero(w):
    w.kmesh = (0, 1, 1)


def _kmesh_large(w):
    w.kmesh = (17, 1, 1)


def _omega(w):
    w.omega = 0.0


def _pair_thresh(w):
    w.pair_thresh = 1.0


def _l3(w):
    w.shells.append(W.Shell(0, 3, True, np.array([1.0]), np.array([1.0])))


def _neg_exp(w):
    w.shells[0] = W.Shell(0, 0, True, np.array([-0.5]), np.array([1.0]))


def _diffuse(w):
    w.shells.append(W.Shell(1, 0, True, np.array([1e-4]), np.array([1.0])))


def _centre(w):
    w.shells.append(W.Shell(5, 0, True, np.array([1.0]), np.array([1.0])))


CASES = [
    ("singular lattice", _singular, {}, "invalid argument", "singular lattice"),
    ("non-finite lattice", _nan_lattice, {}, "invalid argument", "non-finite lattice"),
    ("k-mesh 0", _kmesh_zero, {}, "invalid argument", "k-mesh"),
    ("k-mesh 17", _kmesh_large, {}, "unsupported input", "above 16"),
    ("omega 0", _omega, {}, "invalid argument", "omega"),
    ("pair_thresh 1", _pair_thresh, {}, "invalid argument", "pair_thresh"),
    ("f shell", _l3, {}, "unsupported input", "FTCJ_LMAX"),
    ("negative exponent", _neg_exp, {}, "invalid argument", "exponents"),
    ("diffuse exponent", _diffuse, {}, "unsupported input", "too diffuse"),
    ("shell centre", _centre, {}, "invalid argument", "centre out of range"),
    ("precision", None, {"precision": 7}, "unsupported input", "precision"),
    ("chunk 32", None, {"chunk_points": 32}, "invalid argument", "chunk_points"),
    ("negative cutoff eps", None, {"pair_gcut_eps": -1.0, "precision": 1}, "invalid argument", "pair_gcut_eps"),
    ("contraction 2", None, {"contraction": 2, "precision": 1}, "invalid argument", "contraction"),
    ("wait budget 41", None, {"tc_wait_log2": 41, "precision": 1, "contraction": 1}, "invalid argument",
     "tc_wait_log2"),
    ("classify 2", None, {"classify": 2}, "invalid argument", "classify"),
    ("classified shard", None, {"classify": True, "shard_count": 2, "shard_index": 0}, "unsupported input",
     "record-sharded"),
    ("alpha_cut nan", None, {"classify": True, "alpha_cut": float("nan")}, "invalid argument", "alpha_cut"),
    ("classified with cutoffs", None, {"classify": True, "pair_gcut_eps": 1e-12}, "unsupported input",
     "classified plan"),
]


@pytest.mark.parametrize("name,edit,kw,kind,msg", CASES, ids=[c[0] for c in CASES])
def test_plan_refuses(F, name, edit, kw, kind, msg):
    w = base()
    if edit:
        edit(w)
    with pytest.raises(F.FtcjError) as e:
        plan_of(F, w, **kw)
    assert kind in str(e.value) and msg in str(e.value), str(e.value)


def test_line_longer_than_chunk(F):
    """A 64-point walk chunk cannot hold a G line of a 24-bohr cell at Gcut 12
    (about 90 points)."""
    w = W.tiny(seed=72, A=np.diag([24.0, 21.6, 26.4]))
    w.gcut = 12.0
    with pytest.raises(F.FtcjError, match="longer than the walk chunk"):
        plan_of(F, w, chunk_points=64)


def test_split_form_needs_exact_fp32_powers(F):
    """The split walks hold n^i (i <= 4) as exact FP32 integers: |n_i| <= 63.
    Gcut 20 in a 24-bohr cell reaches |n_i| ~ 84, refused; the FP64 form takes
    the same cell past the check (it then stops at its first device call
    here, with a CUDA error rather than an input error)."""
    w = W.tiny(seed=73, A=np.diag([24.0, 21.6, 26.4]))
    w.gcut = 20.0
    with pytest.raises(F.FtcjError) as e:
        plan_of(F, w, precision=F.FTCJ_PREC_SPLIT)
    assert "unsupported input" in str(e.value) and "63" in str(e.value)
    try:
        plan_of(F, w, precision=F.FTCJ_PREC_FP64).close()
    except F.FtcjError as err:
        assert "unsupported" not in str(err) and "invalid" not in str(err), str(err)
