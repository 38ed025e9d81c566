"""The launch shapes the molecular-crystal cell runs at full size, checked
element by element against the FP64 oracle on a cell small enough for the
oracle: the same orthorhombic lattice (14.0 x 17.8 x 12.9 bohr), omega 0.5 and
2 x 2 x 2 k-mesh, so the same 9,954-point G sphere (4,977 stored half-sphere
points), with two densities in one call, but a reduced basis (one six-ring
and two H-like centres, s p d shells).

With 4096-point walk chunks the half sphere takes two chunks, and shared
memory holds the one-kernel walks below three blocks per SM, so the split
form runs its structure-factor walk as two class parts (classes 3-4, then
0-2) over both chunks and both densities, and its back-contraction as two
class parts side by side on two streams: the shape the full cell runs.  Each
shape is checked on J^k and E_J against the oracle (Alg. 1, Alg. S1, Eq. FT of
J), at the contract bound and at a bar near the measured level, so that a
regression of the double-float path by orders of magnitude does not pass."""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPLIT_J_TOL = 1e-8     # the split form's bound (Eh)
FP64_J_TOL = 1e-10     # the FP64 form's bound (Eh)
MEASURED_J_BAR = 1e-11  # both forms measure ~1e-13 .. 1e-12 here: a 10x-100x margin


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def reduced_crystal():
    w3 = W.cfg3()
    xyz = np.vstack([w3.xyz[0:6], w3.xyz[24:26]])
    spec = []
    for c in range(6):
        spec += [(c, 0, [0.12, 1.5, 20.0]), (c, 1, [0.5]), (c, 2, [0.8])]
    for c in (6, 7):
        spec += [(c, 0, [0.15, 2.0]), (c, 1, [0.6])]
    return W.tiny(seed=36, A=w3.A, centres=xyz, shell_spec=spec, kmesh=(2, 2, 2), omega=0.5, ndens=2, nocc=8)


@pytest.fixture(scope="module")
def case(orc):
    w = reduced_crystal()
    return w, orc.lrj(w, want_j0n=False)


def build(F, w, **kw):
    import torch
    plan = F.Plan.from_workload(w, **kw)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    Jk, EJ = plan.jbuild(Dk)
    torch.cuda.synchronize()
    return plan, Jk.cpu().numpy(), EJ.cpu().numpy()


def errors(Jk, EJ, ref):
    return float(np.abs(Jk - ref["Jk"]).max()), float(np.abs(EJ - ref["EJ"]).max())


def test_class_split_multichunk_two_densities_against_oracle(F, case):
    w, ref = case
    parts, Jp, Ep = build(F, w, precision=F.FTCJ_PREC_SPLIT, chunk_points=4096)
    # 512-point chunks keep three one-kernel J blocks per SM; an explicit block
    # count runs the one-kernel structure-factor walk
    whole, Jw, Ew = build(F, w, precision=F.FTCJ_PREC_SPLIT, chunk_points=512, rho_blocks=2 * 152)
    try:
        assert parts.info["ng_half"] == 4977
        assert parts.info["nchunks"] == 2 and whole.info["nchunks"] > 2
        assert w.ndens == 2 and parts.max_dens == 2
        # rho walk and J walk each in two class launches against one
        assert (parts.info["rho_walk_launches"], parts.info["j_walk_launches"]) == (2, 2)
        assert (whole.info["rho_walk_launches"], whole.info["j_walk_launches"]) == (1, 1)
        assert parts.launches_per_batch() == whole.launches_per_batch() + 2
        assert all(n > 0 for n in parts.info["pairs_by_class"])
        scale = np.abs(ref["Jk"]).max()
        for name, Jk, EJ in (("class parts", Jp, Ep), ("one kernel", Jw, Ew)):
            dJ, dE = errors(Jk, EJ, ref)
            print(f"split {name}: max|dJ|={dJ:.3e} |dE|={dE:.3e} (max|J|={scale:.3e}, E_J={ref['EJ']})")
            assert dJ <= SPLIT_J_TOL and dE <= SPLIT_J_TOL, (name, dJ, dE)
            assert dJ <= MEASURED_J_BAR, (name, dJ)
            assert dE <= MEASURED_J_BAR * max(1.0, float(np.abs(ref["EJ"]).max())), (name, dE)
        # the two launch shapes differ only in summation order
        assert np.abs(Jp - Jw).max() <= 1e-12 * scale
    finally:
        parts.close()
        whole.close()


def test_fp64_form_multichunk_two_densities_against_oracle(F, case):
    w, ref = case
    plan, Jk, EJ = build(F, w, precision=F.FTCJ_PREC_FP64, chunk_points=4096)
    try:
        assert plan.info["nchunks"] == 2
        dJ, dE = errors(Jk, EJ, ref)
        print(f"fp64: max|dJ|={dJ:.3e} |dE|={dE:.3e}")
        assert dJ <= FP64_J_TOL and dE <= FP64_J_TOL * max(1.0, float(np.abs(ref["EJ"]).max()))
        assert dJ <= MEASURED_J_BAR
    finally:
        plan.close()


def test_class_split_multichunk_with_pair_cutoffs_against_oracle(F, case):
    """The same shape with per-pair G cutoffs (Sec. 2.5 screening, eps 1e-12):
    radius-sorted tiles, lines cut to each tile's radius, in both class parts
    and both chunks; the result differs from the whole-sphere oracle only by
    the screened-out terms."""
    w, ref = case
    plan, Jk, EJ = build(F, w, precision=F.FTCJ_PREC_SPLIT, chunk_points=4096, pair_gcut_eps=1e-12)
    try:
        info = plan.info
        assert info["nchunks"] == 2
        assert 0 < info["pair_g_units_screened"] <= info["pair_g_units_walked"] < info["pair_g_units"]
        dJ, dE = errors(Jk, EJ, ref)
        frac = info["pair_g_units_walked"] / info["pair_g_units"]
        print(f"split + pair cutoffs: walked {frac:.3f} of the units, max|dJ|={dJ:.3e} |dE|={dE:.3e}")
        assert dJ <= SPLIT_J_TOL and dE <= SPLIT_J_TOL, (dJ, dE)
    finally:
        plan.close()


def test_fp64_form_with_pair_cutoffs_against_oracle_and_split(F, case):
    """Per-pair G cutoffs in the FP64 walks (Sec. 2.5 screening, eps 1e-12):
    the same radius-sorted tiles and cut lines as the split form, so the two
    forms agree to the split form's rounding, and both differ from the
    whole-sphere oracle only by the screened-out terms."""
    w, ref = case
    f64, Jf, Ef = build(F, w, precision=F.FTCJ_PREC_FP64, chunk_points=4096, pair_gcut_eps=1e-12)
    spl, Js, Es = build(F, w, precision=F.FTCJ_PREC_SPLIT, chunk_points=4096, pair_gcut_eps=1e-12)
    try:
        assert f64.info["pair_g_units_walked"] == spl.info["pair_g_units_walked"] < f64.info["pair_g_units"]
        dJ, dE = errors(Jf, Ef, ref)
        d_forms = float(np.abs(Jf - Js).max())
        print(f"fp64 + pair cutoffs: max|dJ| vs oracle {dJ:.3e} |dE| {dE:.3e}; vs the split form {d_forms:.3e}")
        assert dJ <= SPLIT_J_TOL and dE <= SPLIT_J_TOL
        assert d_forms <= MEASURED_J_BAR
    finally:
        f64.close()
        spl.close()
