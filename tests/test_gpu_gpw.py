"""The classified build (Sec. 2.6) with the DD pair densities on the GPW
route (App. E), against the classified FP64 oracle: J^k element by element
and E_J.  Bars: 1e-10 Eh for the FP64 form and 1e-8 Eh for the split and
tensor-core forms (the GPW route runs in FP64 in the FP64 form; the split form
takes its two grid contractions in double-float, in orthorhombic cells; the
grid keeps every alias of a DD transform below e^{-46} of its peak).  Also: a classified
plan without DD records is the plain build, an explicit denser grid agrees
with the automatic one, the end-to-end call agrees with the device call, and
the plan refuses what it does not run."""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

J_FP64 = 1e-10
J_SPLIT = 1e-8
TRICLINIC = np.array([[6.0, 0.0, 0.0], [1.1, 6.4, 0.0], [-0.7, 0.8, 6.9]])


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def build(F, w, **kw):
    import torch
    plan = F.Plan.from_workload(w, **kw)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    Jk, EJ = plan.jbuild(Dk)
    torch.cuda.synchronize()
    return plan, Jk.cpu().numpy(), EJ.cpu().numpy()


def compare(orc, F, w, acut, tol, ref=None, **kw):
    ref = ref if ref is not None else orc.lrj_classified(w, alpha_cut=acut)
    plan, Jk, EJ = build(F, w, classify=True, alpha_cut=acut, **kw)
    try:
        info = plan.info
        dJ = float(np.abs(Jk - ref["Jk"]).max())
        dE = float(np.abs(EJ - ref["EJ"]).max())
        print(f"{w.name} classified (alpha_cut {info['alpha_cut']:.4g}, precision {kw.get('precision', 0)}, "
              f"contraction {kw.get('contraction', 0)}): max|dJ|={dJ:.3e} |dE|={dE:.3e} "
              f"(max|J|={np.abs(ref['Jk']).max():.3e}, E={ref['EJ']}) DD records {info['dd_pairs']} "
              f"compact {info['npairs']} grid {info['gpw_grid']} separable {info['gpw_separable']} "
              f"GPW launches {info['gpw_launches']}")
        assert info["dd_pairs"] > 0 and info["gpw_launches"] > 0
        assert np.abs(ref["rhoD"]).max() > 1e-3
        assert dJ <= tol, (w.name, dJ)
        assert dE <= tol * max(1.0, float(np.abs(ref["EJ"]).max())), (w.name, dE)
        return info, Jk, EJ
    finally:
        plan.close()


@pytest.mark.parametrize("precision,tol", [(0, J_FP64), (1, J_SPLIT)], ids=["fp64", "split"])
def test_classified_orthorhombic_all_classes(orc, F, precision, tol):
    """alpha_cut = 0.9 makes s, p and d primitives diffuse: DD records of
    classes 0..4, the separable (per-axis table) collocation and integration."""
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    info, _, _ = compare(orc, F, w, 0.9, tol, precision=precision)
    assert info["gpw_separable"] == (2 if precision == 1 else 1)


@pytest.mark.parametrize("precision,tol", [(0, J_FP64), (1, J_SPLIT)], ids=["fp64", "split"])
def test_classified_triclinic(orc, F, precision, tol):
    """A triclinic cell: the Gaussians of the DD records are evaluated point by
    point with their lattice images (the metric Hermite recurrence)."""
    w = W.tiny(seed=7, A=TRICLINIC, kmesh=(2, 1, 2), ndens=2)
    info, _, _ = compare(orc, F, w, 0.9, tol, precision=precision)
    assert info["gpw_separable"] == 0


def test_classified_tensor_core(orc, F):
    """The compact records through the tensor-core contraction, the DD records
    on the grid."""
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    info, _, _ = compare(orc, F, w, 0.9, J_SPLIT, precision=1, contraction=1)
    assert info["contraction"] == 1


@pytest.fixture(scope="module")
def crystal(orc):
    from tests.test_gpu_launch_shapes import reduced_crystal
    w = reduced_crystal()
    return w, orc.lrj_classified(w)


@pytest.mark.parametrize("precision,contraction,tol", [(0, 0, J_FP64), (1, 0, J_SPLIT), (1, 1, J_SPLIT)],
                         ids=["fp64", "split", "tensor-core"])
def test_classified_reduced_crystal_default_cut(orc, F, crystal, precision, contraction, tol):
    """The molecular crystal's lattice and sphere (w = 0.5) with the default
    alpha_cut = w^2/2: the s exponent 0.12 of six centres is diffuse, so their
    s-s pairs (and their images) take the GPW route on the automatic grid."""
    w, ref = crystal
    info, _, _ = compare(orc, F, w, None, tol, ref=ref, precision=precision, contraction=contraction)
    assert abs(info["alpha_cut"] - 0.125) < 1e-15
    assert info["gpw_separable"] == (2 if precision == 1 else 1)


def test_classified_without_diffuse_pairs_is_the_plain_build(F):
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    plain, J0, E0 = build(F, w)
    cls, J1, E1 = build(F, w, classify=True, alpha_cut=0.01)
    try:
        assert cls.info["dd_pairs"] == 0 and cls.info["gpw_launches"] == 0
        # E_J comes from fixed-order sums; the J -> AO map adds with atomics, so J^k
        # agrees to the rounding of its summation order
        assert np.array_equal(E0, E1)
        assert np.abs(J1 - J0).max() <= 1e-14 * float(np.abs(J0).max())
    finally:
        plain.close()
        cls.close()


def test_denser_grid_agrees_with_the_automatic_grid(F):
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    auto, J0, E0 = build(F, w, classify=True, alpha_cut=0.9)
    grid = [int(1.5 * n) for n in auto.info["gpw_grid"]]
    dense, J1, E1 = build(F, w, classify=True, alpha_cut=0.9, gpw_grid=grid)
    try:
        assert list(dense.info["gpw_grid"]) == grid
        d = float(np.abs(J1 - J0).max())
        print(f"grid {auto.info['gpw_grid']} -> {grid}: max|dJ| = {d:.3e}")
        assert d <= 1e-12 * max(1.0, float(np.abs(J0).max()))
        assert np.abs(E1 - E0).max() <= 1e-12 * max(1.0, float(np.abs(E0).max()))
    finally:
        auto.close()
        dense.close()


def test_classified_end_to_end_call(F):
    import torch
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    plan, Jd, Ed = build(F, w, classify=True, alpha_cut=0.9)
    try:
        Dh = torch.from_numpy(np.ascontiguousarray(w.Dk)).pin_memory()
        Jh, Eh = plan.jbuild_host(Dh)
        assert np.abs(Jh.numpy() - Jd).max() <= 1e-13 * max(1.0, float(np.abs(Jd).max()))
        assert np.abs(np.asarray(Eh) - Ed).max() <= 1e-13 * max(1.0, float(np.abs(Ed).max()))
    finally:
        plan.close()


def test_classified_refusals(F):
    import torch
    w = W.tiny(seed=7, kmesh=(2, 1, 2), ndens=2)
    with pytest.raises(F.FtcjError, match="alias"):
        F.Plan.from_workload(w, classify=True, alpha_cut=0.9, gpw_grid=(3, 3, 3))
    plan = F.Plan.from_workload(w, classify=True, alpha_cut=0.9)
    try:
        Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
        with pytest.raises(F.FtcjError, match="classified"):
            plan.rho(plan.fold_density(Dk))
    finally:
        plan.close()
