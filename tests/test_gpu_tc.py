"""The tensor-core separable contraction (Sec. 2.4, orthorhombic fully
separable case) against the FP64 oracle.  rho(G) is a sliced bf16 tcgen05
matrix product over (pair record, i, j) with exact level accumulators and
double-float window sums; the back-contraction J'_ijk (Alg. S1) is one over
the sphere's (n_a, n_b) rows with records as the M side.  The bar is the
split form's: max|dJ| <= 1e-8 Eh and |dE_J| <= 1e-8 Eh, plus rho element by
element at 1e-10 of max|rho|.  Every build must also leave the device error
word of the bounded waits at zero."""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

J_TOL = 1e-8
RHO_REL = 1e-10


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def tc_plan(F, w, **kw):
    return F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT, contraction=F.FTCJ_CONTRACT_TC, **kw)


def check_against_oracle(orc, F, w, **kw):
    import torch
    ref = orc.lrj(w, want_j0n=False)
    plan = tc_plan(F, w, **kw)
    try:
        Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
        Jk, EJ = plan.jbuild(Dk)
        nd = min(w.ndens, plan.max_dens)
        rho = plan.rho(plan.fold_density(Dk[:nd].contiguous())).cpu().numpy()
        torch.cuda.synchronize()
        assert plan.status() == 0
        Jk, EJ = Jk.cpu().numpy(), EJ.cpu().numpy()
        dJ = float(np.abs(Jk - ref["Jk"]).max())
        dE = float(np.abs(EJ - ref["EJ"]).max())
        Gh = plan.gvectors()
        idx = {tuple(g): i for i, g in enumerate(ref["G"].tolist())}
        sel = np.array([idx[tuple(g)] for g in Gh.tolist()])
        rref = ref["rho"][:nd, sel]
        drho = float(np.abs(rho - rref).max())
        scale = float(np.abs(rref).max())
        print(f"{w.name}: tc max|dJ|={dJ:.3e} |dE|={dE:.3e} max|drho|={drho:.3e} (max|rho|={scale:.3e}, "
              f"max|J|={np.abs(ref['Jk']).max():.3e}) launches/pass={plan.info['rho_walk_launches']} "
              f"j form={plan.info['j_contraction']} launches={plan.info['j_walk_launches']}")
        assert plan.info["j_contraction"] == F.FTCJ_CONTRACT_TC
        assert drho <= RHO_REL * max(1.0, scale), (w.name, drho)
        assert dJ <= J_TOL and dE <= J_TOL * max(1.0, float(np.abs(ref["EJ"]).max())), (w.name, dJ, dE)
        return plan.info
    finally:
        plan.close()


def test_tc_cfg1_gamma(orc, F):
    check_against_oracle(orc, F, W.cfg1())


def test_tc_orthorhombic_kmesh_two_densities(orc, F):
    spec = [(0, 0, [0.3, 1.1, 4.0]), (0, 1, [0.5, 1.3]), (0, 2, [0.7]),
            (1, 0, [0.25, 2.0]), (1, 1, [0.8]), (1, 2, [0.45])]
    w = W.tiny(seed=41, A=np.diag([4.6, 5.3, 6.1]), kmesh=(2, 1, 2), shell_spec=spec, omega=0.45, ndens=2)
    check_against_oracle(orc, F, w)


def test_tc_reduced_crystal_many_windows(orc, F):
    """The molecular-crystal lattice and G sphere (4,977 half-sphere points,
    5 row tiles or fewer), a reduced basis with two densities: several K
    windows per group, several groups."""
    from tests.test_gpu_launch_shapes import reduced_crystal
    info = check_against_oracle(orc, F, reduced_crystal())
    assert info["ng_half"] == 4977


def test_tc_cfg3_against_split_walk(F):
    """Full molecular crystal: the tensor-core form against the split form's
    walks (both double-float class; the walk is checked against the oracle
    at sampled G and by invariants)."""
    import torch
    w = W.cfg3()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    walk = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    Jw, Ew = walk.jbuild(Dk)
    rw = walk.rho(walk.fold_density(Dk)).cpu().numpy()
    walk.close()
    tc = tc_plan(F, w)
    info = tc.info
    Jt, Et = tc.jbuild(Dk)
    rt = tc.rho(tc.fold_density(Dk)).cpu().numpy()
    torch.cuda.synchronize()
    assert tc.status() == 0
    tc.close()
    dJ = float((Jt - Jw).abs().max())
    dE = float((Et - Ew).abs().max())
    drho = float(np.abs(rt - rw).max())
    print(f"cfg3 tc vs walk: max|dJ|={dJ:.3e} |dE|={dE:.3e} max|drho|={drho:.3e} max|rho|={np.abs(rw).max():.3e} "
          f"|E_J|={float(Ew.abs().max()):.6e} j form={info['j_contraction']} parts={info['j_walk_launches']}")
    assert drho <= RHO_REL * np.abs(rw).max()
    assert dJ <= J_TOL and dE <= J_TOL * max(1.0, float(Ew.abs().max()))


def test_tc_diamond_against_oracle(orc, F):
    """The diamond-like cubic cell (240 AOs, k 4x4x4, 64 densities folded
    into one real D^{0n}), whole, against the oracle's whole build."""
    check_against_oracle(orc, F, W.cfg2())


def test_tc_slab_against_split_walk(F):
    """The slab (orthorhombic, 940 AOs, k 3x3x1, 30 bohr along c with
    vacuum): tensor-core form against the double-float walks."""
    import torch
    w = W.cfg5()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    walk = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    Jw, Ew = walk.jbuild(Dk)
    torch.cuda.synchronize()
    walk.close()
    tc = tc_plan(F, w)
    info = tc.info
    Jt, Et = tc.jbuild(Dk)
    torch.cuda.synchronize()
    assert tc.status() == 0
    tc.close()
    dJ = float((Jt - Jw).abs().max())
    dE = float((Et - Ew).abs().max())
    print(f"slab tc vs walk: max|dJ|={dJ:.3e} |dE|={dE:.3e} |E_J|={float(Ew.abs().max()):.6e} "
          f"j form={info['j_contraction']}")
    assert dJ <= J_TOL and dE <= J_TOL * max(1.0, float(Ew.abs().max()))


def jback_pair(F, w):
    """J^{0n} from the same potential W through the split walk's and the
    tensor-core back-contraction: the difference is the J pass's alone."""
    import torch
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    walk = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    tc = tc_plan(F, w)
    try:
        assert tc.info["j_contraction"] == F.FTCJ_CONTRACT_TC
        assert walk.info["j_contraction"] == F.FTCJ_CONTRACT_WALK
        nd = min(w.ndens, walk.max_dens)
        rho = walk.rho(walk.fold_density(Dk[:nd].contiguous()))
        W, _ = walk.potential(rho)
        Jw = walk.jback(W).cpu().numpy()
        Jt = tc.jback(W).cpu().numpy()
        torch.cuda.synchronize()
        assert tc.status() == 0
        return Jw, Jt, tc.info
    finally:
        walk.close()
        tc.close()


def test_tc_jback_reduced_crystal_same_potential(F):
    from tests.test_gpu_launch_shapes import reduced_crystal
    Jw, Jt, info = jback_pair(F, reduced_crystal())
    d = float(np.abs(Jt - Jw).max())
    print(f"reduced crystal jback: max|dJ0n|={d:.3e} max|J0n|={np.abs(Jw).max():.3e} "
          f"items={info['j_walk_launches']} mma={info['tc_j_mma_flops']:.3e}")
    assert d <= 1e-9


def test_tc_refusals(F):
    with pytest.raises(F.FtcjError, match="orthorhombic"):
        tc_plan(F, W.tiny(seed=42, A=np.array([[5.0, 0.0, 0.0], [1.2, 5.1, 0.0], [0.0, 0.0, 5.5]])))
    with pytest.raises(F.FtcjError, match="split"):
        F.Plan.from_workload(W.cfg1(), precision=F.FTCJ_PREC_FP64, contraction=F.FTCJ_CONTRACT_TC)
    with pytest.raises(F.FtcjError, match="whole sphere"):
        tc_plan(F, W.cfg1(), pair_gcut_eps=1e-12)


def test_tc_waits_give_up_and_report(orc, F):
    """With a wait budget of 2 clock cycles the tensor-core kernels' waits
    between their roles give up at once: the kernels raise the plan's error
    word, drain what they have in flight and return; the call completes, the
    status reports bit 0 (and is cleared by reading it), and the context stays
    usable: a plan with the default budget then matches the oracle."""
    import torch
    w = W.cfg1()
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    short = tc_plan(F, w, tc_wait_log2=1)
    try:
        short.jbuild(Dk)
        torch.cuda.synchronize()
        assert short.status() & 1
        assert short.status() == 0
    finally:
        short.close()
    check_against_oracle(orc, F, w)
