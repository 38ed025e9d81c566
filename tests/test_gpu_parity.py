"""GPU parity: every step of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C-ABI.

Bars: index work (pair list, G set) bit-exact as sets, except entries whose
screening value lies within 1e-9 (relative) of the threshold, where the two
libm's may round differently; floating point to max|dJ| <= 1e-10 Eh and
|dE_J| <= 1e-10 Eh (the FP64-form bound), rho to 1e-11 relative to max|rho|.
"""
import math

import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

J_TOL = 1e-10
E_TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def F(torch_cuda):
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def run_gpu(F, torch, w, max_dens=None):
    plan = F.Plan.from_workload(w, max_dens=max_dens)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    Jk, EJ = plan.jbuild(Dk)
    torch.cuda.synchronize()
    return plan, Jk.cpu().numpy(), EJ.cpu().numpy()


def expand_pairs(plan):
    _, _, mem = plan.groups()
    by_group = {}
    for g, s, k in mem.tolist():
        by_group.setdefault(g, []).append((s, k))
    out = []
    for ga, gb, l1, l2, l3, wgt in plan.pairs().tolist():
        for sa, ka in by_group[ga]:
            for sb, kb in by_group[gb]:
                out.append((sa, ka, sb, kb, l1, l2, l3))
                if wgt == 2:
                    out.append((sb, kb, sa, ka, -l1, -l2, -l3))
    return out


def screen_value(w, sa, ka, sb, kb, L):
    a = w.shells[sa].exps[ka]
    b = w.shells[sb].exps[kb]
    p = a + b
    R = w.xyz[w.shells[sa].centre] - w.xyz[w.shells[sb].centre] - np.asarray(L) @ w.A
    return (2 * math.sqrt(a * b) / p) ** 1.5 * math.exp(-a * b / p * (R @ R))


def compare_pairs(orc, plan, w):
    gpu = expand_pairs(plan)
    assert len(gpu) == len(set(gpu)), "duplicate pair records"
    ref = set(map(tuple, orc.pairs(w).tolist()))
    g = set(gpu)
    for q in g ^ ref:  # only borderline differences are allowed
        v = screen_value(w, q[0], q[1], q[2], q[3], q[4:])
        assert abs(v - w.pair_thresh) <= 1e-9 * w.pair_thresh, (q, v)
    assert plan.info["npairs_ordered"] == len(gpu)


def compare_rho(orc, plan, rho_gpu, ref):
    Gh = plan.gvectors()
    idx = {tuple(g): i for i, g in enumerate(ref["G"].tolist())}
    # the stored half sphere and its negation make up the oracle's full sphere
    full = set(map(tuple, Gh.tolist())) | set(map(tuple, (-Gh).tolist()))
    assert full == set(idx.keys())
    assert len(Gh) * 2 == len(idx)
    sel = np.array([idx[tuple(g)] for g in Gh.tolist()])
    r_ref = ref["rho"][:, sel]
    scale = max(1.0, np.abs(r_ref).max())
    np.testing.assert_allclose(rho_gpu, r_ref, atol=1e-11 * scale, rtol=0)


def full_check(orc, F, torch, w, max_dens=None, steps=True):
    ref = orc.lrj(w)
    plan, Jk, EJ = run_gpu(F, torch, w, max_dens)
    compare_pairs(orc, plan, w)
    dJ = np.abs(Jk - ref["Jk"]).max()
    dE = np.abs(EJ - ref["EJ"]).max()
    assert dJ <= J_TOL, (w.name, dJ)
    assert dE <= E_TOL, (w.name, dE, EJ, ref["EJ"])
    if steps:
        nd = min(w.ndens, plan.max_dens)
        Dk = torch.from_numpy(np.ascontiguousarray(w.Dk[:nd])).cuda()
        D0n = plan.fold_density(Dk)
        D0n_ref = orc.fold_density(w)[:nd]
        np.testing.assert_allclose(D0n.cpu().numpy(), D0n_ref.real, atol=1e-13 * max(1, np.abs(D0n_ref).max()))
        rho = plan.rho(D0n)
        compare_rho(orc, plan, rho.cpu().numpy(), dict(G=ref["G"], rho=ref["rho"][:nd]))
        Wg, EJg = plan.potential(rho)
        assert np.abs(EJg.cpu().numpy() - ref["EJ"][:nd]).max() <= E_TOL
        J0n = plan.jback(Wg)
        np.testing.assert_allclose(J0n.cpu().numpy(), ref["J0n"][:nd].real, atol=J_TOL, rtol=0)
        Jk2 = plan.unfold_j(J0n)
        assert np.abs(Jk2.cpu().numpy() - ref["Jk"][:nd]).max() <= J_TOL
    plan.close()
    return dJ, dE


# ---------------------------------------------------------------------------

def test_cfg1_gamma_two_centre(orc, F, torch_cuda):
    """Gamma-point two-centre cell with Cartesian s+p sharing exponent 1 (a multi-shell group)."""
    w = W.cfg1()
    plan = F.Plan.from_workload(w)
    assert plan.info["npairs_ordered"] == 1118
    assert plan.info["ng_full"] == 340
    assert plan.info["ngroup"] == 8
    plan.close()
    full_check(orc, F, torch_cuda, w)


def test_tiny_spherical_orthorhombic(orc, F, torch_cuda):
    full_check(orc, F, torch_cuda, W.tiny(seed=21))


@pytest.mark.parametrize("kmesh", [(2, 1, 1), (1, 3, 1), (2, 2, 2), (3, 1, 2)])
def test_tiny_kmesh(orc, F, torch_cuda, kmesh):
    full_check(orc, F, torch_cuda, W.tiny(seed=22, kmesh=kmesh, A=np.diag([4.6, 5.1, 4.9])))


def test_triclinic_two_densities(orc, F, torch_cuda):
    A = np.array([[5.2, 0.0, 0.0], [1.9, 4.8, 0.0], [-1.1, 0.8, 5.5]])
    w = W.tiny(seed=23, A=A, kmesh=(2, 1, 2), ndens=2)
    full_check(orc, F, torch_cuda, w)


def test_density_batches_above_max_dens(orc, F, torch_cuda):
    w = W.tiny(seed=24, kmesh=(1, 2, 1), ndens=3)
    full_check(orc, F, torch_cuda, w, max_dens=2)


def test_cartesian_contracted_and_multishell(orc, F, torch_cuda):
    A = np.array([[5.5, 0.3, 0.0], [0.0, 5.0, 0.4], [0.2, 0.0, 6.0]])
    w = W.tiny(seed=25, A=A, kmesh=(2, 1, 1), spherical=False,
               shell_spec=[(0, 0, [1.5]), (0, 1, [1.5]), (0, 2, [1.5]), (1, 1, [0.6]), (1, 2, [0.9])])
    # add a contracted shell (two primitives) sharing one exponent with the s shell of centre 1
    w.shells.append(W.Shell(1, 0, False, np.array([0.6, 2.2]), np.array([0.7, -0.4])))
    w.Dk = W.random_bloch_density(np.random.default_rng(5), w.nao, w.kmesh, 3)[None]
    full_check(orc, F, torch_cuda, w)


def test_ragged_tiles_many_pairs(orc, F, torch_cuda):
    """More than one walker tile per class with a ragged last tile."""
    A = np.diag([3.6, 3.9, 4.1])
    spec = [(0, 0, [0.3, 1.1, 4.0]), (0, 1, [0.5, 1.3]), (0, 2, [0.7]),
            (1, 0, [0.25, 2.0]), (1, 1, [0.8]), (1, 2, [0.45])]
    w = W.tiny(seed=26, A=A, kmesh=(2, 2, 1), shell_spec=spec, omega=0.45)
    full_check(orc, F, torch_cuda, w)


def test_triclinic_cells_of_uneven_batch(orc, F, torch_cuda):
    """Three of the 64 random triclinic cells of the uneven batch (the smallest ones)."""
    cells = W.cfg4()
    cells = sorted(cells, key=lambda c: c.nao * c.nk)[:3]
    for w in cells:
        full_check(orc, F, torch_cuda, w, steps=False)


def test_host_buffer_variant(orc, F, torch_cuda):
    torch = torch_cuda
    w = W.tiny(seed=27, kmesh=(2, 1, 1))
    ref = orc.lrj(w)
    plan = F.Plan.from_workload(w)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).pin_memory()
    Jk, EJ = plan.jbuild_host(Dk)
    assert np.abs(Jk.numpy() - ref["Jk"]).max() <= J_TOL
    assert np.abs(EJ.numpy() - ref["EJ"]).max() <= E_TOL
    plan.close()


def test_host_buffer_paths_agree(F, torch_cuda):
    """Pinned host buffers are used by the device directly, pageable ones go
    through staging copies: every mix gives the device-buffer result (up to the
    order of the J -> AO atomic additions)."""
    torch = torch_cuda
    w = W.tiny(seed=29, kmesh=(2, 2, 1), ndens=2)
    for prec in (F.FTCJ_PREC_FP64, F.FTCJ_PREC_SPLIT):
        plan = F.Plan.from_workload(w, precision=prec)
        Dd = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
        Jd, Ed = plan.jbuild(Dd)
        torch.cuda.synchronize()
        Jd, Ed = Jd.cpu(), Ed.cpu()
        shp = tuple(Dd.shape)
        for pin_in in (True, False):
            for pin_out in (True, False):
                Dh = torch.from_numpy(np.ascontiguousarray(w.Dk))
                if pin_in:
                    Dh = Dh.pin_memory()
                Jh = torch.full(shp, float("nan"), dtype=torch.complex128, pin_memory=pin_out)
                Eh = torch.empty(shp[0], dtype=torch.float64, pin_memory=pin_out)
                plan.jbuild_host(Dh, Jh, Eh)
                scale = float(Jd.abs().max())
                assert float((Jh - Jd).abs().max()) <= 1e-13 * scale, (prec, pin_in, pin_out)
                assert float((Eh - Ed).abs().max()) <= 1e-13 * float(Ed.abs().max()), (prec, pin_in, pin_out)
        plan.close()


def test_host_buffers_full_size_batched(F, torch_cuda):
    """Diamond-like cell (240 AOs, k 4x4x4), split form, with and without
    per-pair cutoffs: three densities in batches of two through the host-buffer
    entry point, page-locked (read and written over the host link by the
    k-mesh transforms) and pageable (staging copies), on repeated calls, give
    the device-buffer build's J^k and E_J (up to the order of the J -> AO
    atomic additions); E_J scales as the square of the density."""
    torch = torch_cuda
    w = W.cfg2()
    D1 = np.ascontiguousarray(w.Dk)
    D = np.concatenate([D1, 0.5 * D1, -0.25 * D1], axis=0)
    for eps in (0.0, 1e-12):
        plan = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT, max_dens=2, pair_gcut_eps=eps)
        Jd, Ed = plan.jbuild(torch.from_numpy(D).cuda())
        torch.cuda.synchronize()
        Jd, Ed = Jd.cpu(), Ed.cpu()
        scale = float(Jd.abs().max())
        assert abs(float(Ed[1]) - 0.25 * float(Ed[0])) <= 1e-12 * abs(float(Ed[0]))
        assert abs(float(Ed[2]) - 0.0625 * float(Ed[0])) <= 1e-12 * abs(float(Ed[0]))
        Dh = torch.from_numpy(D).pin_memory()
        for pin_out in (True, True, False):
            Jh = torch.full(tuple(D.shape), float("nan"), dtype=torch.complex128, pin_memory=pin_out)
            Eh = torch.empty(D.shape[0], dtype=torch.float64, pin_memory=pin_out)
            plan.jbuild_host(Dh, Jh, Eh)
            assert float((Jh - Jd).abs().max()) <= 1e-13 * scale, (eps, pin_out, float((Jh - Jd).abs().max()))
            assert float((Eh - Ed).abs().max()) <= 1e-13 * float(Ed.abs().max()), (eps, pin_out)
        plan.close()


def test_check_density_flags_broken_input(F, torch_cuda):
    torch = torch_cuda
    w = W.tiny(seed=28, kmesh=(2, 1, 1))
    plan = F.Plan.from_workload(w)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    mi, ma = plan.check_density(Dk)
    assert mi < 1e-14 and ma < 1e-13
    bad = Dk.clone()
    bad[0, 1] = bad[0, 1] * (1.0 + 0.5j)  # breaks D^{-k} = conj(D^k)
    mi2, ma2 = plan.check_density(bad)
    assert mi2 > 1e-3
    plan.close()


def test_invalid_arguments_return_errors(F, torch_cuda):
    w = W.tiny(seed=29)
    with pytest.raises(F.FtcjError):
        F.Plan(w.A, w.xyz, w.shells, w.kmesh, omega=-1.0)
    bad = [W.Shell(0, 3, True, np.array([1.0]), np.array([1.0]))]
    with pytest.raises(F.FtcjError, match="unsupported"):
        F.Plan(w.A, w.xyz, bad, w.kmesh, omega=0.3)
    with pytest.raises(F.FtcjError):
        F.Plan(np.zeros((3, 3)), w.xyz, w.shells, w.kmesh, omega=0.3)


def test_empty_half_sphere(orc, F, torch_cuda):
    """A G cut below the shortest reciprocal vector: no G, J = 0, E_J = 0."""
    torch = torch_cuda
    w = W.tiny(seed=30)
    w.gcut = 0.5  # |b_i| >= 2 pi / 6 > 0.5
    plan = F.Plan.from_workload(w)
    assert plan.ng_half == 0
    Jk, EJ = plan.jbuild(torch.from_numpy(w.Dk).cuda())
    assert float(Jk.abs().max()) == 0.0 and float(EJ.abs().max()) == 0.0
    plan.close()


def test_cfg2_diamond_full(orc, F, torch_cuda):
    """Diamond-like cell, 240 spherical AOs, k 4x4x4: every J^k element against the oracle."""
    dJ, dE = full_check(orc, F, torch_cuda, W.cfg2(), steps=False)
    print(f"cfg2 max|dJ|={dJ:.3e} |dE|={dE:.3e}")


def test_cfg3_sampled_rho_and_invariants(orc, F, torch_cuda):
    """Molecular-crystal cell (1056 AOs, k 2x2x2, 2 spins) at full size: rho at sampled G
    against the oracle one by one, E_J against (1/2Nk) sum_k Tr(D^k J^k), Hermiticity."""
    torch = torch_cuda
    w = W.cfg3()
    plan = F.Plan.from_workload(w)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    Jk, EJ = plan.jbuild(Dk)
    D0n = plan.fold_density(Dk)
    rho = plan.rho(D0n).cpu().numpy()
    Gh = plan.gvectors()
    rng = np.random.default_rng(0)
    sel = rng.choice(len(Gh), size=6, replace=False)
    ref = orc.rho_at(w, Gh[sel])
    scale = np.abs(ref).max()
    np.testing.assert_allclose(rho[:, sel], ref, atol=1e-11 * scale, rtol=0)
    Jk = Jk.cpu().numpy()
    EJ = EJ.cpu().numpy()
    for d in range(w.ndens):
        tr = sum(np.trace(w.Dk[d, k] @ Jk[d, k]) for k in range(w.nk)) / (2 * w.nk)
        assert abs(tr.real - EJ[d]) <= 1e-9 * abs(EJ[d])
        herm = np.abs(Jk[d] - np.conj(np.transpose(Jk[d], (0, 2, 1)))).max()
        assert herm <= 1e-12 * np.abs(Jk[d]).max()
    plan.close()


@pytest.mark.parametrize("prec_name", ["fp64", "split"])
def test_cfg5_slab_sampled_rho_and_invariants(orc, F, torch_cuda, prec_name):
    """Slab + adsorbate cell (~940 AOs, k 3x3x1, 20 bohr vacuum) at full size, in
    the launch shape the library picks: rho at sampled G against the oracle one
    by one, E_J against (1/2Nk) sum_k Tr(D^k J^k), Hermiticity of J^k."""
    torch = torch_cuda
    w = W.cfg5()
    prec = F.FTCJ_PREC_FP64 if prec_name == "fp64" else F.FTCJ_PREC_SPLIT
    plan = F.Plan.from_workload(w, precision=prec)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    Jk, EJ = plan.jbuild(Dk)
    rho = plan.rho(plan.fold_density(Dk)).cpu().numpy()
    Gh = plan.gvectors()
    rng = np.random.default_rng(5)
    sel = np.concatenate([[0], rng.choice(len(Gh), size=5, replace=False)])
    ref = orc.rho_at(w, Gh[sel])
    scale = np.abs(ref).max()
    np.testing.assert_allclose(rho[:, sel], ref, atol=(1e-11 if prec_name == "fp64" else 1e-10) * scale, rtol=0)
    Jk = Jk.cpu().numpy()
    EJ = EJ.cpu().numpy()
    tr = sum(np.trace(w.Dk[0, k] @ Jk[0, k]) for k in range(w.nk)) / (2 * w.nk)
    assert abs(tr.real - EJ[0]) <= 1e-9 * abs(EJ[0])
    herm = np.abs(Jk[0] - np.conj(np.transpose(Jk[0], (0, 2, 1)))).max()
    assert herm <= 1e-12 * np.abs(Jk[0]).max()
    plan.close()
