"""GPU tests of plans used together, of walk chunking, of batches of
independent cells (with CUDA-graph replay) and of the walk-shape autotuner,
all against the FP64 CPU oracle."""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

J_TOL = 1e-10
SPLIT_TOL = 1e-8


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def dk(w):
    import torch
    return torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()


def test_two_live_plans_of_different_cells(orc, F):
    """Per-cell data travels with each plan: two plans of different lattices,
    built alternately, each reproduce their own oracle."""
    import torch
    wa = W.tiny(seed=51, A=np.array([[5.0, 0, 0], [1.2, 4.6, 0], [0.4, -0.7, 5.3]]), kmesh=(2, 1, 1))
    wb = W.tiny(seed=52, A=np.diag([6.1, 4.4, 5.0]), kmesh=(1, 2, 2))
    ra, rb = orc.lrj(wa), orc.lrj(wb)
    for prec, tol in ((F.FTCJ_PREC_FP64, J_TOL), (F.FTCJ_PREC_SPLIT, SPLIT_TOL)):
        pa = F.Plan.from_workload(wa, precision=prec)
        pb = F.Plan.from_workload(wb, precision=prec)
        for _ in range(2):
            Ja, Ea = pa.jbuild(dk(wa))
            Jb, Eb = pb.jbuild(dk(wb))
            torch.cuda.synchronize()
            assert np.abs(Ja.cpu().numpy() - ra["Jk"]).max() <= tol
            assert np.abs(Jb.cpu().numpy() - rb["Jk"]).max() <= tol
            assert np.abs(Ea.cpu().numpy() - ra["EJ"]).max() <= tol
            assert np.abs(Eb.cpu().numpy() - rb["EJ"]).max() <= tol
        pa.close()
        pb.close()


@pytest.mark.parametrize("scale,chunk", [(1.0, 64), (1.0, 100), (1.6, 128), (1.6, 256)])
def test_small_walk_chunks(orc, F, scale, chunk):
    """Chunks that start mid-plane and inside the negative half of a plane take
    their state from the closed forms; results must not depend on the chunking.
    (The half spheres hold 132 and 531 points.)"""
    import torch
    A = np.array([[4.4, 0.0, 0.0], [1.1, 4.1, 0.0], [-0.6, 0.9, 4.7]]) * scale
    w = W.tiny(seed=53, A=A, kmesh=(2, 1, 1), omega=0.5)
    ref = orc.lrj(w)
    for prec, tol in ((F.FTCJ_PREC_FP64, J_TOL), (F.FTCJ_PREC_SPLIT, SPLIT_TOL)):
        p = F.Plan.from_workload(w, precision=prec, chunk_points=chunk)
        assert p.info["nchunks"] > 1
        J, E = p.jbuild(dk(w))
        torch.cuda.synchronize()
        assert np.abs(J.cpu().numpy() - ref["Jk"]).max() <= tol, (prec, chunk)
        assert np.abs(E.cpu().numpy() - ref["EJ"]).max() <= tol
        p.close()


def test_rho_blocks_parameter(orc, F):
    import torch
    w = W.tiny(seed=54, kmesh=(1, 1, 2))
    ref = orc.lrj(w)
    for rb in (1, 2, 7):
        p = F.Plan.from_workload(w, rho_blocks=rb)
        J, E = p.jbuild(dk(w))
        torch.cuda.synchronize()
        assert np.abs(J.cpu().numpy() - ref["Jk"]).max() <= J_TOL
        p.close()


def batch_cells():
    cells = sorted(W.cfg4(), key=lambda c: c.nao * c.nk)
    return cells[:6] + cells[20:22]  # small and medium cells of the uneven set


@pytest.mark.parametrize("prec_name", ["fp64", "split"])
def test_batch_against_oracle_and_graph_replay(orc, F, prec_name):
    import torch
    prec = F.FTCJ_PREC_FP64 if prec_name == "fp64" else F.FTCJ_PREC_SPLIT
    tol = J_TOL if prec_name == "fp64" else SPLIT_TOL
    cells = batch_cells()
    B = F.Batch(cells, precision=prec)
    Dks = [dk(w) for w in cells]
    Jks, EJs = B.jbuild(Dks)
    torch.cuda.synchronize()
    refs = [orc.lrj(w, want_j0n=False) for w in cells]
    for w, J, E, r in zip(cells, Jks, EJs, refs):
        assert np.abs(J.cpu().numpy() - r["Jk"]).max() <= tol, w.name
        assert np.abs(E.cpu().numpy() - r["EJ"]).max() <= tol * max(1.0, abs(r["EJ"][0])), w.name
    # the same batch captured once into a CUDA graph and replayed twice
    s = torch.cuda.Stream()
    Jg, Eg = B.outputs_like(Dks)
    torch.cuda.synchronize()
    B.capture(Dks, Jg, Eg, stream=s)
    for _ in range(2):
        for J in Jg:
            J.zero_()
        torch.cuda.synchronize()
        B.replay(stream=s)
        s.synchronize()
        for J, E, J0, E0 in zip(Jg, Eg, Jks, EJs):
            assert float((J - J0).abs().max()) <= 1e-12 * max(1.0, float(J0.abs().max()))
            assert float((E - E0).abs().max()) <= 1e-12 * max(1.0, float(E0.abs().max()))
    B.close()


def test_autotune_picks_a_valid_shape(orc, F):
    import torch
    w = sorted(W.cfg4(), key=lambda c: c.nao * c.nk)[10]
    chunk, rb, ms = F.autotune(w, precision=F.FTCJ_PREC_SPLIT)
    assert chunk in (0, 512, 1024, 2048, 4096) and rb >= 0 and ms > 0  # 0: the plan's own default
    p = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT, chunk_points=chunk, rho_blocks=rb)
    J, E = p.jbuild(dk(w))
    torch.cuda.synchronize()
    ref = orc.lrj(w, want_j0n=False)
    assert np.abs(J.cpu().numpy() - ref["Jk"]).max() <= SPLIT_TOL
    p.close()
    B = F.Batch([w], precision=F.FTCJ_PREC_SPLIT, autotune=True)
    J2, E2 = B.jbuild([dk(w)])
    torch.cuda.synchronize()
    assert np.abs(J2[0].cpu().numpy() - ref["Jk"]).max() <= SPLIT_TOL
    B.close()


def test_persistent_batch_against_oracle_and_graph_replay(orc, F):
    """The persistent batch: the walks, potentials and energies of all cells in
    one launch over a shared work queue, against the oracle per cell, against
    the stream-per-cell batch, and captured into a graph and replayed."""
    import torch
    cells = batch_cells()
    P = F.Batch(cells, precision=F.FTCJ_PREC_SPLIT, persistent=True)
    S = F.Batch(cells, precision=F.FTCJ_PREC_SPLIT)
    try:
        Dks = [dk(w) for w in cells]
        Jks, EJs = P.jbuild(Dks)
        Jss, Ess = S.jbuild(Dks)
        torch.cuda.synchronize()
        assert P.status() == 0
        refs = [orc.lrj(w, want_j0n=False) for w in cells]
        worst = 0.0
        for w, J, E, Js, Es, r in zip(cells, Jks, EJs, Jss, Ess, refs):
            d = float(np.abs(J.cpu().numpy() - r["Jk"]).max())
            worst = max(worst, d)
            assert d <= SPLIT_TOL, w.name
            assert d <= 1e-11, (w.name, d)
            assert np.abs(E.cpu().numpy() - r["EJ"]).max() <= SPLIT_TOL * max(1.0, abs(r["EJ"][0])), w.name
            # the same walks: only the order of the rho-row and energy sums differs
            assert float((J - Js).abs().max()) <= 1e-12 * max(1.0, float(Js.abs().max())), w.name
            assert float((E - Es).abs().max()) <= 1e-12 * max(1.0, float(Es.abs().max())), w.name
        print(f"persistent batch: max|dJ| vs oracle over {len(cells)} cells {worst:.3e}")
        s = torch.cuda.Stream()
        Jg, Eg = P.outputs_like(Dks)
        torch.cuda.synchronize()
        P.capture(Dks, Jg, Eg, stream=s)
        for _ in range(2):
            for J in Jg:
                J.zero_()
            torch.cuda.synchronize()
            P.replay(stream=s)
            s.synchronize()
            assert P.status(stream=s) == 0
            # the energies are fixed-order sums; J^{0n} is scattered with FP64 atomics by the J -> AO map
            for J, E, J0, E0 in zip(Jg, Eg, Jks, EJs):
                assert float((J - J0).abs().max()) <= 1e-12 * max(1.0, float(J0.abs().max()))
                assert float((E - E0).abs().max()) == 0.0
        # only max_dens densities per cell, only split walks without cutoffs
        with pytest.raises(F.FtcjError, match="max_dens"):
            P.jbuild([D[:0] if D.shape[0] > 1 else torch.cat([D, D]) for D in Dks])
        with pytest.raises(F.FtcjError, match="persistent batch"):
            F.Batch(cells[:2], precision=F.FTCJ_PREC_FP64, persistent=True)
    finally:
        P.close()
        S.close()


def test_persistent_batch_wait_gives_up_and_reports(orc, F):
    """A back-contraction item whose cell's potential is not ready within the
    budget (here 2 clock cycles) raises the batch's error word and skips its
    work: the launch ends, the status call returns FTCJ_ETIMEOUT, and the next
    launch with the default budget matches the oracle.  Two small orthorhombic
    cells give fewer structure-factor items than the grid has CTAs, so
    back-contraction items are taken while those items still run and their
    waits run out."""
    import torch
    cells = [W.tiny(seed=61), W.tiny(seed=62, kmesh=(2, 1, 1), ndens=2)]
    B = F.Batch(cells, precision=F.FTCJ_PREC_SPLIT, persistent=True)
    try:
        Dks = [dk(w) for w in cells]
        B.set_wait(1)
        B.jbuild(Dks)
        torch.cuda.synchronize()
        with pytest.raises(F.FtcjError, match="timed out|gave up"):
            B.status()
        B.set_wait(0)
        Jks, EJs = B.jbuild(Dks)
        torch.cuda.synchronize()
        assert B.status() == 0
        for w, J, E in zip(cells, Jks, EJs):
            r = orc.lrj(w, want_j0n=False)
            assert np.abs(J.cpu().numpy() - r["Jk"]).max() <= SPLIT_TOL, w.name
            assert np.abs(E.cpu().numpy() - r["EJ"]).max() <= SPLIT_TOL, w.name
    finally:
        B.close()
