"""Record-sharded plans (shard_count > 1) on one GPU: the shares' partial rho
and J^{0n}, summed here in one process as the all-reduce across GPUs would sum
them, give the whole plan's J^k and E_J and the oracle's.  The shares
partition the record list exactly."""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def ragged():
    spec = [(0, 0, [0.3, 1.1, 4.0]), (0, 1, [0.5, 1.3]), (0, 2, [0.7]),
            (1, 0, [0.25, 2.0]), (1, 1, [0.8]), (1, 2, [0.45])]
    return W.tiny(seed=41, A=np.diag([3.6, 3.9, 4.1]), kmesh=(2, 2, 1), shell_spec=spec, omega=0.45, ndens=2)


@pytest.mark.parametrize("precision,S,eps", [(0, 2, 0.0), (1, 3, 0.0), (1, 2, 1e-12), (0, 2, 1e-12)])
def test_shards_sum_to_the_whole_build(orc, F, precision, S, eps):
    import torch
    w = ragged()
    ref = orc.lrj(w)
    whole = F.Plan.from_workload(w, precision=precision, pair_gcut_eps=eps)
    shards = [F.Plan.from_workload(w, precision=precision, pair_gcut_eps=eps, shard_count=S, shard_index=s)
              for s in range(S)]
    assert sum(p.info["npairs"] for p in shards) == whole.info["npairs"]
    assert sum(p.info["npairs_ordered"] for p in shards) == whole.info["npairs_ordered"]
    assert all(p.info["npairs"] > 0 for p in shards)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    D0n = shards[0].fold_density(Dk)
    rho = sum(p.rho(D0n) for p in shards)
    Wg, E = shards[0].potential(rho)
    J0n = sum(p.jback(Wg) for p in shards)
    Jk = shards[0].unfold_j(J0n)
    Jw, Ew = whole.jbuild(Dk)
    torch.cuda.synchronize()
    scale = float(Jw.abs().max())
    assert float((Jk - Jw).abs().max()) <= 1e-12 * scale
    assert float((E - Ew).abs().max()) <= 1e-12 * float(Ew.abs().max())
    tol = 1e-10 if precision == 0 else 1e-8
    if eps == 0.0:
        assert np.abs(Jk.cpu().numpy() - ref["Jk"]).max() <= tol
        assert np.abs(E.cpu().numpy() - ref["EJ"]).max() <= tol
    with pytest.raises(F.FtcjError, match="shard plan"):
        shards[0].jbuild(Dk)
    for p in shards + [whole]:
        p.close()


def test_tensor_core_shards_sum_to_the_whole_build(orc, F):
    """The tensor-core form on record shards (what `bench.py --gpus N` runs):
    each share's windows and items hold different records, so the shares'
    slice scales differ from the whole plan's and the sums agree to the
    form's rounding, not bit for bit."""
    import torch
    w = ragged()
    ref = orc.lrj(w)
    kw = dict(precision=F.FTCJ_PREC_SPLIT, contraction=F.FTCJ_CONTRACT_TC)
    whole = F.Plan.from_workload(w, **kw)
    shards = [F.Plan.from_workload(w, shard_count=2, shard_index=s, **kw) for s in range(2)]
    try:
        assert all(p.info["contraction"] == F.FTCJ_CONTRACT_TC for p in shards + [whole])
        assert sum(p.info["npairs"] for p in shards) == whole.info["npairs"]
        Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
        D0n = shards[0].fold_density(Dk)
        rho = sum(p.rho(D0n) for p in shards)
        Wg, E = shards[0].potential(rho)
        J0n = sum(p.jback(Wg) for p in shards)
        Jk = shards[0].unfold_j(J0n)
        Jw, Ew = whole.jbuild(Dk)
        torch.cuda.synchronize()
        assert all(p.status() == 0 for p in shards + [whole])
        scale = float(Jw.abs().max())
        d_whole = float((Jk - Jw).abs().max())
        d_ref = float(np.abs(Jk.cpu().numpy() - ref["Jk"]).max())
        print(f"tc shards: max|dJ| vs whole {d_whole:.3e} (max|J| {scale:.3e}), vs oracle {d_ref:.3e}")
        assert d_whole <= 1e-10 * scale
        assert float((E - Ew).abs().max()) <= 1e-10 * float(Ew.abs().max())
        assert d_ref <= 1e-8
        assert np.abs(E.cpu().numpy() - ref["EJ"]).max() <= 1e-8 * max(1.0, float(np.abs(ref["EJ"]).max()))
    finally:
        for p in shards + [whole]:
            p.close()
