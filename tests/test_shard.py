"""The record-sharded build on host ranks, without a GPU: the share bounds
(ftcj_shard_bounds) and the orchestration of `ftcj.sharded_jbuild` (partial
rho and J^{0n} summed across ranks between the library's steps) over two
gloo ranks.  The steps themselves are stood in for by a small linear model
with the same data flow (a partial sum over each rank's records), so that the
sharded result can be compared with the unsharded one exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


@pytest.fixture(scope="module")
def F():
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


def cost(L, precision):
    return 38 * L + 100 if precision == 1 else 4 * L + 24


@pytest.mark.parametrize("precision", [0, 1])
def test_share_bounds_balance_the_walk_cost(F, precision):
    rng = np.random.default_rng(7)
    for _ in range(50):
        counts = [int(c) for c in rng.integers(0, 2000, size=5)]
        n = sum(counts)
        cls = np.repeat(np.arange(5), counts)
        w = np.array([cost(L, precision) for L in cls], dtype=float)
        run = np.concatenate([[0.0], np.cumsum(w)])
        total = run[-1]
        for S in (1, 2, 3, 4, 7, 8):
            b = F.shard_bounds(counts, precision, S)
            assert b[0] == 0 and b[-1] == n and all(b[i] <= b[i + 1] for i in range(S))
            for s in range(1, S):
                # the first record index whose running cost reaches s/S of the total (to rounding)
                target = total * s / S
                eps = 1e-9 * max(1.0, target)
                assert run[b[s]] >= target - eps, (counts, S, s, b[s])
                assert b[s] == 0 or run[b[s] - 1] < target + eps, (counts, S, s, b[s])
            for s in range(S):
                share = run[b[s + 1]] - run[b[s]]
                assert abs(share - total / S) <= 2 * w.max(initial=0.0) + 1e-9, (counts, S, s)


def test_share_bounds_reject_bad_input(F):
    with pytest.raises(F.FtcjError):
        F.shard_bounds([1, 2, 3, 4, 5], 1, 0)
    with pytest.raises(F.FtcjError):
        F.shard_bounds([1, -2, 3, 4, 5], 1, 2)


class LinearModel:
    """Stands in for a plan with the library's data flow: rho_d(G) = sum over
    this plan's records r of a_r(G) <m_r, D0n_d>; W = 2 v conj(rho),
    E = sum v |rho|^2; J0n_d = sum_r m_r Re sum_G a_r(G) W_d(G)."""

    def __init__(self, a, m, v, records, max_dens, nk, nao):
        import torch
        self.a = torch.from_numpy(a[records])
        self.m = torch.from_numpy(m[records])
        self.v = torch.from_numpy(v)
        self.max_dens, self.nk, self.nao = max_dens, nk, nao

    def fold_density(self, Dk):
        return Dk.real.contiguous()

    def rho(self, D0n):
        h = D0n.reshape(D0n.shape[0], -1) @ self.m.T  # [nd, records]
        return h.to(self.a.dtype) @ self.a  # [nd, G]

    def potential(self, rho):
        W = 2.0 * self.v * rho.conj()
        return W, (self.v * rho.abs() ** 2).sum(dim=1)

    def jback(self, W):
        c = (W @ self.a.T).real  # [nd, records]
        return (c @ self.m).reshape(W.shape[0], self.nk, self.nao, self.nao)

    def unfold_j(self, J0n):
        import torch
        return J0n.to(torch.complex128)


def model_inputs(seed=3):
    rng = np.random.default_rng(seed)
    R, G, nk, nao, nd = 37, 23, 2, 4, 3
    a = rng.normal(size=(R, G)) + 1j * rng.normal(size=(R, G))
    m = rng.normal(size=(R, nk * nao * nao))
    v = rng.uniform(0.1, 1.0, size=G)
    cls = np.sort(rng.integers(0, 5, size=R))
    Dk = rng.normal(size=(nd, nk, nao, nao)) + 1j * rng.normal(size=(nd, nk, nao, nao))
    return a, m, v, cls, Dk, nk, nao


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2509_16460_gb300 import ftcj
        a, m, v, cls, Dk, nk, nao = model_inputs()
        counts = [int((cls == L).sum()) for L in range(5)]
        b = ftcj.shard_bounds(counts, 1, world)
        plan = LinearModel(a, m, v, np.arange(b[rank], b[rank + 1]), 2, nk, nao)
        Jk, EJ = ftcj.sharded_jbuild(plan, torch.from_numpy(Dk))
        q.put((rank, b, Jk.numpy(), EJ.numpy()))
    finally:
        dist.destroy_process_group()


def test_sharded_build_over_two_gloo_ranks(F):
    import torch
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    a, m, v, cls, Dk, nk, nao = model_inputs()
    whole = LinearModel(a, m, v, np.arange(len(cls)), 2, nk, nao)

    def no_reduce(t):
        return None

    J_ref, E_ref = F.sharded_jbuild(whole, torch.from_numpy(Dk), all_reduce=no_reduce)
    b = got[0][1]
    assert b[0] == 0 and b[-1] == len(cls) and 0 < b[1] < len(cls)  # both ranks hold records
    for rank, _, Jk, EJ in got:
        np.testing.assert_allclose(Jk, J_ref.numpy(), rtol=0, atol=1e-12 * np.abs(J_ref.numpy()).max())
        np.testing.assert_allclose(EJ, E_ref.numpy(), rtol=1e-13)
