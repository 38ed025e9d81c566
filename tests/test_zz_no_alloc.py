"""The allocation-free potential/energy entry point (ftcj_potential_noalloc).

It serves callers that cannot call cudaMalloc (another allocator owns the
device memory, or allocation is forbidden in their loop), so it takes no plan
and keeps its scratch in a fixed device array inside the library.  Checked
through the C-ABI against ftcj_potential on the same rho and G list, on two
calls in a row (the second call finds the first call's partial sums in the
shared array).  This file is collected last so that a failure here comes
after every other test has run.
"""
import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # same bar as the FP64 parity tests (hartree)


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_16460_gb300 import build
    build.build()
    from paper_2509_16460_gb300 import ftcj
    return ftcj


@pytest.mark.parametrize("make", [lambda: W.cfg1(), lambda: W.tiny(seed=41, kmesh=(2, 1, 2), ndens=3)])
def test_noalloc_matches_potential_twice(F, make):
    import torch
    w = make()
    plan = F.Plan.from_workload(w)
    Dk = torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()
    rho = plan.rho(plan.fold_density(Dk))
    W_ref, E_ref = plan.potential(rho)
    gvec = torch.from_numpy(np.ascontiguousarray(plan.gvectors())).cuda()
    for _ in range(2):
        W2, E2 = F.potential_noalloc(w.A, w.omega, gvec, rho)
        torch.cuda.synchronize()
        assert float((W2 - W_ref).abs().max()) <= TOL
        assert float((E2 - E_ref).abs().max()) <= TOL
        assert torch.isfinite(E2).all()
    plan.close()


def test_noalloc_rejects_sizes_beyond_the_array(F):
    import torch
    ng = 256 * 4097  # 4097 blocks
    rho = torch.zeros((4, ng), dtype=torch.complex128, device="cuda")
    gvec = torch.ones((ng, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FtcjError, match="FTCJ_NOALLOC_MAX_PARTIALS"):
        F.potential_noalloc(np.eye(3) * 5.0, 0.4, gvec, rho)
