"""Nuclear gradient (ftcj_grad) and the autograd.Function on the GPU, against
the oracle's analytic gradient and central finite differences."""
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


def dk(w):
    import torch
    return torch.from_numpy(np.ascontiguousarray(w.Dk)).cuda()


SYSTEMS = {
    "tiny-triclinic": lambda: W.tiny(seed=61, A=np.array([[5.0, 0.0, 0.0], [0.9, 5.3, 0.0], [-0.4, 0.6, 5.6]]),
                                     kmesh=(2, 1, 1), centres=[[0.1, 0.2, 0.3], [1.5, 0.7, -0.5]], ndens=2),
    "cfg1": lambda: W.cfg1(),
    "cartesian-multishell": lambda: W.tiny(seed=62, A=np.diag([5.2, 4.9, 5.5]), kmesh=(1, 2, 1), spherical=False,
                                           shell_spec=[(0, 0, [1.2]), (0, 1, [1.2]), (0, 2, [0.8]),
                                                       (1, 1, [0.6]), (1, 2, [1.4])]),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_gradient_matches_oracle(orc, F, name):
    import torch
    w = SYSTEMS[name]()
    ref = orc.grad(w)
    for prec in (F.FTCJ_PREC_FP64, F.FTCJ_PREC_SPLIT):
        p = F.Plan.from_workload(w, precision=prec)
        assert p.info["grad_split"] == (1 if prec == F.FTCJ_PREC_SPLIT else 0)
        E, g = p.grad(dk(w))
        torch.cuda.synchronize()
        g = g.cpu().numpy()
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(g - ref).max() <= 1e-10 * scale, (name, prec, np.abs(g - ref).max())
        assert np.abs(g.sum(axis=1)).max() <= 1e-10 * scale  # translational invariance
        p.close()


def test_split_gradient_beyond_the_exact_fp32_powers(orc, F):
    """The split gradient's degree-(L+1) sums hold n^5 in FP32, exact only for
    |n_i| <= 27: a 24-bohr cell with Gcut 8 (|n_i| up to ~34) runs them in FP64
    and must still match the oracle; with Gcut 20 (|n_i| > 63) the split form
    is refused, since its degree-4 powers would round."""
    import torch
    w = W.tiny(seed=63, A=np.diag([24.0, 21.6, 26.4]), centres=[[0.1, 0.2, 0.3], [1.5, 0.7, -0.5]])
    w.gcut = 8.0
    p = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    assert 27 < p.info["n_abs_max"] <= 63 and p.info["grad_split"] == 0
    E, g = p.grad(dk(w))
    _, Eb = p.jbuild(dk(w))
    torch.cuda.synchronize()
    p.close()
    g = g.cpu().numpy()
    ref = orc.grad(w)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(g - ref).max() <= 1e-10 * scale, np.abs(g - ref).max()
    assert abs(float(E[0] - Eb[0])) <= 1e-12 * max(1.0, abs(float(Eb[0])))
    w.gcut = 20.0
    with pytest.raises(F.FtcjError, match="63"):
        F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)


def test_split_gradient_with_pair_cutoffs_is_that_of_the_screened_energy(F):
    """Diamond-like cell, split form, per-pair cutoffs at 1e-12: the gradient
    walks the points the build walks, so it matches central differences
    (h = 1e-4 bohr) of the screened GPU energies and stays within the
    screening error of the whole-sphere gradient."""
    import torch
    w = W.cfg2()
    D = dk(w)
    eps = 1e-12
    full = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    _, g_full = full.grad(D)
    full.close()
    p = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT, pair_gcut_eps=eps)
    assert p.info["pair_g_units_walked"] < 0.5 * p.info["pair_g_units"] and p.info["grad_split"] == 1
    E, g = p.grad(D)
    _, Eb = p.jbuild(D)
    torch.cuda.synchronize()
    p.close()
    g = g.cpu().numpy()
    g_full = g_full.cpu().numpy()
    scale = max(1.0, np.abs(g_full).max())
    assert abs(float(E[0] - Eb[0])) <= 1e-12 * abs(float(Eb[0]))
    assert np.abs(g - g_full).max() <= 1e-8 * scale, np.abs(g - g_full).max()
    assert np.abs(g.sum(axis=1)).max() <= 1e-9 * scale
    h = 1e-4
    x0 = w.xyz.copy()
    for c, d in ((0, 0), (5, 2)):
        e = []
        for sgn in (1, -1):
            w.xyz = x0.copy()
            w.xyz[c, d] += sgn * h
            q = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT, pair_gcut_eps=eps)
            _, Eq = q.jbuild(D)
            torch.cuda.synchronize()
            e.append(float(Eq[0]))
            q.close()
        fd = (e[0] - e[1]) / (2 * h)
        assert abs(fd - g[0, c, d]) <= 1e-6 * scale, (c, d, fd, g[0, c, d])
    w.xyz = x0


def test_gradient_central_differences_of_gpu_energy(F):
    """dE/dR from ftcj_grad against (E(R+h) - E(R-h)) / 2h of GPU builds at displaced
    geometries (new plans), h = 1e-4 bohr."""
    import torch
    w = SYSTEMS["tiny-triclinic"]()
    p = F.Plan.from_workload(w)
    _, g = p.grad(dk(w))
    g = g.cpu().numpy()
    p.close()
    h = 1e-4
    x0 = w.xyz.copy()
    for c in range(2):
        for d in range(3):
            e = []
            for sgn in (1, -1):
                w.xyz = x0.copy()
                w.xyz[c, d] += sgn * h
                q = F.Plan.from_workload(w)
                _, E = q.jbuild(dk(w))
                torch.cuda.synchronize()
                e.append(E.cpu().numpy())
                q.close()
            fd = (e[0] - e[1]) / (2 * h)
            assert np.abs(fd - g[:, c, d]).max() <= 1e-7 * max(1.0, np.abs(fd).max()), (c, d, fd, g[:, c, d])
    w.xyz = x0


def test_autograd_function(F):
    """torch.autograd through long_range_energy: dE/dD^k = J^k/Nk checked by a
    directional central difference (exact for the quadratic E_J), dE/dR by ftcj_grad."""
    import torch
    w = SYSTEMS["tiny-triclinic"]()
    p = F.Plan.from_workload(w)
    D = dk(w).requires_grad_(True)
    xyz = torch.tensor(w.xyz, dtype=torch.float64, requires_grad=True)
    E = F.long_range_energy(D, xyz, p)
    (E * torch.tensor([1.0, 0.5], dtype=torch.float64, device=E.device)).sum().backward()
    rng = np.random.default_rng(3)
    dirn = torch.from_numpy(rng.normal(size=w.Dk.shape) + 1j * rng.normal(size=w.Dk.shape)).cuda()
    h = 1e-3
    with torch.no_grad():
        _, Ep = p.jbuild((D + h * dirn).contiguous())
        _, Em = p.jbuild((D - h * dirn).contiguous())
        fd = float(((Ep - Em) / (2 * h) * torch.tensor([1.0, 0.5], device=Ep.device, dtype=torch.float64)).sum())
    an = float((torch.conj(D.grad) * dirn).real.sum())
    assert abs(fd - an) <= 1e-9 * max(1.0, abs(fd)), (fd, an)
    _, g = p.grad(D.detach())
    gref = (g[0] + 0.5 * g[1]).cpu()
    assert float((xyz.grad - gref).abs().max()) <= 1e-12 * max(1.0, float(gref.abs().max()))
    p.close()


def test_cfg5_slab_gradient_at_full_size(F):
    """The slab + adsorbate cell at full size (~940 AOs, k 3x3x1): the oracle
    cannot differentiate it in seconds, so the analytic GPU gradient is checked
    by properties that hold at any size and by central differences of GPU
    energies (h = 1e-4 bohr) for sampled coordinates: the adsorbate's C and O
    along z and a top-layer atom along x.  Both forms must agree."""
    import torch
    w = W.cfg5()
    D = dk(w)
    p64 = F.Plan.from_workload(w)
    E64, g64 = p64.grad(D)
    p64.close()
    psp = F.Plan.from_workload(w, precision=F.FTCJ_PREC_SPLIT)
    Esp, gsp = psp.grad(D)
    psp.close()
    torch.cuda.synchronize()
    g64 = g64.cpu().numpy()
    gsp = gsp.cpu().numpy()
    scale = max(1.0, np.abs(g64).max())
    assert np.abs(g64.sum(axis=1)).max() <= 1e-9 * scale  # translation sum rule
    assert np.abs(gsp - g64).max() <= 1e-8 * scale
    # E_J is 4.4e6 Eh here: double-float resolves ~2^-47 (7e-15) of |E_J|, so the
    # bound is 1e-8 Eh plus 1e-14 |E_J|
    assert abs(float(Esp[0] - E64[0])) <= 1e-8 + 1e-14 * abs(float(E64[0]))
    nat = w.xyz.shape[0]
    top = int(np.argmax(w.xyz[:nat - 2, 2]))
    h = 1e-4
    x0 = w.xyz.copy()
    for c, d in ((nat - 2, 2), (nat - 1, 2), (top, 0)):
        e = []
        for sgn in (1, -1):
            w.xyz = x0.copy()
            w.xyz[c, d] += sgn * h
            q = F.Plan.from_workload(w)
            _, E = q.jbuild(D)
            torch.cuda.synchronize()
            e.append(float(E[0]))
            q.close()
        fd = (e[0] - e[1]) / (2 * h)
        assert abs(fd - g64[0, c, d]) <= 1e-6 * scale, (c, d, fd, g64[0, c, d])
    w.xyz = x0
