"""Backward of the distortion (differentiable form) vs the oracle's analytic
gradient and FP64 central finite differences, through the C ABI and through
the torch.autograd.Function.

Workload: Gaussian-mixture vectors (L = 32, 512 components with sigma 0.1,
means uniform in [0,1]^32) at reduced size, codebook from the library's LBG.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbg():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    return m


@pytest.fixture(scope="module")
def gmm_problem(lbg):
    from paper_0910_4711_gb300 import synth
    X, _, _ = synth.gmm(4, 16384, L=32, K=512, sigma=0.1)
    Xd = torch.from_numpy(X).cuda()
    C = lbg.lbg_train(Xd, 64, 0.01, 1e-3).C
    # move the codebook off its fixed point (there dD/dC ~ 0 and only rounding is left)
    g = torch.Generator(device="cuda").manual_seed(5)
    C = (C + 0.05 * torch.randn(C.shape, device="cuda", generator=g)).contiguous()
    enc = lbg.vq_encode(Xd, C)
    return X, Xd, C, enc.idx


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_backward_matches_oracle_analytic(lbg, gmm_problem):
    X, Xd, C, idx = gmm_problem
    D, dC, dX, _ = lbg.distortion_backward(Xd, C, idx, grad_D=1.0)
    a = idx.cpu().numpy()
    Cn = C.cpu().numpy().astype(np.float64)
    gC, gX = oracle.grad(X, Cn, a)
    assert rel(dC.cpu().numpy(), gC) < 1e-5
    assert rel(dX.cpu().numpy(), gX) < 1e-6
    assert D == pytest.approx(oracle.distortion_fixed(X, Cn, a), rel=1e-5)


def test_backward_scales_and_is_deterministic(lbg, gmm_problem):
    X, Xd, C, idx = gmm_problem
    _, dC1, dX1, _ = lbg.distortion_backward(Xd, C, idx, grad_D=1.0)
    _, dC2, dX2, _ = lbg.distortion_backward(Xd, C, idx, grad_D=-2.5)
    _, dC3, _, _ = lbg.distortion_backward(Xd, C, idx, grad_D=1.0, want_dX=False)
    assert torch.equal(dC1, dC3)
    torch.testing.assert_close(dC2, -2.5 * dC1, rtol=1e-6, atol=1e-3)
    torch.testing.assert_close(dX2, -2.5 * dX1, rtol=1e-6, atol=1e-6)


def test_backward_finite_differences_away_from_ties(lbg, gmm_problem):
    """FP64 central differences (h = 1e-6) of the true distortion (nearest
    codevector re-found for every perturbation) on a 1024-vector subset, at
    entries whose perturbation cannot change a cell (gap far above h)."""
    X, Xd, C, idx = gmm_problem
    sub = X[:1024]
    subd = torch.from_numpy(sub).cuda()
    Cn = C.cpu().numpy().astype(np.float64)
    a, _, gap = oracle.assign(sub, Cn)
    _, dC, dX, _ = lbg.distortion_backward(subd, C, torch.from_numpy(a).cuda(), grad_D=1.0)
    dC, dX = dC.cpu().numpy(), dX.cpu().numpy()
    h = 1e-6

    def Dtrue(Xv, Cv):
        # FP64 distortion with re-assignment, straight from the definition
        d = ((Xv[:, None, :] - Cv[None, :, :]) ** 2).sum(-1)
        return d.min(1).sum()

    Xs = sub.astype(np.float64)
    rng = np.random.default_rng(0)
    used = np.unique(a)
    for n in rng.choice(used, 8, replace=False):
        for l in rng.choice(32, 2, replace=False):
            Cp, Cm = Cn.copy(), Cn.copy()
            Cp[n, l] += h
            Cm[n, l] -= h
            fd = (Dtrue(Xs, Cp) - Dtrue(Xs, Cm)) / (2 * h)
            assert fd == pytest.approx(dC[n, l], rel=2e-4, abs=2e-3)
    rows = np.flatnonzero(gap > 1e-3)[:16]
    for m in rows:
        for l in rng.choice(32, 2, replace=False):
            Xp, Xm = Xs.copy(), Xs.copy()
            Xp[m, l] += h
            Xm[m, l] -= h
            fd = (Dtrue(Xp, Cn) - Dtrue(Xm, Cn)) / (2 * h)
            assert fd == pytest.approx(dX[m, l], rel=2e-4, abs=2e-4)


def test_autograd_function(lbg, gmm_problem):
    from paper_0910_4711_gb300.autograd import distortion
    X, Xd, C, idx = gmm_problem
    Xg = Xd.clone().requires_grad_(True)
    Cg = C.clone().requires_grad_(True)
    D = distortion(Xg, Cg)
    D.backward()
    D2, dC, dX, _ = lbg.distortion_backward(Xd, C, idx, grad_D=1.0)
    assert float(D.detach()) == pytest.approx(D2, rel=1e-9)
    assert torch.equal(Cg.grad, dC) and torch.equal(Xg.grad, dX)
    # one gradient step on C lowers D (descent direction of the distortion)
    with torch.no_grad():
        C2 = C - 1e-6 * dC
    assert float(distortion(Xd, C2)) < float(D.detach())


def test_autograd_needs_no_host_sync(lbg, gmm_problem):
    """Forward and backward of the autograd function enqueue only: no torch operation on the
    way synchronises with the device (the upstream gradient stays a device scalar), and the
    results are those of the synchronous calls, scaled by the upstream gradient."""
    from paper_0910_4711_gb300.autograd import distortion
    X, Xd, C, idx = gmm_problem
    Xg = Xd.clone().requires_grad_(True)
    Cg = C.clone().requires_grad_(True)
    torch.cuda.synchronize()
    torch.cuda.set_sync_debug_mode("error")
    try:
        D = distortion(Xg, Cg)
        (3.0 * D).backward()
    finally:
        torch.cuda.set_sync_debug_mode(0)
    D2, dC, dX, _ = lbg.distortion_backward(Xd, C, idx, grad_D=3.0)
    assert float(D.detach()) == D2
    assert torch.equal(Cg.grad, dC) and torch.equal(Xg.grad, dX)


def test_backward_async_report(lbg, gmm_problem):
    X, Xd, C, idx = gmm_problem
    buf = lbg.step_result_buffer()
    g = torch.tensor([0.5], device="cuda")
    _, dC, dX, _ = lbg.distortion_backward(Xd, C, idx, grad_scale=g, result_out=buf)
    D, n_exact, status = lbg.read_step_result(buf)
    D2, dC2, dX2, _ = lbg.distortion_backward(Xd, C, idx, grad_D=0.5)
    assert status == 0 and D == D2
    assert torch.equal(dC, dC2) and torch.equal(dX, dX2)


def test_backward_empty_rows(lbg):
    C = torch.randn(8, 16, device="cuda")
    D, dC, dX, _ = lbg.distortion_backward(torch.zeros((0, 16), device="cuda"), C,
                                           torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert D == 0.0 and torch.count_nonzero(dC) == 0
