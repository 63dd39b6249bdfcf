"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times: the 8-image 8x8-block workload (M = 524,288, L = 64, N = 4096) with
one oracle pass over every row; the 64-problem ragged batch (sum M ~ 3.6 M,
L = 16) with one oracle pass per problem; the 64-image 4x4-block workload
(M = 16.8 M, L = 16, N = 4096) on rows sampled for the oracle; the
Gaussian-mixture workload of the differentiation form (M = 262,144, L = 32,
N = 512).  Training runs are checked re-anchored (one oracle allocation from
the GPU's final codebook reproduces its cell table and D), since a single
near-tie may legitimately change a long trajectory.
"""
import numpy as np
import pytest

import oracle
from _gpu_helpers import GAP_TOL, check_assign, check_codebook, check_D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbg():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    return m


def host(t):
    return t.detach().cpu().numpy()


def check_cells(X, a, C_in, C_out, cells):
    """Sampled cells of an update: FP64 mean of the rows the GPU put there (or
    the old codevector for an empty cell) against the GPU's new codevector."""
    X64 = np.asarray(X, np.float64)
    ref = np.asarray(C_in, np.float64)[cells].copy()
    for k, n in enumerate(cells):
        rows = np.flatnonzero(a == n)
        if rows.size:
            ref[k] = X64[rows].mean(0)
    check_codebook(np.asarray(C_out)[cells], ref)


@pytest.fixture(scope="module")
def image8(lbg):
    from paper_0910_4711_gb300 import synth
    X, N = synth.workload("img2048x8_b8_n4096")
    Xd = torch.from_numpy(X).cuda()
    tr = lbg.lbg_train(Xd, N, 0.01, 1e-3, precision="bf16")
    return X, Xd, N, tr


def test_fullsize_image_train_reanchored(lbg, image8):
    X, Xd, N, tr = image8
    C = host(tr.C)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(tr.assign), a_ref, e_ref, gap)
    check_D(tr.D, float(e_ref.sum()))


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_fullsize_image_lloyd_step(lbg, image8, precision):
    X, Xd, N, tr = image8
    C = host(tr.C)
    r = lbg.lbg_lloyd_step(Xd, tr.C, precision=precision)
    s = oracle.lloyd_step(X, C.astype(np.float64))
    a = host(r.assign)
    n_alt = check_assign(X, C, a, s.a, s.e, s.gap)
    check_D(r.D, s.D)
    cells = np.random.default_rng(1).choice(N, 256, replace=False)
    check_cells(X, a, C, host(r.C), cells)
    if n_alt == 0:
        check_codebook(host(r.C), s.C)
    assert r.n_exact < 0.01 * X.shape[0]


def test_fullsize_batched_reanchored(lbg):
    from paper_0910_4711_gb300 import synth
    spec = synth.batched_sets(3000)
    parts = [synth.blocks(synth.make_image(seed, 2048, 2048), 4)[:M] for seed, M, _ in spec]
    Ns = [n for _, _, n in spec]
    row_off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])])
    r = lbg.lbg_train_batched(torch.from_numpy(np.concatenate(parts)).cuda(), row_off, Ns)
    assert r.status == 0 and len(Ns) == 64
    A = host(r.assign)
    for s, X in enumerate(parts):
        C = host(r.codebook(s))
        a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
        check_assign(X, C, A[row_off[s]:row_off[s + 1]], a_ref, e_ref, gap)
        check_D(r.D[s], float(e_ref.sum()))


def test_fullsize_large_train_and_encode_sampled(lbg):
    from paper_0910_4711_gb300 import synth
    X, N = synth.workload("img2048x64_b4_n4096")
    Xd = torch.from_numpy(X).cuda()
    tr = lbg.lbg_train(Xd, N, 0.01, 1e-3, precision="bf16")
    C = host(tr.C)
    rows = np.sort(np.random.default_rng(5).choice(X.shape[0], 20000, replace=False))
    a_ref, e_ref, gap = oracle.assign(X[rows], C.astype(np.float64))
    check_assign(X[rows], C, host(tr.assign)[rows], a_ref, e_ref, gap)
    # encode the same 16.8 M rows in both precisions: the same cells outside near-ties
    for precision in ("bf16", "fp32"):
        enc = lbg.vq_encode(Xd, tr.C, precision=precision)
        check_assign(X[rows], C, host(enc.idx)[rows], a_ref, e_ref, gap)
        # every row, not only the sample: D equals the training run's (same codebook, same
        # exact FP32 distances) up to the summation order of the FP64 total
        check_D(enc.D, tr.D)


def test_fullsize_gmm_backward(lbg):
    from paper_0910_4711_gb300 import synth
    X, _, _ = synth.gmm(4, 262144, 32, 512, 0.1)
    Xd = torch.from_numpy(X).cuda()
    tr = lbg.lbg_train(Xd, 512, 0.01, 1e-3)
    C = host(tr.C).astype(np.float64)
    a = host(tr.assign)
    D, dC, dX, _ = lbg.distortion_backward(Xd, tr.C, tr.assign)
    gC_ref, gX_ref = oracle.grad(X, C, a)
    assert np.abs(host(dC) - gC_ref).max() <= 1e-4 * np.abs(gC_ref).max()
    assert np.abs(host(dX) - gX_ref).max() <= 1e-5 * max(np.abs(gX_ref).max(), 1.0)
    check_D(D, oracle.distortion_fixed(X, C, a))
