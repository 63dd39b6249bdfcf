"""Opt-in LBG variants (not the paper's defaults) on the GPU vs the oracle:
multiplicative split c (1 +- delta) and empty-cell re-seeding from the largest
cell (see the readings at the top of oracle/lbg_oracle.c)."""
import numpy as np
import pytest

import oracle
from _gpu_helpers import check_assign, check_codebook, check_D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbg():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_multiplicative_split_closed_form(lbg):
    M, N = 64, 8
    X = (np.arange(M, dtype=np.float32) + 1)[:, None]
    r = lbg.lbg_train(dev(X), N, 0.01, 1e-3, split_multiplicative=True)
    t = oracle.lbg_train(X, N, 0.01, 1e-3, split_multiplicative=True)
    np.testing.assert_array_equal(r.C.cpu().numpy()[:, 0], t.C[:, 0])
    assert r.passes_per_stage() == t.passes_per_stage() == [2, 3, 3, 3]


def test_multiplicative_split_image_blocks(lbg):
    from paper_0910_4711_gb300 import synth
    X = synth.blocks(synth.make_image(9, 256, 256), 4)
    r = lbg.lbg_train(dev(X), 32, 0.01, 1e-3, split_multiplicative=True)
    C = r.C.cpu().numpy()
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, r.assign.cpu().numpy(), a_ref, e_ref, gap)
    t = oracle.lbg_train(X, 32, 0.01, 1e-3, split_multiplicative=True)
    if t.near_ties() == 0:
        assert r.passes_per_stage() == t.passes_per_stage()
        check_codebook(C, t.C)


def test_reseed_step_hand_example(lbg):
    """One Lloyd pass whose update leaves cells 2 and 3 empty: counts [2, 4, 0, 0]
    -> cell 2 from cell 1, cell 3 from cell 0 (the oracle's hand example)."""
    X = np.array([[0, 1], [0, 1], [10, 10], [10, 10], [10, 10], [10, 10]], np.float32)
    C = np.array([[0, 1], [10, 10], [100, 100], [-100, -100]], np.float32)
    r = lbg.lbg_lloyd_step(dev(X), dev(C), reseed_empty=True, delta_reseed=0.5)
    np.testing.assert_array_equal(r.C.cpu().numpy(),
                                  [[-0.5, 0.5], [9.5, 9.5], [10.5, 10.5], [0.5, 1.5]])


def test_reseed_train_matches_oracle(lbg):
    rng = np.random.default_rng(3)
    centers = rng.uniform(0, 100, (5, 4))
    X = (centers[rng.integers(0, 5, 400)] + rng.standard_normal((400, 4))).astype(np.float32)
    r = lbg.lbg_train(dev(X), 16, 0.25, 1e-3, reseed_empty=True)
    t = oracle.lbg_train(X, 16, 0.25, 1e-3, reseed_empty=True)
    C = r.C.cpu().numpy()
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, r.assign.cpu().numpy(), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    if t.near_ties() == 0:
        assert r.passes_per_stage() == t.passes_per_stage()
        check_codebook(C, t.C)
        check_D(r.D, t.D)
