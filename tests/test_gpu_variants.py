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


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_zero_mean_variants_hand_example(lbg, precision):
    """X = {-3, -1, 1, 3}, N = 2, delta = 0.5, worked by hand (the oracle's pin
    of the same case): the additive split ends at [2, -2]; the multiplicative
    split of the zero mean gives two equal codevectors, every row ties and goes
    to the lowest index, and the empty cell keeps 0; re-seeding then splits the
    full cell and ends at [-2, 2]."""
    X = np.array([-3, -1, 1, 3], np.float32)[:, None]
    cases = [  # (multiplicative, reseed, D per pass, final C, final cell table, D)
        (False, False, [20, 20, 13, 4, 4], [2, -2], [1, 1, 0, 0], 4.0),
        (True, False, [20, 20, 20, 20], [0, 0], [0, 0, 0, 0], 20.0),
        (True, True, [20, 20, 20, 13, 4, 4], [-2, 2], [0, 0, 1, 1], 4.0),
    ]
    for mult, reseed, trace_D, C, a, D in cases:
        r = lbg.lbg_train(dev(X), 2, 0.5, 1e-3, split_multiplicative=mult, reseed_empty=reseed,
                          precision=precision)
        assert [rec["D"] for rec in r.records] == trace_D, (mult, reseed)
        np.testing.assert_array_equal(r.C.cpu().numpy()[:, 0], C)
        assert r.assign.cpu().numpy().tolist() == a
        assert r.D == D
