"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-derive the oracle's own code path: they use exact
integer / rational brute force on tiny inputs, closed forms of LBG on inputs
whose answer is known (uniform scalar quantizer, identical vectors, separated
blobs), a hand-derived worked example (tests/golden), invariants of the
Lloyd iteration, an independent library (scipy.cluster.vq) and finite
differences for the gradient.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _int_problem(rng, M, N, L, lo=-3, hi=4):
    X = rng.integers(lo, hi, size=(M, L))
    C = rng.integers(lo, hi, size=(N, L))
    return X, C


# ---------------------------------------------------------------- allocation
def test_assign_exact_bruteforce_tiny():
    """Cell allocation (Alg. 1; Sec. 2.2 step 1) on small integer inputs
    against exact integer arithmetic over every codevector, ties to the
    lowest index; gap against exact rationals."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        M, N, L = int(rng.integers(1, 13)), int(rng.integers(1, 5)), int(rng.integers(1, 4))
        X, C = _int_problem(rng, M, N, L)
        a, e, gap = oracle.assign(X.astype(np.float32), C.astype(np.float64))
        for m in range(M):
            d = [sum(int(X[m, l] - C[n, l]) ** 2 for l in range(L)) for n in range(N)]
            best = min(range(N), key=lambda n: (d[n], n))
            assert a[m] == best
            assert e[m] == d[best]
            if N == 1:
                assert gap[m] == math.inf
            else:
                rest = sorted(d)
                d1, d2 = rest[0], rest[1]
                if d1 == 0:
                    assert gap[m] == (math.inf if d2 > 0 else 0.0)
                else:
                    assert gap[m] == pytest.approx(float(Fraction(d2 - d1, d1)), rel=1e-15)


def test_assign_matches_scipy_vq():
    """Nearest codevector on random real data against scipy.cluster.vq.vq
    (Euclidean distance), an implementation independent of the oracle."""
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3000, 7)).astype(np.float32)
    C = rng.standard_normal((37, 7))
    a, e, gap = oracle.assign(X, C)
    code, dist = vq.vq(X.astype(np.float64), C)
    safe = gap > 1e-9
    assert np.array_equal(a[safe], code[safe])
    np.testing.assert_allclose(e, dist ** 2, rtol=1e-12)


def test_assign_threads_do_not_change_results():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((5001, 5)).astype(np.float32)
    C = rng.standard_normal((64, 5))
    r1 = oracle.assign(X, C, nthreads=1)
    r4 = oracle.assign(X, C, nthreads=4)
    for u, v in zip(r1, r4):
        assert np.array_equal(u, v)


# ------------------------------------------------------------------ updation
def test_update_exact_rational_centroids():
    """Updation (Alg. 1; Sec. 2.2 step 3): centroid of each cell in exact
    rationals; an empty cell keeps its codevector."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        M, N, L = int(rng.integers(1, 15)), int(rng.integers(1, 6)), int(rng.integers(1, 4))
        X = rng.integers(-50, 50, size=(M, L))
        a = rng.integers(0, N, size=M)
        C_in = rng.standard_normal((N, L))
        C_out, counts = oracle.update(X.astype(np.float32), a, C_in)
        for n in range(N):
            rows = [m for m in range(M) if a[m] == n]
            assert counts[n] == len(rows)
            for l in range(L):
                if rows:
                    exact = Fraction(sum(int(X[m, l]) for m in rows), len(rows))
                    assert C_out[n, l] == float(exact)
                else:
                    assert C_out[n, l] == C_in[n, l]


def test_mean_is_centroid():
    """Initial codebook (Alg. 1 'centroid(input)', Table 1): the mean of an
    arithmetic progression is its midpoint; random data against numpy."""
    X = (np.arange(101, dtype=np.float32) * 3 - 40)[:, None]
    assert oracle.mean(X)[0, 0] == 110.0  # (-40 + 260) / 2
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((777, 9)).astype(np.float32)
    np.testing.assert_allclose(oracle.mean(Y)[0], Y.astype(np.float64).mean(0), rtol=0,
                               atol=1e-15)


def test_split_interleaves_plus_then_minus():
    """Codebook splitting (Alg. 1; Sec. 3.2): [c+delta], [c-delta] per centroid."""
    C = np.array([[1.0, 2.0], [-4.0, 0.5]])
    S = oracle.split(C, 0.25)
    np.testing.assert_array_equal(S, [[1.25, 2.25], [0.75, 1.75], [-3.75, 0.75], [-4.25, 0.25]])


# ------------------------------------------------------------- whole design
@pytest.mark.parametrize("theta", [0.0, 1e-3])
@pytest.mark.parametrize("k,j", [(3, 1), (4, 2), (6, 3), (8, 4), (9, 9)])
def test_uniform_scalar_quantizer_closed_form(k, j, theta):
    """L = 1, X = each integer 0..2^k-1 once, N = 2^j.  Every split cuts each
    cell exactly in half at a half-integer (no ties), so LBG ends with cells of
    w = 2^(k-j) consecutive integers, codevectors at the cell midpoints in
    descending order (child 2i = c+delta comes first), D = M (w^2 - 1) / 12,
    and 2 passes at N = 1 and 3 at every later stage -- except a last stage
    with w = 1, whose second pass reaches D = 0 and ends the stage there.
    theta = 0 must give the same result: a repeated D has ratio 0 <= 0."""
    M, N = 2 ** k, 2 ** j
    rng = np.random.default_rng(k * 10 + j)
    X = rng.permutation(M).astype(np.float32)[:, None]
    t = oracle.lbg_train(X, N, delta=0.25, theta=theta, max_passes=50)
    w = M // N
    mids = np.array([(c * w + (c + 1) * w - 1) / 2.0 for c in range(N)])[::-1]
    assert t.status == oracle.OK
    np.testing.assert_array_equal(t.C[:, 0], mids)
    assert t.D == M * (w * w - 1) / 12.0
    expect_passes = [2] + [3] * j
    if w == 1:
        expect_passes[-1] = 2
    assert t.passes_per_stage() == expect_passes
    expect_a = (N - 1) - (X[:, 0].astype(np.int64) // w)
    np.testing.assert_array_equal(t.a, expect_a)


def test_identical_vectors_zero_distortion():
    """All input vectors equal: D == 0 ends every stage (ratio 0/0 avoided),
    ties go to the lowest index, empty cells keep their codevector."""
    x = np.array([3.0, -1.5], np.float32)
    X = np.tile(x, (10, 1))
    d = 0.25
    t = oracle.lbg_train(X, 4, delta=d, theta=1e-3)
    expect = np.array([x + d, x - d, x, x - 2 * d], np.float64)
    np.testing.assert_array_equal(t.C, expect)
    assert t.D == 0.0
    assert np.all(t.a == 2)
    assert t.passes_per_stage() == [1, 2, 1]
    np.testing.assert_array_equal(t.trace_D, [0.0, 10 * 2 * d * d, 0.0, 0.0])
    # a near-tie is a gap <= the tolerance: right after the first split every
    # row is equally far from both children (gap exactly 0), and nowhere else
    t0 = oracle.lbg_train(X, 4, delta=d, theta=1e-3, near_tol=0.0)
    assert t0.trace_near.tolist() == [0, 10, 0, 0]


def test_separated_blobs_end_at_blob_means():
    """Four tight blobs spaced along (1,1,1): LBG to N = 4 ends with the blob
    sample means (order fixed by the splits: largest first)."""
    rng = np.random.default_rng(3)
    centers = [-30.0, -10.0, 10.0, 30.0]
    parts = [t + 0.5 * rng.standard_normal((60, 3)) for t in centers]
    X = np.concatenate(parts).astype(np.float32)
    t = oracle.lbg_train(X, 4, delta=0.01, theta=1e-6)
    means = np.array([p.astype(np.float32).astype(np.float64).mean(0) for p in parts])[::-1]
    np.testing.assert_allclose(t.C, means, rtol=1e-12, atol=1e-12)


def test_stop_rule_golden_l1():
    """Hand-derived worked example (tests/golden/stop_rule_l1.json) that tells
    the Sec. 2.2 stop test (divide by D_m) from the Sec. 3.2 one (divide by
    D_{m-1}), checks '<=' at ratio 0, and pins every pass's distortion."""
    with open(os.path.join(GOLDEN, "stop_rule_l1.json")) as f:
        g = json.load(f)
    X = np.array(g["X"], np.float32)[:, None]
    t = oracle.lbg_train(X, g["N"], g["delta"], g["theta"])
    assert t.trace_n.tolist() == g["trace_n"]
    D_exact = [n / d for n, d in zip(g["trace_D_num"], g["trace_D_den"])]
    np.testing.assert_allclose(t.trace_D, D_exact, rtol=1e-14)
    np.testing.assert_array_equal(t.C, g["final_C"])
    assert t.a.tolist() == g["final_a"]
    assert t.D == g["final_D"]


def test_max_passes_cap_warns_and_continues():
    """A stage stopped by the pass cap returns WARN_MAXPASS; training still
    reaches N codevectors; each stage ran at most max_passes passes."""
    X = np.array([0, 2, 2, 3, 5, 6, 15], np.float32)[:, None]
    t = oracle.lbg_train(X, 2, 0.5, 0.3, max_passes=2)
    assert t.status == oracle.WARN_MAXPASS
    assert t.passes_per_stage() == [2, 2]
    # the stage stopped after pass 1 of stage 2, with the codebook of that pass
    np.testing.assert_array_equal(t.C[:, 0], [26 / 3, 7 / 4])
    assert t.D == pytest.approx(9005 / 144, rel=1e-15)


def test_initial_alphabet_resume():
    """Starting from A_0 = the centroid (Sec. 2.2 Initialization) is the
    default run; starting from a finished stage's codebook runs that stage's
    Lloyd iteration again and then continues the splits."""
    X, _ = _random_problem(30, M=1500, L=3)
    t = oracle.lbg_train(X, 16, 0.01, 1e-3)
    t1 = oracle.lbg_train(X, 16, 0.01, 1e-3, C_init=oracle.mean(X))
    np.testing.assert_array_equal(t.C, t1.C)
    np.testing.assert_array_equal(t.trace_D, t1.trace_D)
    # uniform quantizer: resuming from the finished N/2 codebook ends at the same closed form
    M = 64
    U = np.arange(M, dtype=np.float32)[:, None]
    half = oracle.lbg_train(U, 4, 0.25, 1e-3)
    full = oracle.lbg_train(U, 8, 0.25, 1e-3, C_init=half.C)
    w = 8
    mids = np.array([(c * w + (c + 1) * w - 1) / 2.0 for c in range(8)])[::-1]
    np.testing.assert_array_equal(full.C[:, 0], mids)
    assert full.passes_per_stage() == [2, 3]


def test_multiplicative_split_values_and_closed_form():
    """Variant V1: c (1 + delta), c (1 - delta); on the uniform scalar quantizer
    over 1..2^k the children are symmetric around c, so the closed form of the
    additive split holds unchanged."""
    S = oracle.split(np.array([[2.0, -4.0]]), 0.5, multiplicative=True)
    np.testing.assert_array_equal(S, [[3.0, -6.0], [1.0, -2.0]])
    M, N = 64, 8
    X = (np.arange(M, dtype=np.float32) + 1)[:, None]
    t = oracle.lbg_train(X, N, 0.01, 1e-3, split_multiplicative=True)
    w = M // N
    mids = np.array([(c * w + (c + 1) * w - 1) / 2.0 + 1 for c in range(N)])[::-1]
    np.testing.assert_array_equal(t.C[:, 0], mids)
    assert t.passes_per_stage() == [2, 3, 3, 3]


def test_variants_in_training_zero_mean_hand_example():
    """X = {-3, -1, 1, 3} (mean 0), N = 2, delta = 0.5, worked by hand.
    Paper split (additive): children 0.5, -0.5 -> cells {1, 3}, {-3, -1}:
    D 20, 20 | 13, 4, 4, ending at C = [2, -2].
    Multiplicative split (V1): 0 (1 +- delta) = 0 twice, every row ties and
    goes to child 0, child 1 stays empty and keeps 0: D 20, 20 | 20, 20.
    V1 with re-seeding (V2): after the first update child 1 takes 0 + delta
    and child 0 becomes 0 - delta, each with 2 rows: D 20, 20 | 20, 13, 4, 4,
    ending at C = [-2, 2]."""
    X = np.array([-3, -1, 1, 3], np.float32)[:, None]
    add = oracle.lbg_train(X, 2, 0.5, 1e-3)
    np.testing.assert_array_equal(add.trace_D, [20, 20, 13, 4, 4])
    np.testing.assert_array_equal(add.C[:, 0], [2, -2])
    assert add.a.tolist() == [1, 1, 0, 0] and add.D == 4
    mult = oracle.lbg_train(X, 2, 0.5, 1e-3, split_multiplicative=True)
    np.testing.assert_array_equal(mult.trace_D, [20, 20, 20, 20])
    np.testing.assert_array_equal(mult.C[:, 0], [0, 0])
    assert mult.a.tolist() == [0, 0, 0, 0] and mult.D == 20
    both = oracle.lbg_train(X, 2, 0.5, 1e-3, split_multiplicative=True, reseed_empty=True)
    np.testing.assert_array_equal(both.trace_D, [20, 20, 20, 13, 4, 4])
    np.testing.assert_array_equal(both.C[:, 0], [-2, 2])
    assert both.a.tolist() == [0, 0, 1, 1] and both.D == 4
    assert both.passes_per_stage() == [2, 4]


def test_reseed_empty_cells_hand_example():
    """Variant V2 by hand: counts [2, 4, 0, 0] -> cell 2 takes from cell 1
    (largest): c2 = c1 + d, c1 = c1 - d, counts [2, 2, 2, 0]; cell 3 then takes
    from cell 0 (largest, lowest index): c3 = c0 + d, c0 = c0 - d."""
    C = np.array([[0.0, 1.0], [10.0, 10.0], [7.0, 7.0], [8.0, 8.0]])
    C2, cnt = oracle.reseed(C, [2, 4, 0, 0], 0.5)
    np.testing.assert_array_equal(C2, [[-0.5, 0.5], [9.5, 9.5], [10.5, 10.5], [0.5, 1.5]])
    np.testing.assert_array_equal(cnt, [1, 2, 2, 1])
    # odd count: the empty cell takes floor(5 / 2) = 2, the donor keeps 3 and so
    # is still the largest when cell 2 is re-seeded: c2 = c0' + d, c0 = c0' - d
    C = np.array([[1.0, 2.0], [9.0, 9.0], [4.0, 4.0]])
    C2, cnt = oracle.reseed(C, [5, 0, 0], 0.5)
    np.testing.assert_array_equal(C2, [[0.0, 1.0], [1.5, 2.5], [1.0, 2.0]])
    np.testing.assert_array_equal(cnt, [2, 2, 1])
    # a largest cell of one row has nothing to give: the empty cells stay as they are
    C = np.array([[1.0, 2.0], [9.0, 9.0], [4.0, 4.0]])
    C2, cnt = oracle.reseed(C, [1, 0, 1], 0.5)
    np.testing.assert_array_equal(C2, C)
    np.testing.assert_array_equal(cnt, [1, 0, 1])


def test_arguments_rejected():
    X = np.zeros((4, 2), np.float32)
    with pytest.raises(ValueError):
        oracle.lbg_train(X, 3, 0.1, 0.1)  # N not a power of 2 (Sec. 2.2 terms: powers of 2)
    with pytest.raises(ValueError):
        oracle.lbg_train(X, 4, -0.1, 0.1)
    with pytest.raises(ValueError):
        oracle.lbg_train(X, 4, 0.1, -1.0)


# ---------------------------------------------------------------- invariants
def _random_problem(seed, M=3000, L=4, N=32):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((M, L)) * rng.uniform(0.5, 3, L)).astype(np.float32)
    C = X[rng.choice(M, N, replace=False)].astype(np.float64)
    return X, C


def test_lloyd_step_invariants():
    """One pass: D equals the recomputed sum of squared distances, counts sum
    to M, mass is conserved (sum counts*c = sum x over non-empty cells), the
    new codevectors are cell means, and the next pass's D is not larger."""
    X, C = _random_problem(21)
    s = oracle.lloyd_step(X, C)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(s.D, ((Xd - C[s.a]) ** 2).sum(), rtol=1e-12)
    assert s.counts.sum() == X.shape[0]
    nz = s.counts > 0
    np.testing.assert_allclose((s.counts[nz, None] * s.C[nz]).sum(0), Xd.sum(0), rtol=1e-11,
                               atol=1e-9)
    for n in np.flatnonzero(nz)[:10]:
        np.testing.assert_allclose(s.C[n], Xd[s.a == n].mean(0), rtol=1e-13)
    s2 = oracle.lloyd_step(X, s.C)
    assert s2.D <= s.D * (1 + 1e-12)


def test_train_invariants_random():
    """Whole design on random data: codebook size doubles per stage up to N,
    D never increases within a stage, the returned D matches the returned
    (C, a), and the returned a is the nearest-codevector map of C."""
    X, _ = _random_problem(22, M=4000, L=3)
    t = oracle.lbg_train(X, 16, 0.01, 1e-3)
    sizes = []
    for n, p in zip(t.trace_n, t.trace_pass):
        if p == 0:
            sizes.append(int(n))
    assert sizes == [1, 2, 4, 8, 16]
    for n in sizes:
        Ds = t.trace_D[t.trace_n == n]
        assert np.all(np.diff(Ds) <= 1e-12 * Ds[:-1])
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(t.D, ((Xd - t.C[t.a]) ** 2).sum(), rtol=1e-12)
    a, _, _ = oracle.assign(X, t.C)
    assert np.array_equal(a, t.a)
    assert t.D == t.trace_D[-1]


# ------------------------------------------------------------------ gradient
def test_gradient_matches_central_differences():
    """D at a fixed cell table is quadratic in C and X, so FP64 central
    differences are exact up to rounding."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((40, 3)).astype(np.float32)
    C = rng.standard_normal((5, 3))
    a, _, _ = oracle.assign(X, C)
    gC, gX = oracle.grad(X, C, a)
    h = 1e-3
    for n in range(5):
        for l in range(3):
            Cp, Cm = C.copy(), C.copy()
            Cp[n, l] += h
            Cm[n, l] -= h
            fd = (oracle.distortion_fixed(X, Cp, a) - oracle.distortion_fixed(X, Cm, a)) / (2 * h)
            assert fd == pytest.approx(gC[n, l], rel=1e-7, abs=1e-8)
    # dD/dx via the same construction on a float64 copy: perturb one row
    Xd = X.astype(np.float64)
    for m in range(0, 40, 7):
        for l in range(3):
            xp, xm = Xd.copy(), Xd.copy()
            xp[m, l] += h
            xm[m, l] -= h
            fp = ((xp - C[a]) ** 2).sum()
            fm = ((xm - C[a]) ** 2).sum()
            assert (fp - fm) / (2 * h) == pytest.approx(gX[m, l], rel=1e-7, abs=1e-8)
