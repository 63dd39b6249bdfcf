"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (the parity contract): assignments equal index-for-index except on
near-ties whose two best FP64 distances differ by <= 1e-5 relative (where the
GPU's choice must itself be within 1e-5 of the minimum); codebooks within 1e-4
relative (max over codevectors of the inf-norm error over max(inf-norm, 1));
total distortion within 1e-5 relative.
"""
import json
import os

import numpy as np
import pytest

import oracle
from _gpu_helpers import check_assign, check_codebook, check_D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lbg():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def image_data(seed, H, W, b):
    from paper_0910_4711_gb300 import synth
    return synth.blocks(synth.make_image(seed, H, W), b)


def random_codebook(X, N, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(X.shape[0], N, replace=X.shape[0] < N)
    C = X[idx].astype(np.float32) + rng.uniform(-0.5, 0.5, (N, X.shape[1])).astype(np.float32)
    return C


# ------------------------------------------------------------------ encode
@pytest.mark.parametrize("M,L,N", [(4096, 16, 256), (5000, 64, 300), (1000, 3, 7), (777, 1, 5),
                                   (2000, 128, 129), (333, 17, 1)])
def test_encode_matches_oracle(lbg, M, L, N):
    rng = np.random.default_rng(M + L + N)
    if L in (16, 64):
        X = image_data(M, 256, 256, int(np.sqrt(L)))[:M]
    else:
        X = (rng.standard_normal((M, L)) * 20 + 5).astype(np.float32)
    C = random_codebook(X, N, 1)
    r = lbg.vq_encode(dev(X), dev(C), decode=True)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    np.testing.assert_array_equal(host(r.Xhat), C[host(r.idx)])


def test_encode_host_buffers_match_device(lbg):
    X = image_data(7, 256, 256, 4)
    C = random_codebook(X, 64, 2)
    rd = lbg.vq_encode(dev(X), dev(C))
    rh = lbg.vq_encode(X, C)
    np.testing.assert_array_equal(host(rd.idx), rh.idx)
    assert rd.D == rh.D


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("b", [4, 8])
def test_host_buffers_many_pieces_match_device(lbg, precision, b):
    """Host X of several copy pieces (pageable numpy and pinned torch): encode and a
    Lloyd step give the bits of the device-resident calls, the assignment included
    (its copy back runs on the copy stream during the update)."""
    X = image_data(13, 2048, 2048 if b == 8 else 1024, b)[:200000]
    C = random_codebook(X, 512, 3)
    rd = lbg.vq_encode(dev(X), dev(C), precision=precision)
    sd = lbg.lbg_lloyd_step(dev(X), dev(C), precision=precision)
    for Xh in (X, torch.from_numpy(X).pin_memory()):
        rh = lbg.vq_encode(Xh, C, precision=precision)
        np.testing.assert_array_equal(host(rd.idx), host(torch.as_tensor(rh.idx)))
        assert rd.D == rh.D
        Ah = torch.empty(X.shape[0], dtype=torch.int32).pin_memory()
        sh = lbg.lbg_lloyd_step(Xh, C, assign_out=Ah, precision=precision)
        np.testing.assert_array_equal(host(sd.assign), Ah.numpy())
        np.testing.assert_array_equal(host(sd.C), host(torch.as_tensor(sh.C)))
        assert sd.D == sh.D


def test_encode_empty_input(lbg):
    r = lbg.vq_encode(dev(np.zeros((0, 16), np.float32)), dev(np.zeros((4, 16), np.float32)))
    assert r.D == 0.0 and r.idx.numel() == 0


def test_encode_rejects_nonfinite(lbg):
    X = np.zeros((300, 16), np.float32)
    X[123, 5] = np.nan
    with pytest.raises(lbg.LBGError) as ei:
        lbg.vq_encode(dev(X), dev(np.zeros((4, 16), np.float32)))
    assert ei.value.status == -3
    C = np.zeros((4, 16), np.float32)
    C[2, 0] = np.inf
    with pytest.raises(lbg.LBGError) as ei:
        lbg.vq_encode(dev(np.zeros((300, 16), np.float32)), dev(C))
    assert ei.value.status == -3


def test_exact_ties_go_to_lowest_index(lbg):
    """Duplicate codevectors: every row must take the lower index of each
    duplicated pair (exact ties are decided by the exact fallback)."""
    rng = np.random.default_rng(3)
    base = rng.integers(0, 255, (32, 16)).astype(np.float32)
    C = np.repeat(base, 2, axis=0)          # rows 2i and 2i+1 identical
    X = base[rng.integers(0, 32, 5000)] + rng.integers(-3, 4, (5000, 16)).astype(np.float32)
    r = lbg.vq_encode(dev(X), dev(C))
    a_ref, _, _ = oracle.assign(X, C.astype(np.float64))
    np.testing.assert_array_equal(host(r.idx), a_ref)
    assert np.all(host(r.idx) % 2 == 0)


# ------------------------------------------------------------------ step
@pytest.mark.parametrize("M,L,N", [(16384, 16, 256), (20000, 64, 512), (3000, 5, 64),
                                   (100, 16, 256), (4097, 32, 1000)])
def test_lloyd_step_matches_oracle(lbg, M, L, N):
    if L in (16, 64):
        X = image_data(100 + N, 512, 512, int(np.sqrt(L)))[:M]
        M = X.shape[0]
    else:
        rng = np.random.default_rng(M)
        X = (rng.standard_normal((M, L)) * 10).astype(np.float32)
    C = random_codebook(X, N, 5)
    r = lbg.lbg_lloyd_step(dev(X), dev(C))
    s = oracle.lloyd_step(X, C.astype(np.float64))
    a = host(r.assign)
    n_alt = check_assign(X, C, a, s.a, s.e, s.gap)
    check_D(r.D, s.D)
    # the update given the GPU's own cell table is pinned exactly ...
    C_upd, _ = oracle.update(X, a, C.astype(np.float64))
    check_codebook(host(r.C), C_upd)
    # ... and equals the oracle's own step when no row was exempt
    if n_alt == 0:
        check_codebook(host(r.C), s.C)


def test_lloyd_step_aliasing_and_host_buffers(lbg):
    X = image_data(11, 256, 256, 4)
    C = random_codebook(X, 128, 9)
    r1 = lbg.lbg_lloyd_step(X, C)                     # host buffers
    Cd = dev(C)
    r2 = lbg.lbg_lloyd_step(dev(X), Cd, C_out=Cd)     # in place on the device
    np.testing.assert_array_equal(r1.C, host(Cd))
    np.testing.assert_array_equal(r1.assign, host(r2.assign))
    assert r1.D == r2.D


def test_lloyd_step_empty_rows_copy_codebook(lbg):
    C = np.arange(32, dtype=np.float32).reshape(8, 4)
    r = lbg.lbg_lloyd_step(dev(np.zeros((0, 4), np.float32)), dev(C))
    np.testing.assert_array_equal(host(r.C), C)
    assert r.D == 0.0


def test_lloyd_step_is_deterministic(lbg):
    X = image_data(12, 512, 512, 4)
    C = random_codebook(X, 256, 4)
    r1 = lbg.lbg_lloyd_step(dev(X), dev(C))
    r2 = lbg.lbg_lloyd_step(dev(X), dev(C))
    assert torch.equal(r1.C, r2.C) and torch.equal(r1.assign, r2.assign) and r1.D == r2.D


# ------------------------------------------------------------------ train
@pytest.mark.parametrize("k,j", [(6, 3), (9, 4), (8, 8)])
def test_train_uniform_scalar_quantizer(lbg, k, j):
    """Closed form (see the oracle pins): midpoints of 2^(k-j)-wide cells,
    descending, D = M (w^2 - 1) / 12, 2 then 3 passes per stage."""
    M, N = 2 ** k, 2 ** j
    X = np.random.default_rng(k).permutation(M).astype(np.float32)[:, None]
    r = lbg.lbg_train(dev(X), N, delta=0.25, theta=1e-3)
    w = M // N
    mids = np.array([(c * w + (c + 1) * w - 1) / 2.0 for c in range(N)])[::-1]
    np.testing.assert_array_equal(host(r.C)[:, 0], mids)
    assert r.D == M * (w * w - 1) / 12.0
    expect = [2] + [3] * j
    if w == 1:
        expect[-1] = 2
    assert r.passes_per_stage() == expect
    assert r.status == 0


def test_train_identical_vectors(lbg):
    x = np.array([3.0, -1.5, 7.0, 0.25], np.float32)
    X = np.tile(x, (1000, 1))
    r = lbg.lbg_train(dev(X), 4, delta=0.25, theta=1e-3)
    np.testing.assert_array_equal(host(r.C), np.array([x + 0.25, x - 0.25, x, x - 0.5]))
    assert r.D == 0.0 and np.all(host(r.assign) == 2)
    assert r.passes_per_stage() == [1, 2, 1]


def test_train_stop_rule_golden(lbg):
    with open(os.path.join(GOLDEN, "stop_rule_l1.json")) as f:
        g = json.load(f)
    X = np.array(g["X"], np.float32)[:, None]
    r = lbg.lbg_train(dev(X), g["N"], g["delta"], g["theta"])
    assert [rec["stage_n"] for rec in r.records] == g["trace_n"]
    D_exact = [n / d for n, d in zip(g["trace_D_num"], g["trace_D_den"])]
    np.testing.assert_allclose([rec["D"] for rec in r.records], D_exact, rtol=1e-6)
    np.testing.assert_allclose(host(r.C), g["final_C"], rtol=1e-6)
    assert host(r.assign).tolist() == g["final_a"]


def test_train_maxpass_warns(lbg):
    X = np.array([0, 2, 2, 3, 5, 6, 15], np.float32)[:, None]
    r = lbg.lbg_train(dev(X), 2, 0.5, 0.3, max_passes=2)
    assert r.status == 1 and r.passes_per_stage() == [2, 2]


def test_train_image_blocks_matches_oracle(lbg):
    """Image-block workload at reduced size: whole-run comparison with the
    oracle when no pass has an exempt row, and in any case the final state
    re-anchored: one oracle allocation from the GPU's codebook reproduces the
    GPU's cell table and distortion."""
    X = image_data(1, 256, 256, 4)
    r = lbg.lbg_train(dev(X), 64, delta=0.01, theta=1e-3)
    C = host(r.C)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.assign), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    t = oracle.lbg_train(X, 64, 0.01, 1e-3)
    if t.near_ties() == 0:
        assert r.passes_per_stage() == t.passes_per_stage()
        check_codebook(C, t.C)
        check_D(r.D, t.D)
    sizes = [rec["stage_n"] for rec in r.records if rec["pass"] == 0]
    assert sizes == [1, 2, 4, 8, 16, 32, 64]


def test_train_resume_from_codebook(lbg):
    """Resume from an initial alphabet A_0 (Sec. 2.2): the 16-entry result of
    a first run seeds a 32-entry run; compared with the oracle run from the
    same A_0 (re-anchored like the other whole-run checks)."""
    X = image_data(2, 256, 256, 4)
    r16 = lbg.lbg_train(dev(X), 16, 0.01, 1e-3)
    res = lbg.lbg_train(dev(X), 32, 0.01, 1e-3, C_init=r16.C)
    t = oracle.lbg_train(X, 32, 0.01, 1e-3, C_init=host(r16.C).astype(np.float64))
    assert [rec["stage_n"] for rec in res.records if rec["pass"] == 0] == [16, 32]
    C = host(res.C)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(res.assign), a_ref, e_ref, gap)
    check_D(res.D, float(e_ref.sum()))
    if t.near_ties() == 0:
        assert res.passes_per_stage() == t.passes_per_stage()
        check_codebook(C, t.C)


def test_train_fewer_rows_than_codevectors(lbg):
    """M < N: most cells end empty and keep split copies c +- delta, which tie
    exactly; a dyadic delta keeps those ties exact in FP32 too, so the whole
    run must match the oracle (ties to the lowest index on both sides)."""
    rng = np.random.default_rng(4)
    X = rng.integers(0, 50, (20, 8)).astype(np.float32)
    r = lbg.lbg_train(dev(X), 64, 0.25, 1e-3)
    t = oracle.lbg_train(X, 64, 0.25, 1e-3)
    assert r.passes_per_stage() == t.passes_per_stage()
    check_codebook(host(r.C), t.C)
    check_D(r.D, t.D)
