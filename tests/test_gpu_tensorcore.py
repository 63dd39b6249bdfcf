"""Tensor-core (BF16 operands, FP32 accumulation) nearest-codevector path vs the
FP64 oracle and vs the FP32 path, through the C ABI (precision = LBG_PREC_BF16).

Same parity rules as tests/test_gpu_parity.py.  On integer image data the
BF16 path must give the oracle's assignments outside near-ties (it certifies
every row or re-scores it exactly).  On real-valued data with L <= 32 the x
rows go in two BF16 pieces and most rows are still certified; with L > 32 a
tile that is not BF16-exact sends every row to the exact fallback.
"""
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


def host(t):
    return t.detach().cpu().numpy()


def image_data(seed, H, W, b):
    from paper_0910_4711_gb300 import synth
    return synth.blocks(synth.make_image(seed, H, W), b)


def codebook_from(X, N, seed):
    rng = np.random.default_rng(seed)
    return (X[rng.choice(X.shape[0], N, replace=False)] +
            rng.uniform(-0.5, 0.5, (N, X.shape[1]))).astype(np.float32)


@pytest.mark.parametrize("H,b,N", [(256, 4, 256), (512, 8, 1000), (256, 8, 64), (512, 4, 4096),
                                   (128, 4, 7)])
def test_encode_bf16_matches_oracle(lbg, H, b, N):
    X = image_data(H + N, H, H, b)
    X = X[: X.shape[0] - 37]                      # ragged tail of the 512-row tiles
    C = codebook_from(X, N, 1)
    r = lbg.vq_encode(dev(X), dev(C), precision="bf16")
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    assert r.n_exact < 0.05 * X.shape[0]          # integer data: almost every row certified


def test_encode_bf16_equals_fp32(lbg):
    X = image_data(5, 512, 512, 8)
    C = codebook_from(X, 512, 2)
    r16 = lbg.vq_encode(dev(X), dev(C), precision="bf16")
    r32 = lbg.vq_encode(dev(X), dev(C), precision="fp32")
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    diff = host(r16.idx) != host(r32.idx)
    assert np.all(gap[diff] <= 1e-5)
    check_D(r16.D, r32.D)


def test_bf16_non_integer_data_falls_back_exactly(lbg):
    """L = 64 has no second x piece: x~ not exact in BF16 sends every row to the
    exact fallback."""
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((3000, 64)) * 3.3).astype(np.float32)
    C = codebook_from(X, 100, 3)
    r = lbg.vq_encode(dev(X), dev(C), precision="bf16")
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
    assert r.n_exact == X.shape[0]


@pytest.mark.parametrize("M,N,L", [(20000, 1024, 32), (30001, 512, 16), (4099, 129, 5), (5000, 4096, 24)])
@pytest.mark.parametrize("offset", [0, 1])
def test_split_form_certifies_non_integer_data(lbg, M, N, L, offset):
    """L <= 32: x~ = x_hi + x_lo + rem in two BF16 pieces; rows of real-valued data are
    certified by the tensor-core pass (the split terms in the certificate) instead of all
    falling back.  offset = 1 starts X 4 bytes past a 16-byte boundary (the per-tile
    kernel); both kernels give the same cells."""
    rng = np.random.default_rng(M + N + L)
    X = (rng.standard_normal((M, L)) * 3.3 + 0.7).astype(np.float32)
    C = (X[rng.choice(M, N, replace=False)] + rng.normal(0, 0.05, (N, L))).astype(np.float32)
    if offset:
        buf = torch.empty(M * L + 1, dtype=torch.float32, device="cuda")
        Xd = buf[1:].view(M, L)
        Xd.copy_(torch.from_numpy(X))
        assert Xd.data_ptr() % 16 == 4
    else:
        Xd = dev(X)
    r = lbg.vq_encode(Xd, dev(C), precision="bf16")
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    assert r.n_exact < 0.05 * M, r.n_exact
    if offset:
        # same cells; e(m) is the FP32 direct form summed in another order (scalar
        # loads instead of the aligned path's float4 butterfly)
        al = lbg.vq_encode(dev(X), dev(C), precision="bf16")
        assert torch.equal(al.idx, r.idx)
        check_D(al.D, r.D)


def test_split_form_gmm_train_every_pass(lbg):
    """LBG in BF16 on mixture data (L = 32, not integer), checked pass by pass."""
    from paper_0910_4711_gb300 import synth
    from oracle import trajectory as tj
    X, _, _ = synth.gmm(6, 20000, 32, 64, 0.1)
    r = lbg.lbg_train(dev(X), 64, 0.01, 1e-3, precision="bf16", trace=512, trace_passes=512)
    rep = tj.compare(X, 64, 0.01, 1e-3, r.records, host(r.pass_C), host(r.pass_assign),
                     host(r.C), host(r.assign), r.D)
    s = rep.summary()
    assert s["assign_rows_outside_tolerance"] == 0 and s["worst_D_rel"] <= 1e-5, s
    assert s["worst_codebook_rel"] <= 1e-4 and s["stop_decisions_wrong"] == 0, s
    assert s["final_state_is_last_pass"], s
    assert sum(rec["n_exact"] for rec in r.records) < 0.05 * X.shape[0] * len(r.records)


@pytest.mark.parametrize("M,N,L", [(64, 4096, 48), (20000, 1024, 64), (3001, 512, 64), (33, 129, 37)])
def test_exact_fallback_spread_over_ctas(lbg, M, N, L):
    """Every row re-scored exactly (L > 32 and data not exact in BF16), at sizes where a
    group of 32 flagged rows is cut across many CTAs (its per-CTA minima merged), across
    two, or held whole by one, with a ragged last group and chunk.  A codebook that
    repeats its first half must give the first half's result bit for bit: equal FP32
    distances in different CTAs keep the lowest index."""
    rng = np.random.default_rng(M + N + L)
    X = (rng.standard_normal((M, L)) * 3.3).astype(np.float32)
    C = (rng.standard_normal((N, L)) * 3.3).astype(np.float32)
    r = lbg.vq_encode(dev(X), dev(C), precision="bf16")
    assert r.n_exact == M
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    H = C[: N // 2]
    half = lbg.vq_encode(dev(X), dev(H), precision="bf16")
    dup = lbg.vq_encode(dev(X), dev(np.concatenate([H, H])), precision="bf16")
    assert np.array_equal(host(dup.idx), host(half.idx)) and dup.D == half.D


@pytest.mark.parametrize("L,N,real", [(16, 1500, False), (64, 700, False), (32, 1024, True), (48, 333, True)])
def test_group_sizes_give_the_same_cells(lbg, L, N, real):
    """Every epilogue group size (2, 4, 8 codevectors; forced by tc_group) gives the
    oracle's cells, the same ones; a lloyd step and a training run too."""
    rng = np.random.default_rng(L * N)
    if real:
        X = (rng.standard_normal((9000, L)) * 2.0).astype(np.float32)
        C = (X[rng.choice(9000, N, replace=False)] + rng.normal(0, 0.1, (N, L))).astype(np.float32)
    else:
        X = image_data(L + N, 512, 512, int(round(L ** 0.5)))[:9000]
        C = codebook_from(X, N, 5)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    first = None
    for g in (2, 4, 8):
        r = lbg.vq_encode(dev(X), dev(C), precision="bf16", tc_group=g)
        check_assign(X, C, host(r.idx), a_ref, e_ref, gap)
        check_D(r.D, float(e_ref.sum()))
        s = lbg.lbg_lloyd_step(dev(X), dev(C), precision="bf16", tc_group=g)
        assert torch.equal(s.assign, r.idx)
        if first is None:
            first = (host(r.idx), host(s.C))
        else:
            assert np.array_equal(host(r.idx), first[0])
            check_codebook(host(s.C), first[1])
    t = [lbg.lbg_train(dev(X), 64, 0.01, 1e-3, precision="bf16", tc_group=g) for g in (2, 8)]
    assert torch.equal(t[0].assign, t[1].assign) and t[0].records == [
        dict(r, n_exact=t[0].records[i]["n_exact"], ms=t[0].records[i]["ms"], D=t[0].records[i]["D"])
        for i, r in enumerate(t[1].records)]
    check_D(t[0].D, t[1].D)


def test_bf16_rejects_large_dimension(lbg):
    X = np.zeros((10, 128), np.float32)
    with pytest.raises(lbg.LBGError) as ei:
        lbg.vq_encode(dev(X), dev(X[:2]), precision="bf16")
    assert ei.value.status == -7


def test_lloyd_step_bf16_matches_oracle(lbg):
    X = image_data(77, 512, 512, 8)
    C = codebook_from(X, 512, 4)
    r = lbg.lbg_lloyd_step(dev(X), dev(C), precision="bf16")
    s = oracle.lloyd_step(X, C.astype(np.float64))
    a = host(r.assign)
    check_assign(X, C, a, s.a, s.e, s.gap)
    check_D(r.D, s.D)
    C_upd, _ = oracle.update(X, a, C.astype(np.float64))
    check_codebook(host(r.C), C_upd)


def test_train_bf16_matches_oracle(lbg):
    X = image_data(1, 256, 256, 4)
    r = lbg.lbg_train(dev(X), 64, delta=0.01, theta=1e-3, precision="bf16")
    C = host(r.C)
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(r.assign), a_ref, e_ref, gap)
    check_D(r.D, float(e_ref.sum()))
    t = oracle.lbg_train(X, 64, 0.01, 1e-3)
    if t.near_ties() == 0:
        assert r.passes_per_stage() == t.passes_per_stage()
        check_codebook(C, t.C)
