"""Batched ragged LBG (many independent problems advanced together) vs one
lbg_train per problem (bitwise: the batched launches run the same per-problem
arithmetic) and vs the FP64 oracle."""
import numpy as np
import pytest

import oracle
from _gpu_helpers import check_assign, check_D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbg():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    return m


def ragged_sets(seed, sizes, Ns):
    from paper_0910_4711_gb300 import synth
    parts = []
    for k, M in enumerate(sizes):
        X = synth.blocks(synth.make_image(seed + k, 512, 512), 4)
        parts.append(X[:M])
    row_off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])])
    return parts, np.concatenate(parts), row_off, list(Ns)


def test_batched_equals_single_problem_runs(lbg):
    parts, Xc, row_off, Ns = ragged_sets(40, [500, 16384, 3000, 12345, 777, 9000],
                                         [4, 256, 64, 128, 16, 32])
    r = lbg.lbg_train_batched(torch.from_numpy(Xc).cuda(), row_off, Ns)
    assert r.status == 0
    for s, (X, N) in enumerate(zip(parts, Ns)):
        single = lbg.lbg_train(torch.from_numpy(X).cuda(), N, 0.01, 1e-3)
        assert torch.equal(r.codebook(s), single.C), s
        a = r.assign[row_off[s]:row_off[s + 1]]
        assert torch.equal(a, single.assign), s
        assert r.D[s] == single.D, s


def test_batched_matches_oracle(lbg):
    parts, Xc, row_off, Ns = ragged_sets(60, [2048, 5000, 1500], [64, 128, 8])
    r = lbg.lbg_train_batched(torch.from_numpy(Xc).cuda(), row_off, Ns)
    for s, X in enumerate(parts):
        C = r.codebook(s).cpu().numpy()
        a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
        check_assign(X, C, r.assign[row_off[s]:row_off[s + 1]].cpu().numpy(), a_ref, e_ref, gap)
        check_D(r.D[s], float(e_ref.sum()))


def test_batched_host_buffers_and_single_problem(lbg):
    parts, Xc, row_off, Ns = ragged_sets(70, [3000], [32])
    rd = lbg.lbg_train_batched(torch.from_numpy(Xc).cuda(), row_off, Ns)
    rh = lbg.lbg_train_batched(Xc, row_off, Ns)
    np.testing.assert_array_equal(rd.C.cpu().numpy(), rh.C)
    assert rd.D == rh.D


def test_batched_rejects_bad_sizes(lbg):
    X = np.zeros((10, 16), np.float32)
    with pytest.raises(lbg.LBGError):
        lbg.lbg_train_batched(X, [0, 5, 10], [4, 3])       # 3 not a power of 2
    with pytest.raises(lbg.LBGError):
        lbg.lbg_train_batched(X, [0, 0, 10], [4, 4])       # empty problem


def test_tile_choice_does_not_change_results(lbg):
    """Every candidate tile of the batched assignment (rows per work item x CTAs
    per SM) gives the same bits as the fixed default and as the autotuned run."""
    parts, Xc, row_off, Ns = ragged_sets(70, [4096, 20000, 777, 9000], [64, 512, 16, 128])
    Xd = torch.from_numpy(Xc).cuda()
    ref = lbg.lbg_train_batched(Xd, row_off, Ns, autotune=False, per_phase=True)
    assert ref.tune["tile_rows"] == 128 and ref.tune["ctas_per_sm"] == 2 and not ref.tune["persistent"]
    for rows, ctas in ((128, 1), (128, 2), (64, 2), (64, 4)):
        r = lbg.lbg_train_batched(Xd, row_off, Ns, tile_rows=rows, ctas_per_sm=ctas)
        assert (r.tune["tile_rows"], r.tune["ctas_per_sm"]) == (rows, ctas)
        assert torch.equal(r.C, ref.C) and torch.equal(r.assign, ref.assign) and r.D == ref.D, (rows, ctas)
    tuned = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True)
    assert torch.equal(tuned.C, ref.C) and torch.equal(tuned.assign, ref.assign) and tuned.D == ref.D


def test_autotune_report_and_cache(lbg):
    parts, Xc, row_off, Ns = ragged_sets(90, [3000, 5000, 7000], [32, 64, 1024])
    Xd = torch.from_numpy(Xc).cuda()
    first = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True)
    t = first.tune
    if not t["from_cache"]:                  # a calibration ran in this call
        c = t["candidates"]
        assert len(c) == 4 and all(x["ms"] > 0 for x in c)
        best = min(c, key=lambda x: x["ms"])
        assert (t["tile_rows"], t["ctas_per_sm"]) == (best["tile_rows"], best["ctas_per_sm"])
    again = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True)
    assert again.tune["from_cache"] and again.tune["candidates"] == []
    assert (again.tune["tile_rows"], again.tune["ctas_per_sm"]) == (t["tile_rows"], t["ctas_per_sm"])
    assert torch.equal(again.C, first.C) and again.D == first.D


def test_persistent_pass_equals_per_phase_launches(lbg):
    """One cooperative launch per Lloyd pass of all problems (the default) gives the bits of the
    one-launch-per-phase form and of lbg_train per problem; the library's launch count shows one
    kernel per pass (plus the initial centroid's two) instead of thirteen."""
    parts, Xc, row_off, Ns = ragged_sets(110, [4096, 20000, 777, 9000, 130], [64, 512, 16, 128, 256])
    Xd = torch.from_numpy(Xc).cuda()
    phased = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True)
    l0 = lbg.launch_count()
    r = lbg.lbg_train_batched(Xd, row_off, Ns)
    launches = lbg.launch_count() - l0
    assert r.tune["persistent"] and r.tune["tile_rows"] == 64 and r.tune["ctas_per_sm"] >= 1
    assert torch.equal(r.C, phased.C) and torch.equal(r.assign, phased.assign) and r.D == phased.D
    passes = r.max_passes_run
    assert passes <= launches <= 2 * passes + 2 + 3          # batches of passes; mean, final copies
    single = lbg.lbg_train(torch.from_numpy(parts[1]).cuda(), Ns[1], 0.01, 1e-3)
    assert torch.equal(r.codebook(1), single.C) and r.D[1] == single.D


def test_persistent_pass_multiplicative_split_and_pass_cap(lbg):
    parts, Xc, row_off, Ns = ragged_sets(120, [3000, 6000], [32, 128])
    Xd = torch.from_numpy(Xc).cuda()
    for kw in ({"split_multiplicative": True}, {"max_passes": 2}):
        a = lbg.lbg_train_batched(Xd, row_off, Ns, **kw)
        b = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True, **kw)
        assert a.tune["persistent"] and not b.tune["persistent"]
        assert a.status == b.status and torch.equal(a.C, b.C) and a.D == b.D, kw


@pytest.mark.parametrize("L,real", [(5, True), (64, False), (32, True)])
def test_persistent_pass_other_dimensions(lbg, L, real):
    """One launch per pass, one launch per phase and lbg_train per problem agree bit for bit
    at an odd L (scalar loads, the any-L cell sums), at L = 64 and on real values; one problem
    has a codebook of 2 over 40,000 rows, so its cells hold hundreds of pieces (the two-level
    combine); the final states re-anchor to the oracle."""
    rng = np.random.default_rng(L)
    sizes, Ns = [40000, 3000, 777, 12000], [2, 64, 16, 256]
    if real:
        parts = [(rng.standard_normal((M, L)) * 3.0 + k).astype(np.float32) for k, M in enumerate(sizes)]
    else:
        from paper_0910_4711_gb300 import synth
        parts = [synth.blocks(synth.make_image(500 + k, 2048, 2048), 8)[:M] for k, M in enumerate(sizes)]
    row_off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])])
    Xd = torch.from_numpy(np.concatenate(parts)).cuda()
    a = lbg.lbg_train_batched(Xd, row_off, Ns)
    b = lbg.lbg_train_batched(Xd, row_off, Ns, per_phase=True)
    assert a.tune["persistent"] and not b.tune["persistent"]
    assert torch.equal(a.C, b.C) and torch.equal(a.assign, b.assign) and a.D == b.D
    A = a.assign.cpu().numpy()
    for s, X in enumerate(parts):
        single = lbg.lbg_train(torch.from_numpy(X).cuda(), Ns[s], 0.01, 1e-3)
        assert torch.equal(a.codebook(s), single.C) and a.D[s] == single.D
        C = a.codebook(s).cpu().numpy()
        a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
        check_assign(X, C, A[row_off[s]:row_off[s + 1]], a_ref, e_ref, gap)
        check_D(a.D[s], float(e_ref.sum()))


def test_small_codebook_stages_score_every_codevector(lbg):
    """Training stages of at most 64 (FP32) or 8 (BF16) codevectors score every row against
    every codevector in the FP32 direct form: such passes re-score no row, and the FP32 run
    still equals the batched pass (which keeps the tiled search) bit for bit."""
    parts, Xc, row_off, Ns = ragged_sets(70, [60000], [256])
    X = torch.from_numpy(parts[0]).cuda()
    for precision, direct in (("fp32", 64), ("bf16", 8)):
        r = lbg.lbg_train(X, 256, 0.01, 1e-3, precision=precision)
        small = [rec for rec in r.records if rec["stage_n"] <= direct]
        assert small and all(rec["n_exact"] == 0 for rec in small), precision
        if precision == "fp32":
            b = lbg.lbg_train_batched(X, row_off, Ns)
            assert torch.equal(b.codebook(0), r.C) and b.D[0] == r.D
