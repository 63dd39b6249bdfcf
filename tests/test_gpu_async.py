"""Replayed and asynchronous forms of lbg_lloyd_step / vq_encode.

A call's device sequence is recorded into a CUDA graph under its key (device
pointers, sizes, options) and replayed by later calls; with a device report
buffer (lbg_opts.result_dev) the call only enqueues.  Every form must give
the results of the directly launched call (phase_ms set) bit for bit, and
those are the oracle-checked results of the parity tests; the oracle is
re-checked here on the replayed form.
"""
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


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def workload(seed, M, b, N):
    from paper_0910_4711_gb300 import synth
    X = synth.blocks(synth.make_image(seed, 512, 512), b)[:M]
    rng = np.random.default_rng(seed)
    C = X[rng.choice(X.shape[0], N, replace=False)] + rng.uniform(-0.5, 0.5, (N, X.shape[1]))
    return np.ascontiguousarray(X, np.float32), np.ascontiguousarray(C, np.float32)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_step_replay_and_async_match_direct(lbg, precision):
    X, C = workload(11, 16384, 8, 256)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    Co, A = torch.empty_like(Cd), torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    direct = lbg.lbg_lloyd_step(Xd, Cd, phase_ms=True, precision=precision)
    s = oracle.lloyd_step(X, C.astype(np.float64))
    check_assign(X, C, host(direct.assign), s.a, s.e, s.gap)
    check_D(direct.D, s.D)
    for _ in range(3):   # the first call records the graph, the others replay it
        r = lbg.lbg_lloyd_step(Xd, Cd, C_out=Co, assign_out=A, precision=precision)
        assert np.array_equal(host(r.assign), host(direct.assign))
        assert np.array_equal(host(r.C), host(direct.C))
        assert r.D == direct.D and r.n_exact == direct.n_exact
    buf = lbg.step_result_buffer()
    Co.zero_()
    A.fill_(-1)
    for _ in range(3):
        r = lbg.lbg_lloyd_step(Xd, Cd, C_out=Co, assign_out=A, precision=precision, result_out=buf)
        assert r.result is buf and np.isnan(r.D) and r.n_exact == -1
    D, n_exact, status = lbg.read_step_result(buf)
    assert status == 0 and D == direct.D and n_exact == direct.n_exact
    assert np.array_equal(host(A), host(direct.assign))
    assert np.array_equal(host(Co), host(direct.C))


def test_async_steps_chain_on_one_stream(lbg):
    """K enqueued passes, each from the previous one's codebook, reproduce K
    synchronous passes; no host wait happens between them."""
    X, C = workload(12, 8192, 4, 64)
    Xd = torch.from_numpy(X).cuda()
    C0 = torch.from_numpy(C).cuda()
    ref = C0.clone()
    Ds = []
    for _ in range(4):
        r = lbg.lbg_lloyd_step(Xd, ref)
        ref = r.C
        Ds.append(r.D)
    bufs = [lbg.step_result_buffer() for _ in range(4)]
    cur, nxt = C0.clone(), torch.empty_like(C0)
    for k in range(4):
        lbg.lbg_lloyd_step(Xd, cur, C_out=nxt, result_out=bufs[k])
        cur, nxt = nxt, cur
    assert np.array_equal(host(cur), host(ref))
    assert [lbg.read_step_result(b)[0] for b in bufs] == Ds


def test_async_then_other_stream_waits(lbg):
    """A call on another stream waits for an enqueued pass before reusing the
    shared scratch."""
    X, C = workload(13, 16384, 8, 512)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    want = lbg.lbg_lloyd_step(Xd, Cd, precision="bf16")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    buf = lbg.step_result_buffer()
    Co = torch.empty_like(Cd)
    torch.cuda.synchronize()
    lbg.lbg_lloyd_step(Xd, Cd, C_out=Co, precision="bf16", stream=s1.cuda_stream, result_out=buf)
    r2 = lbg.lbg_lloyd_step(Xd, Cd, precision="bf16", stream=s2.cuda_stream)
    torch.cuda.synchronize()
    assert lbg.read_step_result(buf)[0] == want.D == r2.D
    assert np.array_equal(host(Co), host(want.C)) and np.array_equal(host(r2.C), host(want.C))


def test_encode_replay_and_async(lbg):
    X, C = workload(14, 20000, 4, 1024)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    direct = lbg.vq_encode(Xd, Cd, decode=True, phase_ms=True, precision="bf16")
    a_ref, e_ref, gap = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, host(direct.idx), a_ref, e_ref, gap)
    I = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    for _ in range(2):
        r = lbg.vq_encode(Xd, Cd, decode=True, idx_out=I, precision="bf16")
        assert np.array_equal(host(r.idx), host(direct.idx)) and r.D == direct.D
        assert np.array_equal(host(r.Xhat), host(direct.Xhat))
    buf = lbg.step_result_buffer()
    I.fill_(-1)
    lbg.vq_encode(Xd, Cd, idx_out=I, precision="bf16", result_out=buf)
    D, n_exact, status = lbg.read_step_result(buf)
    assert status == 0 and D == direct.D and n_exact == direct.n_exact
    assert np.array_equal(host(I), host(direct.idx))


def test_async_rejects_host_arrays_and_handles_empty(lbg):
    X, C = workload(15, 1024, 4, 16)
    buf = lbg.step_result_buffer()
    with pytest.raises(lbg.LBGError) as ei:
        lbg.lbg_lloyd_step(X, C, result_out=buf)          # host X and C
    assert ei.value.status == -1
    Cd = torch.from_numpy(C).cuda()
    buf.fill_(7)
    r = lbg.lbg_lloyd_step(torch.empty((0, 16), device="cuda"), Cd, result_out=buf)
    assert lbg.read_step_result(buf) == (0.0, 0, 0)
    assert np.array_equal(host(r.C), C)


def test_graph_cache_eviction_keeps_results(lbg):
    """More distinct keys than the cache holds: old graphs are evicted and
    re-recorded, results unchanged."""
    X, C = workload(16, 4096, 4, 32)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    want = lbg.lbg_lloyd_step(Xd, Cd, phase_ms=True)
    outs = [torch.empty_like(Cd) for _ in range(40)]
    for rep in range(2):
        for Co in outs:
            r = lbg.lbg_lloyd_step(Xd, Cd, C_out=Co)
            assert r.D == want.D
    for Co in outs:
        assert np.array_equal(host(Co), host(want.C))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_host_input_pieces_match_device_input(lbg, precision):
    """A host-resident X is copied and searched piece by piece (one search wave per
    piece); the step and the encode must give the device-input call's results bit
    for bit, for a size with several pieces and a ragged last one."""
    from paper_0910_4711_gb300 import synth
    X = np.ascontiguousarray(synth.blocks(synth.make_image(17, 1024, 2048), 4)[: 100000 - 77], np.float32)
    rng = np.random.default_rng(17)
    C = np.ascontiguousarray(X[rng.choice(X.shape[0], 512, replace=False)] + rng.uniform(-0.5, 0.5, (512, 16)),
                             np.float32)
    assert X.shape[0] > 2 * 152 * 256      # three pieces, the last one ragged
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    dev_step = lbg.lbg_lloyd_step(Xd, Cd, precision=precision)
    host_step = lbg.lbg_lloyd_step(torch.from_numpy(X).pin_memory(), torch.from_numpy(C), precision=precision)
    assert np.array_equal(host(host_step.assign), host(dev_step.assign))
    assert np.array_equal(host(host_step.C), host(dev_step.C))
    assert host_step.D == dev_step.D and host_step.n_exact == dev_step.n_exact
    dev_enc = lbg.vq_encode(Xd, Cd, precision=precision)
    host_enc = lbg.vq_encode(X, C, precision=precision)            # pageable host memory
    assert np.array_equal(host(host_enc.idx), host(dev_enc.idx)) and host_enc.D == dev_enc.D
