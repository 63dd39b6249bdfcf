"""Failure paths and corners of the C ABI on the GPU, in the forms that fault,
trap or hang nothing:

* a bounded wait that runs out: the FP32 nearest-codevector kernel's test hook
  makes every CTA's first wait give up at once; the CTAs drain the copies they
  issued, the call reports LBG_ERR_TIMEOUT, and the next default call is bit
  for bit a clean run's;
* a refused allocation: a workspace cap below what a call needs makes the
  allocation fail as cudaMalloc refusing would (LBG_ERR_NOMEM, cached
  workspace released); lifting the cap, the library recovers;
* the largest codebook the ABI accepts (N = 8192) and an X that is not
  16-byte aligned, in both precisions, against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0910_4711_gb300 as lbg
from paper_0910_4711_gb300 import synth
from _gpu_helpers import check_assign, check_codebook, check_D

pytestmark = pytest.mark.gpu


def data(seed, H, W, b):
    return synth.blocks(synth.make_image(seed, H, W), b)


def clean_step(Xd, Cd):
    r = lbg.lbg_lloyd_step(Xd, Cd)
    torch.cuda.synchronize()
    return r.C.clone(), r.assign.clone(), r.D


def test_forced_timeout_then_clean_run():
    X = data(41, 256, 320, 4)                                    # M = 5120, L = 16
    Xd = torch.from_numpy(X).cuda()
    Cd = Xd[::17][:300].contiguous() + 0.5
    C0, A0, D0 = clean_step(Xd, Cd)
    for call in (lambda: lbg.lbg_lloyd_step(Xd, Cd, test_expire_wait=True),
                 lambda: lbg.vq_encode(Xd, Cd, test_expire_wait=True)):
        with pytest.raises(lbg.LBGError) as ei:
            call()
        assert ei.value.status == -6                              # LBG_ERR_TIMEOUT
        C1, A1, D1 = clean_step(Xd, Cd)                           # default call, replayed graph
        assert torch.equal(C1, C0) and torch.equal(A1, A0) and D1 == D0
    enc = lbg.vq_encode(Xd, Cd)
    assert torch.equal(enc.idx, A0) and enc.D == D0
    # the hook is ignored by the tensor-core form
    t = lbg.lbg_lloyd_step(Xd, Cd, precision="bf16", test_expire_wait=True)
    assert t.status == 0


def test_workspace_cap_refuses_then_recovers():
    X = data(42, 512, 512, 4)                                    # M = 16384
    Xd = torch.from_numpy(X).cuda()
    Cd = Xd[::61][:256].contiguous()
    C0, A0, D0 = clean_step(Xd, Cd)
    try:
        lbg.set_workspace_limit(4096)                             # far below any call's scratch
        for call in (lambda: lbg.lbg_lloyd_step(Xd, Cd), lambda: lbg.vq_encode(Xd, Cd),
                     lambda: lbg.lbg_train(Xd, 16)):
            with pytest.raises(lbg.LBGError) as ei:
                call()
            assert ei.value.status == -5                          # LBG_ERR_NOMEM
    finally:
        lbg.set_workspace_limit(0)
    C1, A1, D1 = clean_step(Xd, Cd)
    assert torch.equal(C1, C0) and torch.equal(A1, A0) and D1 == D0


def parity(X, C, r_assign, r_D, r_C=None):
    a, e, g = oracle.assign(X, C.astype(np.float64))
    check_assign(X, C, r_assign, a, e, g)
    check_D(r_D, float(e.sum()))
    if r_C is not None:
        want, _ = oracle.update(X, np.asarray(r_assign), C.astype(np.float64))
        check_codebook(r_C, want)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_largest_codebook_8192(precision):
    X = data(43, 512, 640, 4)                                    # M = 20480, L = 16
    rng = np.random.default_rng(43)
    C = (X[rng.choice(X.shape[0], 8192, replace=False)] + rng.integers(-2, 3, (8192, 16))).astype(np.float32)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    s = lbg.lbg_lloyd_step(Xd, Cd, precision=precision)
    parity(X, C, s.assign.cpu().numpy(), s.D, s.C.cpu().numpy())
    e = lbg.vq_encode(Xd, Cd, precision=precision)
    parity(X, C, e.idx.cpu().numpy(), e.D)


def test_train_to_8192_every_pass():
    """LBG to the largest codebook (M = 16384 < N for the last stage: empty cells keep their
    codevector), checked pass by pass."""
    from oracle import trajectory as tj
    X = data(44, 512, 512, 4)
    Xd = torch.from_numpy(X).cuda()
    r = lbg.lbg_train(Xd, 8192, 0.01, 1e-3, trace=1024, trace_passes=1024)
    rep = tj.compare(X, 8192, 0.01, 1e-3, r.records, r.pass_C.cpu().numpy(), r.pass_assign.cpu().numpy(),
                     r.C.cpu().numpy(), r.assign.cpu().numpy(), r.D)
    s = rep.summary()
    assert s["assign_rows_outside_tolerance"] == 0 and s["worst_D_rel"] <= 1e-5, s
    assert s["worst_codebook_rel"] <= 1e-4 and s["stop_decisions_wrong"] == 0, s
    assert s["empty_cell_count_mismatches"] == 0 and s["final_state_is_last_pass"], s
    assert r.records[-1]["stage_n"] == 8192 and r.records[-1]["n_empty"] > 0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("L_b", [(16, 4), (64, 8)])
def test_unaligned_x(precision, L_b):
    """X starting 4 bytes past a 16-byte boundary (L a multiple of 4): the tensor-core
    launcher takes its per-tile kernel, the FP32 kernels read X with scalar loads."""
    L, b = L_b
    X = data(45, 256, 512, b)
    M = X.shape[0]
    buf = torch.empty(M * L + 1, dtype=torch.float32, device="cuda")
    Xu = buf[1:].view(M, L)
    Xu.copy_(torch.from_numpy(X))
    assert Xu.data_ptr() % 16 == 4
    C = X[::7][:200].copy() + 0.25
    Cd = torch.from_numpy(C).cuda()
    s = lbg.lbg_lloyd_step(Xu, Cd, precision=precision)
    parity(X, C, s.assign.cpu().numpy(), s.D, s.C.cpu().numpy())
    e = lbg.vq_encode(Xu, Cd, precision=precision)
    parity(X, C, e.idx.cpu().numpy(), e.D)
    aligned = lbg.vq_encode(torch.from_numpy(X).cuda(), Cd, precision=precision)
    assert torch.equal(aligned.idx, e.idx)
