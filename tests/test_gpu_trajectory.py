"""lbg_train checked against the oracle at every pass (re-anchored trajectory).

The design keeps, on the device, the codebook and the cell table of every
pass (lbg_opts.trace_C / trace_assign) and records each pass's D, action and
empty cells.  oracle.trajectory.compare then runs the oracle's Lloyd step from
each pass's own FP32 codebook and checks the allocation (outside near-ties),
D, the empty-cell count, the update or split that follows, the stop decision
and the final state (Sec. 2.2 steps 1-3; Algorithm 1).  This holds at image
sizes where a whole-run comparison cannot: there a single near-tie resolved
the other way changes every later pass.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import trajectory as tj
import paper_0910_4711_gb300 as lbg
from paper_0910_4711_gb300 import synth

pytestmark = pytest.mark.gpu


def traced(X, N, precision, cap, **kw):
    Xd = torch.from_numpy(X).cuda()
    r = lbg.lbg_train(Xd, N, 0.01, 1e-3, precision=precision, trace=cap, trace_passes=cap, **kw)
    assert 0 < r.n_passes <= cap
    rep = tj.compare(X, N, 0.01, 1e-3, r.records, r.pass_C.cpu().numpy(), r.pass_assign.cpu().numpy(),
                     r.C.cpu().numpy(), r.assign.cpu().numpy(), r.D, max_passes=kw.get("max_passes", 1000))
    return r, rep


def assert_trajectory(r, rep, N):
    s = rep.summary()
    assert s["passes_checked"] == r.n_passes
    assert s["assign_rows_outside_tolerance"] == 0, s
    assert s["worst_D_rel"] <= 1e-5, s
    assert s["worst_codebook_rel"] <= 1e-4, s
    assert s["empty_cell_count_mismatches"] == 0, s
    assert s["stop_decisions_wrong"] == 0, s
    assert s["stop_decisions_vs_oracle_D_wrong"] == 0, s
    assert s["final_state_is_last_pass"], s
    # invariants of the trace: sizes double stage by stage up to N, D never rises in a stage
    sizes = [rec["stage_n"] for rec in r.records if rec["pass"] == 0]
    assert sizes == [2 ** k for k in range(len(sizes))] and sizes[-1] == N
    for a, b in zip(r.records, r.records[1:]):
        if b["pass"] > 0:
            assert b["D"] <= a["D"] * (1 + 1e-5)
    assert all(rec["ms"] > 0 for rec in r.records)
    return s


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_image_512_4x4_n256_every_pass(precision):
    """One 512x512 image, 4x4 blocks (M = 16384, L = 16), LBG to N = 256: every pass."""
    X, N = synth.workload("img512_b4_n256")
    r, rep = traced(X, N, precision, 1024)
    s = assert_trajectory(r, rep, N)
    print(precision, s)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_image_8x8_blocks_n512_every_pass(precision):
    """Two 1024x1024 images, 8x8 blocks (M = 32768, L = 64), LBG to N = 512: every pass."""
    X = synth.image_blocks([2001, 2002], 1024, 1024, 8)
    r, rep = traced(X, 512, precision, 1024)
    s = assert_trajectory(r, rep, 512)
    print(precision, s)


def test_pass_cap_and_trace_beyond_capacity():
    """A stage cut at max_passes is a legal stop (R11) and the checker agrees; passes beyond
    the trace capacity are run but not written."""
    X, N = synth.workload("img512_b4_n256")
    r, rep = traced(X[:4096], 16, "fp32", 256, max_passes=3)
    assert r.status == 1            # LBG_WARN_MAXPASS
    assert_trajectory(r, rep, 16)
    Xd = torch.from_numpy(X[:4096]).cuda()
    full = lbg.lbg_train(Xd, 16, 0.01, 1e-3, trace=256)
    part = lbg.lbg_train(Xd, 16, 0.01, 1e-3, trace=256, trace_passes=3)
    assert part.n_passes == full.n_passes > 3
    assert part.pass_C.shape[0] == 3
    assert torch.equal(part.C, full.C)


def test_trace_rejects_host_buffers():
    from paper_0910_4711_gb300 import _binding
    import ctypes
    X = torch.from_numpy(synth.blocks(synth.make_image(3, 64, 64), 4)).cuda()
    o, keep = _binding._opts(X)
    host = np.zeros((4, 4, 16), np.float32)
    o.trace_C, o.trace_cap = host.ctypes.data, 4
    C = torch.empty((4, 16), device="cuda")
    rc = _binding.lib().lbg_train(X.data_ptr(), X.shape[0], 16, 4, 0.01, 1e-3, C.data_ptr(), 0, None,
                                  None, ctypes.byref(o))
    assert rc == -1
