"""vq_encode_noalloc: the encoder for callers that cannot allocate device memory
(serving loops with a fixed memory budget, processes whose framework allocator
holds the device memory, code that may allocate only at start-up).

It is called straight through the C ABI and compared with vq_encode, the
entry point that grows a cached workspace: same nearest codevectors (outside
near-ties, the parity rule of the other tests) and the same distortion within
1e-5, on two calls in a row -- the second call must not see the first call's
leftovers in the shared fixed scratch.  This file is collected last so that a
`-x` run has already run every other test when it starts, and it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _gpu_helpers import GAP_TOL, check_D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_0910_4711_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0910_4711_gb300 as m
    L = m.lib()
    P = ctypes.c_void_p
    L.vq_encode_noalloc.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32, P, P, P]
    L.vq_encode_noalloc.restype = ctypes.c_int
    return m, L


def noalloc(L, X, C):
    idx = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    D = ctypes.c_double(-1.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.vq_encode_noalloc(X.data_ptr(), X.shape[0], X.shape[1], C.data_ptr(), C.shape[0],
                             idx.data_ptr(), ctypes.byref(D), stream)
    return rc, idx, D.value


def compare(m, L, X, C):
    rc, idx, D = noalloc(L, X, C)
    assert rc == 0, m.lib().lbg_status_string(rc)
    ref = m.vq_encode(X, C)
    a, b = idx.cpu().numpy(), ref.idx.cpu().numpy()
    diff = np.flatnonzero(a != b)
    if diff.size:   # only near-ties may differ: check them against the oracle's gap
        _, _, gap = oracle.assign(X.cpu().numpy()[diff], C.cpu().numpy().astype(np.float64))
        assert np.all(gap <= GAP_TOL)
    check_D(D, ref.D)


def test_noalloc_matches_vq_encode_twice(lib):
    m, L = lib
    from paper_0910_4711_gb300 import synth
    X1 = torch.from_numpy(synth.blocks(synth.make_image(31, 1024, 1024), 8)).cuda()
    C1 = X1[torch.randperm(X1.shape[0], generator=torch.Generator().manual_seed(1))[:4096]] + 0.25
    X2 = torch.from_numpy(synth.image_blocks(range(32, 38), 2048, 1536, 4)).cuda()  # 1,179,648 rows: two chunks
    C2 = X2[:300].clone() - 0.5
    compare(m, L, X1, C1.contiguous())     # first call: L = 64, N = 4096 (the limits' corner)
    compare(m, L, X2, C2.contiguous())     # second call: different sizes, two row chunks


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    m, L = lib
    X = torch.zeros((10, 16), device="cuda")
    rc, _, _ = noalloc(L, X, torch.zeros((4097, 16), device="cuda"))
    assert rc == -7          # LBG_ERR_UNSUPPORTED: N above the fixed scratch's limit
    Xh = np.zeros((10, 16), np.float32)
    idx = torch.empty(10, dtype=torch.int32, device="cuda")
    C = torch.zeros((4, 16), device="cuda")
    rc = L.vq_encode_noalloc(Xh.ctypes.data, 10, 16, C.data_ptr(), 4, idx.data_ptr(), None, None)
    assert rc == -1          # host arrays need staging memory: rejected
