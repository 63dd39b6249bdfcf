"""vq_encode_noalloc: the encoder for callers that cannot allocate device memory
(serving loops with a fixed memory budget, processes whose framework allocator
holds the device memory, code that may allocate only at start-up).

It is called straight through the C ABI and checked against the FP64 oracle
(nearest codevector index for index outside near-ties, distortion within
1e-5) and against vq_encode, the entry point that grows a cached workspace,
on two calls in a row -- the second call must not see the first call's
leftovers in the shared fixed scratch -- and at the largest dimension and
codebook size its fixed scratch is sized for (L = 128, N = 4096).  A call on a
fresh size must leave the device's free memory unchanged.  This file is
collected last so that a `-x` run has already run every other test when it
starts, and it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _gpu_helpers import GAP_TOL, check_assign, check_D

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


def noalloc(L, X, C, idx=None):
    if idx is None:
        idx = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    D = ctypes.c_double(-1.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.vq_encode_noalloc(X.data_ptr(), X.shape[0], X.shape[1], C.data_ptr(), C.shape[0],
                             idx.data_ptr(), ctypes.byref(D), stream)
    return rc, idx, D.value


def compare(m, L, X, C):
    rc, idx, D = noalloc(L, X, C)
    assert rc == 0, m.lib().lbg_status_string(rc)
    Xn, Cn = X.cpu().numpy(), C.cpu().numpy()
    a_ref, e_ref, gap = oracle.assign(Xn, Cn.astype(np.float64))
    a = idx.cpu().numpy()
    check_assign(Xn, Cn, a, a_ref, e_ref, gap)
    check_D(D, float(e_ref.sum()))
    ref = m.vq_encode(X, C)            # the workspace encoder: same rule, same D
    diff = np.flatnonzero(a != ref.idx.cpu().numpy())
    assert np.all(gap[diff] <= GAP_TOL)
    check_D(D, ref.D)


def test_noalloc_matches_oracle_twice(lib):
    m, L = lib
    from paper_0910_4711_gb300 import synth
    X1 = torch.from_numpy(synth.blocks(synth.make_image(31, 1024, 1024), 8)).cuda()
    C1 = X1[torch.randperm(X1.shape[0], generator=torch.Generator().manual_seed(1))[:4096]] + 0.25
    X2 = torch.from_numpy(synth.image_blocks(range(32, 38), 2048, 1536, 4)).cuda()  # 1,179,648 rows: two chunks
    C2 = X2[:300].clone() - 0.5
    compare(m, L, X1, C1.contiguous())     # first call: L = 64, N = 4096
    compare(m, L, X2, C2.contiguous())     # second call: different sizes, two row chunks


def test_noalloc_largest_dimension(lib):
    """L = 128 and N = 4096, the corner of the fixed scratch's limits (the padded dimension
    sets the layout of the prepared codebook), on a few thousand rows."""
    m, L = lib
    g = torch.Generator().manual_seed(7)
    X = torch.randint(0, 256, (3000, 128), generator=g).float().cuda()
    C = (X[torch.randperm(3000, generator=g)[:2048]].repeat(2, 1)
         + torch.randn((4096, 128), generator=g).cuda()).contiguous()
    compare(m, L, X, C)


def test_noalloc_allocates_no_device_memory(lib):
    m, L = lib
    g = torch.Generator().manual_seed(9)
    X = torch.rand((50000, 32), generator=g).cuda()
    C = torch.rand((1000, 32), generator=g).cuda()
    idx = torch.empty(50000, dtype=torch.int32, device="cuda")
    assert noalloc(L, X[:20000], C[:500], idx)[0] == 0   # first call: loads the kernels it uses
    m.release_workspace()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc, _, _ = noalloc(L, X, C, idx)                      # a size not seen before
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.cuda.mem_get_info()[0] == free0


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
