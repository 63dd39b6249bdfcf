"""ctypes binding of ``_lib/liblbgvq.so`` (the C ABI of ``include/lbgvq.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; CUDA tensors are passed as device pointers on torch's current
stream, CPU tensors and numpy arrays as host pointers (the library copies
them to the device and back inside the call).  If the library is missing or
cannot be loaded, every call raises ``RuntimeError``: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbgvq.so")

LBG_OK, LBG_WARN_MAXPASS = 0, 1
STATUS = {0: "LBG_OK", 1: "LBG_WARN_MAXPASS", -1: "LBG_ERR_ARG", -2: "LBG_ERR_NOT_POW2",
          -3: "LBG_ERR_NONFINITE", -4: "LBG_ERR_CUDA", -5: "LBG_ERR_NOMEM", -6: "LBG_ERR_TIMEOUT",
          -7: "LBG_ERR_UNSUPPORTED"}
PHASES = ("prep", "assign", "exact", "update", "total")
ACTIONS = ("update", "split", "finish")
EXPORTS = ("lbg_opts_init", "lbg_train", "lbg_lloyd_step", "vq_encode", "lbg_status_string",
           "lbg_release_workspace", "lbg_version", "lbg_distortion_backward", "lbg_train_batched",
           "vq_encode_noalloc", "lbg_set_workspace_limit", "lbg_launch_count",
           "lbg_measure_fp32_peak")


class LBGError(RuntimeError):
    def __init__(self, status: int, text: str):
        super().__init__(f"{STATUS.get(status, status)}: {text}")
        self.status = status


class PassRecord(ctypes.Structure):
    _fields_ = [("stage_n", ctypes.c_int32), ("pass_", ctypes.c_int32), ("action", ctypes.c_int32),
                ("n_exact", ctypes.c_int32), ("D", ctypes.c_double), ("n_empty", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class TuneReport(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("cand_tile_rows", ctypes.c_int32 * 8), ("cand_ctas_per_sm", ctypes.c_int32 * 8),
                ("cand_ms", ctypes.c_float * 8), ("persistent", ctypes.c_int32)]

    def as_dict(self):
        n = self.n_candidates
        return {"tile_rows": self.tile_rows, "ctas_per_sm": self.ctas_per_sm,
                "from_cache": bool(self.from_cache), "persistent": bool(self.persistent),
                "candidates": [{"tile_rows": self.cand_tile_rows[k],
                                "ctas_per_sm": self.cand_ctas_per_sm[k], "ms": self.cand_ms[k]}
                               for k in range(n)]}


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("records", ctypes.POINTER(PassRecord)),
                ("max_records", ctypes.c_int32), ("n_records", ctypes.POINTER(ctypes.c_int32)),
                ("phase_ms", ctypes.POINTER(ctypes.c_float)),
                ("n_exact", ctypes.POINTER(ctypes.c_int32)),
                ("split_multiplicative", ctypes.c_int32), ("reseed_empty", ctypes.c_int32),
                ("delta_reseed", ctypes.c_double), ("autotune", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tune_report", ctypes.POINTER(TuneReport)),
                ("result_dev", ctypes.c_void_p),
                ("trace_C", ctypes.c_void_p), ("trace_assign", ctypes.c_void_p),
                ("trace_cap", ctypes.c_int32), ("test_expire_wait", ctypes.c_int32),
                ("batched_per_phase", ctypes.c_int32), ("grad_scale_dev", ctypes.c_void_p),
                ("tc_group", ctypes.c_int32)]


STEP_RESULT_BYTES = 16   # lbg_step_result: double D, int32 n_exact, int32 status


def step_result_buffer(device=None):
    """A zeroed device buffer for an asynchronous step / encode report
    (lbg_step_result, 16 bytes)."""
    import torch
    return torch.zeros(STEP_RESULT_BYTES, dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def read_step_result(buf):
    """(D, n_exact, status) of a report written by an asynchronous call (waits
    for the stream that wrote it, through the device-to-host copy)."""
    raw = np.ascontiguousarray(buf.detach().cpu().numpy()).view(np.uint8)[:STEP_RESULT_BYTES]
    D = float(raw[:8].view(np.float64)[0])
    n_exact, status = (int(v) for v in raw[8:16].view(np.int32))
    return D, n_exact, status


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (raises RuntimeError if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblbgvq is not built ({LIB_PATH} missing); run "
                               "paper_0910_4711_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.lbg_opts_init.argtypes = [ctypes.POINTER(Opts)]
        L.lbg_opts_init.restype = None
        L.lbg_train.argtypes = [P, i64, i32, i32, f64, f64, P, i32, P, P, ctypes.POINTER(Opts)]
        L.lbg_train.restype = ctypes.c_int
        L.lbg_lloyd_step.argtypes = [P, i64, i32, i32, P, P, P, P, ctypes.POINTER(Opts)]
        L.lbg_lloyd_step.restype = ctypes.c_int
        L.vq_encode.argtypes = [P, i64, i32, P, i32, P, P, P, ctypes.POINTER(Opts)]
        L.vq_encode.restype = ctypes.c_int
        L.lbg_distortion_backward.argtypes = [P, i64, i32, P, i32, P, ctypes.c_float, P, P, P,
                                              ctypes.POINTER(Opts)]
        L.lbg_distortion_backward.restype = ctypes.c_int
        L.lbg_train_batched.argtypes = [i32, P, P, i32, P, f64, f64, P, P, P, ctypes.POINTER(Opts)]
        L.lbg_train_batched.restype = ctypes.c_int
        L.lbg_status_string.argtypes = [ctypes.c_int]
        L.lbg_status_string.restype = ctypes.c_char_p
        L.lbg_release_workspace.argtypes = []
        L.lbg_release_workspace.restype = ctypes.c_int
        L.lbg_version.argtypes = []
        L.lbg_version.restype = ctypes.c_int32
        L.vq_encode_noalloc.argtypes = [P, i64, i32, P, i32, P, P, P]
        L.vq_encode_noalloc.restype = ctypes.c_int
        L.lbg_set_workspace_limit.argtypes = [ctypes.c_size_t]
        L.lbg_set_workspace_limit.restype = ctypes.c_int
        L.lbg_launch_count.argtypes = []
        L.lbg_launch_count.restype = ctypes.c_int64
        L.lbg_measure_fp32_peak.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int32)]
        L.lbg_measure_fp32_peak.restype = ctypes.c_int
        _lib = L
        return L


def _check(rc: int) -> int:
    if rc < 0:
        raise LBGError(rc, lib().lbg_status_string(rc).decode())
    return rc


# ------------------------------------------------------------ marshalling
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _prep(a, dtype: str, name: str):
    """Return (array object kept alive, pointer, is_cuda)."""
    if a is None:
        return None, None, False
    if _is_torch(a):
        import torch
        want = {"f32": torch.float32, "i32": torch.int32}[dtype]
        if a.dtype != want:
            raise TypeError(f"{name} must be {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return a, a.data_ptr(), a.is_cuda
    want = {"f32": np.float32, "i32": np.int32}[dtype]
    if not isinstance(a, np.ndarray) or a.dtype != want or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy {want.__name__} array or torch tensor")
    return a, a.ctypes.data, False


def _empty_like_src(src, shape, dtype: str):
    if _is_torch(src):
        import torch
        t = {"f32": torch.float32, "i32": torch.int32}[dtype]
        return torch.empty(shape, dtype=t, device=src.device)
    return np.empty(shape, dtype={"f32": np.float32, "i32": np.int32}[dtype])


PRECISION = {"fp32": 0, "bf16": 1}


def _opts(cuda_ref, max_passes=1000, records=0, phase=False, stream=None, precision="fp32",
          split_multiplicative=False, reseed_empty=False, delta_reseed=0.0, result=None,
          test_expire_wait=False, tc_group=0):
    o = Opts()
    lib().lbg_opts_init(ctypes.byref(o))
    o.max_passes = int(max_passes)
    o.test_expire_wait = int(bool(test_expire_wait))
    o.tc_group = int(tc_group)
    o.split_multiplicative = int(bool(split_multiplicative))
    o.reseed_empty = int(bool(reseed_empty))
    o.delta_reseed = float(delta_reseed)
    if precision not in PRECISION:
        raise ValueError(f"precision must be one of {sorted(PRECISION)}")
    o.precision = PRECISION[precision]
    keep = {}
    if stream is not None:
        o.stream = ctypes.c_void_p(int(stream))
    elif cuda_ref is not None:
        import torch
        o.stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_ref.device).cuda_stream)
    if records:
        keep["rec"] = (PassRecord * records)()
        keep["nrec"] = ctypes.c_int32(0)
        o.records = ctypes.cast(keep["rec"], ctypes.POINTER(PassRecord))
        o.max_records = records
        o.n_records = ctypes.pointer(keep["nrec"])
    if phase:
        keep["ph"] = (ctypes.c_float * 5)()
        o.phase_ms = ctypes.cast(keep["ph"], ctypes.POINTER(ctypes.c_float))
    keep["nex"] = ctypes.c_int32(-1)
    if result is not None:
        if not (_is_torch(result) and result.is_cuda and result.is_contiguous()
                and result.numel() * result.element_size() >= STEP_RESULT_BYTES):
            raise ValueError("result must be a contiguous CUDA tensor of >= 16 bytes "
                             "(see step_result_buffer)")
        o.result_dev = ctypes.c_void_p(result.data_ptr())
    else:
        o.n_exact = ctypes.pointer(keep["nex"])
    return o, keep


def _cuda_ref(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            return a
    return None


def _phases(keep):
    if "ph" not in keep:
        return None
    return {k: float(v) for k, v in zip(PHASES, keep["ph"])}


@dataclass
class TrainResult:
    status: int
    C: object
    assign: object
    D: float
    records: list
    n_passes: int
    phase_ms: dict | None
    pass_C: object = None       # [passes, N, L] device: codebook each pass's allocation used
    pass_assign: object = None  # [passes, M] device: each pass's cell table

    def passes_per_stage(self):
        out = []
        for r in self.records:
            if r["pass"] == 0:
                out.append(0)
            out[-1] += 1
        return out


@dataclass
class StepResult:
    status: int
    C: object
    assign: object
    D: float            # nan for an asynchronous call (read its report instead)
    n_exact: int        # -1 for an asynchronous call
    phase_ms: dict | None
    result: object = None   # the device report buffer of an asynchronous call


@dataclass
class EncodeResult:
    status: int
    idx: object
    Xhat: object
    D: float            # nan for an asynchronous call or with_distortion=False
    n_exact: int        # -1 for an asynchronous call
    phase_ms: dict | None
    result: object = None   # the device report buffer of an asynchronous call


# ------------------------------------------------------------ entry points
def lbg_train(X, N: int, delta: float = 0.01, theta: float = 1e-3, C_init=None,
              max_passes: int = 1000, trace: int = 4096, phase_ms: bool = False, C_out=None,
              assign_out=None, stream=None, precision: str = "fp32",
              split_multiplicative: bool = False, reseed_empty: bool = False,
              trace_passes: int = 0, tc_group: int = 0) -> TrainResult:
    """Design an N-entry codebook from X [M, L] (see lbg_train in lbgvq.h).  With
    trace_passes > 0 (X on a CUDA device) the codebook and the cell table of each of the first
    trace_passes passes are kept on the device (result.pass_C, result.pass_assign, one entry
    per pass run)."""
    Xo, xp, _ = _prep(X, "f32", "X")
    M, L = int(X.shape[0]), int(X.shape[1])
    C = C_out if C_out is not None else _empty_like_src(X, (N, L), "f32")
    n_init = 0
    if C_init is not None:
        n_init = int(C_init.shape[0])
        C[:n_init] = C_init
    A = assign_out if assign_out is not None else _empty_like_src(X, (M,), "i32")
    Co, cp, _ = _prep(C, "f32", "C")
    Ao, ap, _ = _prep(A, "i32", "assign")
    o, keep = _opts(_cuda_ref(X, C, A), max_passes, trace, phase_ms, stream, precision,
                    split_multiplicative, reseed_empty, tc_group=tc_group)
    pC = pA = None
    if trace_passes > 0:
        ref = _cuda_ref(X)
        if ref is None:
            raise ValueError("trace_passes needs X on a CUDA device (the trace is device memory)")
        import torch
        pC = torch.zeros((trace_passes, N, L), dtype=torch.float32, device=ref.device)
        pA = torch.full((trace_passes, M), -1, dtype=torch.int32, device=ref.device)
        o.trace_C, o.trace_assign, o.trace_cap = pC.data_ptr(), pA.data_ptr(), int(trace_passes)
    D = ctypes.c_double(0.0)
    rc = _check(lib().lbg_train(xp, M, L, int(N), float(delta), float(theta), cp, n_init, ap,
                                ctypes.byref(D), ctypes.byref(o)))
    recs = []
    if trace:
        n = min(keep["nrec"].value, trace)
        for r in keep["rec"][:n]:
            recs.append({"stage_n": r.stage_n, "pass": r.pass_, "action": ACTIONS[r.action],
                         "n_exact": r.n_exact, "D": r.D, "n_empty": r.n_empty, "ms": r.ms})
    n_passes = keep["nrec"].value if trace else -1
    if pC is not None and n_passes >= 0:
        pC, pA = pC[:n_passes], pA[:n_passes]
    return TrainResult(rc, C, A, D.value, recs, n_passes, _phases(keep), pC, pA)


def lbg_lloyd_step(X, C_in, C_out=None, assign_out=None, phase_ms: bool = False,
                   stream=None, precision: str = "fp32", reseed_empty: bool = False,
                   delta_reseed: float = 0.01, result_out=None,
                   test_expire_wait: bool = False, tc_group: int = 0) -> StepResult:
    """One Lloyd pass from C_in (see lbg_lloyd_step in lbgvq.h).  With result_out (a
    step_result_buffer) the pass is only enqueued on the stream: D, n_exact and the
    device status land in result_out (read_step_result)."""
    Xo, xp, _ = _prep(X, "f32", "X")
    M, L = int(X.shape[0]), int(X.shape[1])
    N = int(C_in.shape[0])
    Ci, cip, _ = _prep(C_in, "f32", "C_in")
    Co = C_out if C_out is not None else _empty_like_src(C_in, (N, L), "f32")
    Co, cop, _ = _prep(Co, "f32", "C_out")
    A = assign_out if assign_out is not None else _empty_like_src(X, (M,), "i32")
    A, ap, _ = _prep(A, "i32", "assign")
    o, keep = _opts(_cuda_ref(X, C_in, Co, A), stream=stream, phase=phase_ms, precision=precision,
                    reseed_empty=reseed_empty, delta_reseed=delta_reseed, result=result_out,
                    test_expire_wait=test_expire_wait, tc_group=tc_group)
    if result_out is not None:
        rc = _check(lib().lbg_lloyd_step(xp, M, L, N, cip, cop, ap, None, ctypes.byref(o)))
        return StepResult(rc, Co, A, float("nan"), -1, None, result_out)
    D = ctypes.c_double(0.0)
    rc = _check(lib().lbg_lloyd_step(xp, M, L, N, cip, cop, ap, ctypes.byref(D), ctypes.byref(o)))
    return StepResult(rc, Co, A, D.value, keep["nex"].value, _phases(keep))


def vq_encode(X, C, decode: bool = False, with_distortion: bool = True, phase_ms: bool = False,
              idx_out=None, stream=None, precision: str = "fp32", result_out=None,
              test_expire_wait: bool = False, tc_group: int = 0) -> EncodeResult:
    """Nearest codevector of every row of X (see vq_encode in lbgvq.h).  With result_out
    (a step_result_buffer) the call is only enqueued, as for lbg_lloyd_step."""
    Xo, xp, _ = _prep(X, "f32", "X")
    M, L = int(X.shape[0]), int(X.shape[1])
    N = int(C.shape[0])
    Co, cp, _ = _prep(C, "f32", "C")
    I = idx_out if idx_out is not None else _empty_like_src(X, (M,), "i32")
    I, ip, _ = _prep(I, "i32", "idx")
    H = _empty_like_src(X, (M, L), "f32") if decode else None
    H, hp, _ = _prep(H, "f32", "Xhat")
    o, keep = _opts(_cuda_ref(X, C, I), stream=stream, phase=phase_ms, precision=precision,
                    result=result_out, test_expire_wait=test_expire_wait, tc_group=tc_group)
    if result_out is not None:
        rc = _check(lib().vq_encode(xp, M, L, cp, N, ip, hp, None, ctypes.byref(o)))
        return EncodeResult(rc, I, H, float("nan"), -1, None, result_out)
    D = ctypes.c_double(0.0)
    rc = _check(lib().vq_encode(xp, M, L, cp, N, ip, hp, ctypes.byref(D) if with_distortion else None,
                                ctypes.byref(o)))
    return EncodeResult(rc, I, H, D.value if with_distortion else float("nan"), keep["nex"].value,
                        _phases(keep))


def distortion_backward(X, C, assign, grad_D: float = 1.0, want_dC: bool = True,
                        want_dX: bool = True, phase_ms: bool = False, stream=None,
                        grad_scale=None, result_out=None):
    """D at the fixed cell table `assign` and its gradients (see lbg_distortion_backward in
    lbgvq.h).  Returns (D, dC or None, dX or None, phase_ms).  grad_scale: a one-element
    float32 CUDA tensor holding the upstream gradient (read on the device; grad_D is then
    ignored).  result_out (a step_result_buffer): the call is only enqueued, D lands there
    (the returned D is nan)."""
    Xo, xp, _ = _prep(X, "f32", "X")
    M, L = int(X.shape[0]), int(X.shape[1])
    N = int(C.shape[0])
    Co, cp, _ = _prep(C, "f32", "C")
    Ao, ap, _ = _prep(assign, "i32", "assign")
    dC = _empty_like_src(C, (N, L), "f32") if want_dC else None
    dX = _empty_like_src(X, (M, L), "f32") if want_dX else None
    dC, dcp, _ = _prep(dC, "f32", "dC")
    dX, dxp, _ = _prep(dX, "f32", "dX")
    o, keep = _opts(_cuda_ref(X, C, assign), stream=stream, phase=phase_ms, result=result_out)
    if grad_scale is not None:
        gs, gp, gcuda = _prep(grad_scale, "f32", "grad_scale")
        if not gcuda:
            raise ValueError("grad_scale must be a CUDA tensor")
        o.grad_scale_dev = gp
        grad_D = 0.0
    if result_out is not None:
        _check(lib().lbg_distortion_backward(xp, M, L, cp, N, ap, float(grad_D), dcp, dxp, None,
                                             ctypes.byref(o)))
        return float("nan"), dC, dX, None
    D = ctypes.c_double(0.0)
    _check(lib().lbg_distortion_backward(xp, M, L, cp, N, ap, float(grad_D), dcp, dxp,
                                         ctypes.byref(D), ctypes.byref(o)))
    return D.value, dC, dX, _phases(keep)


@dataclass
class BatchedResult:
    status: int
    C: object            # [sum N_s, L] codebooks concatenated
    assign: object       # [sum M_s] local cell indices
    D: list
    code_off: list       # codebook s is C[code_off[s]:code_off[s+1]]
    max_passes_run: int
    phase_ms: dict | None
    tune: dict | None = None   # tile of the batched assignment and its calibration

    def codebook(self, s):
        return self.C[self.code_off[s]:self.code_off[s + 1]]


def lbg_train_batched(X, row_off, N, delta: float = 0.01, theta: float = 1e-3,
                      max_passes: int = 1000, phase_ms: bool = False, stream=None,
                      split_multiplicative: bool = False, autotune: bool = True,
                      tile_rows: int = 0, ctas_per_sm: int = 0, per_phase: bool = False) -> BatchedResult:
    """S independent LBG designs at once (see lbg_train_batched in lbgvq.h).  X holds the rows
    of all problems concatenated; row_off (S+1 offsets) and N (S sizes) are Python sequences.
    The tile of the batched nearest-codevector launch is autotuned (or forced with tile_rows /
    ctas_per_sm); the choice is in the result's ``tune``.  Each pass is one persistent launch
    unless per_phase (or a forced tile) asks for one launch per phase."""
    Xo, xp, _ = _prep(X, "f32", "X")
    L = int(X.shape[1])
    S = len(N)
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    Nn = np.ascontiguousarray(N, dtype=np.int32)
    if ro.shape[0] != S + 1:
        raise ValueError("row_off must have len(N) + 1 entries")
    code_off = [0]
    for n in Nn.tolist():
        code_off.append(code_off[-1] + n)
    C = _empty_like_src(X, (code_off[-1], L), "f32")
    A = _empty_like_src(X, (int(ro[-1]),), "i32")
    Co, cp, _ = _prep(C, "f32", "C")
    Ao, ap, _ = _prep(A, "i32", "assign")
    D = np.zeros(S, np.float64)
    o, keep = _opts(_cuda_ref(X, C), max_passes, 0, phase_ms, stream, "fp32", split_multiplicative)
    nrec = ctypes.c_int32(0)
    o.n_records = ctypes.pointer(nrec)
    o.autotune = int(bool(autotune))
    o.tile_rows = int(tile_rows)
    o.ctas_per_sm = int(ctas_per_sm)
    o.batched_per_phase = int(bool(per_phase))
    rep = TuneReport()
    o.tune_report = ctypes.pointer(rep)
    rc = _check(lib().lbg_train_batched(S, xp, ro.ctypes.data, L, Nn.ctypes.data, float(delta),
                                        float(theta), cp, ap, D.ctypes.data, ctypes.byref(o)))
    return BatchedResult(rc, C, A, D.tolist(), code_off, nrec.value, _phases(keep), rep.as_dict())


def vq_encode_noalloc(X, C, idx_out=None, with_distortion: bool = True, stream=None):
    """(idx, D) of vq_encode_noalloc (see lbgvq.h): X, C and idx are CUDA tensors; the call
    allocates no device memory (D is nan without with_distortion)."""
    Xo, xp, xc = _prep(X, "f32", "X")
    Co, cp, cc = _prep(C, "f32", "C")
    if not (xc and cc):
        raise ValueError("vq_encode_noalloc needs X and C on a CUDA device")
    M, L, N = int(X.shape[0]), int(X.shape[1]), int(C.shape[0])
    I = idx_out if idx_out is not None else _empty_like_src(X, (M,), "i32")
    I, ip, _ = _prep(I, "i32", "idx")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(X.device).cuda_stream
    D = ctypes.c_double(float("nan"))
    _check(lib().vq_encode_noalloc(xp, M, L, cp, N, ip, ctypes.byref(D) if with_distortion else None,
                                   ctypes.c_void_p(int(stream))))
    return I, D.value


def release_workspace() -> None:
    _check(lib().lbg_release_workspace())


def set_workspace_limit(nbytes: int) -> None:
    """Cap the library's cached device scratch at nbytes (0: no cap); see lbg_set_workspace_limit."""
    _check(lib().lbg_set_workspace_limit(int(nbytes)))


def launch_count() -> int:
    """Kernels this library has launched in this process (graph replays included)."""
    return int(lib().lbg_launch_count())


def measure_fp32_peak(stream=None):
    """(TFLOP/s of FP32 FMA measured on the current device, its SM count)."""
    tf = ctypes.c_double(0.0)
    sms = ctypes.c_int32(0)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().lbg_measure_fp32_peak(ctypes.c_void_p(int(stream)), ctypes.byref(tf), ctypes.byref(sms)))
    return tf.value, sms.value


def version() -> int:
    return int(lib().lbg_version())
