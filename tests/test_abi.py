"""The C-ABI library builds, loads without a GPU, exports every function that
include/lbgvq.h declares, and rejects invalid arguments before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_0910_4711_gb300 as lbgvq
from paper_0910_4711_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbgvq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(\w+)\s*\([^;{]*\)\s*;", text)) - {"if", "while"})


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbgvq.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("lbg_train", "lbg_lloyd_step", "vq_encode", "lbg_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings_and_version(lib):
    assert lib.lbg_version() == 2
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert lib.lbg_status_string(s)


def _err(fn, *args):
    with pytest.raises(lbgvq.LBGError) as ei:
        fn(*args)
    return ei.value.status


def test_train_rejects_bad_arguments(lib):
    X = np.zeros((8, 4), np.float32)
    assert _err(lbgvq.lbg_train, X, 3) == -2          # N not a power of 2
    assert _err(lbgvq.lbg_train, X, 0) == -1
    assert _err(lbgvq.lbg_train, X, 2 * 8192) == -1   # above LBG_MAX_CODEBOOK
    assert _err(lbgvq.lbg_train, X, 4, -0.5) == -1    # delta < 0
    assert _err(lbgvq.lbg_train, X, 4, 0.1, -1.0) == -1
    assert _err(lbgvq.lbg_train, X, 4, 0.1, float("nan")) == -1
    assert _err(lbgvq.lbg_train, np.zeros((8, 129), np.float32), 4) == -1   # L > LBG_MAX_DIM
    assert _err(lbgvq.lbg_train, np.zeros((0, 4), np.float32), 4) == -1     # M = 0
    assert _err(lbgvq.lbg_train, X, 4, 0.1, 0.1, np.zeros((3, 4), np.float32)) == -2  # n_init


def test_step_and_encode_reject_bad_arguments(lib):
    X = np.zeros((8, 4), np.float32)
    assert _err(lbgvq.lbg_lloyd_step, np.zeros((8, 0), np.float32), np.zeros((2, 0), np.float32)) == -1
    assert _err(lbgvq.vq_encode, X, np.zeros((0, 4), np.float32)) == -1
    assert _err(lbgvq.vq_encode, X, np.zeros((9000, 4), np.float32)) == -1
    P = ctypes.c_void_p
    # null codebook through the raw ABI
    assert lib.vq_encode(None, 8, 4, None, 2, None, None, None, None) == -1
    assert lib.lbg_lloyd_step(None, 8, 4, 2, None, None, None, None, None) == -1


def test_opts_defaults(lib):
    from paper_0910_4711_gb300 import _binding
    o = _binding.Opts()
    lib.lbg_opts_init(ctypes.byref(o))
    assert o.precision == 0 and o.max_passes == 1000
    assert o.autotune == 1 and o.tile_rows == 0 and o.ctas_per_sm == 0
    assert not o.tune_report and not o.records and not o.phase_ms


def test_batched_rejects_bad_tile_options(lib):
    X = np.zeros((256, 16), np.float32)
    ro, N = [0, 256], [4]
    assert _err(lbgvq.lbg_train_batched, X, ro, N, 0.01, 1e-3, 1000, False, None, False, True, 96) == -1
    assert _err(lbgvq.lbg_train_batched, X, ro, N, 0.01, 1e-3, 1000, False, None, False, True, 64, 3) == -1
    assert _err(lbgvq.lbg_train_batched, X, ro, N, 0.01, 1e-3, 1000, False, None, False, True, 128, 4) == -1


def test_struct_layout_matches_header(tmp_path):
    """The binding's ctypes mirrors have the C compiler's sizes and offsets."""
    import subprocess
    from paper_0910_4711_gb300 import _binding
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "lbgvq.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbg_opts), offsetof(lbg_opts, tune_report),\n'
        "         offsetof(lbg_opts, result_dev), sizeof(lbg_step_result),\n"
        "         offsetof(lbg_step_result, n_exact), offsetof(lbg_step_result, status));\n"
        '  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbg_pass_record),\n'
        "         offsetof(lbg_pass_record, D), offsetof(lbg_pass_record, n_empty),\n"
        "         offsetof(lbg_pass_record, ms), offsetof(lbg_opts, trace_C),\n"
        "         offsetof(lbg_opts, trace_cap), offsetof(lbg_opts, test_expire_wait));\n"
        '  printf("%zu %zu\\n", offsetof(lbg_opts, grad_scale_dev), offsetof(lbg_opts, tc_group));\n'
        "  return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    O, R = _binding.Opts, _binding.PassRecord
    assert got[:3] == [ctypes.sizeof(O), O.tune_report.offset, O.result_dev.offset]
    assert got[3:6] == [_binding.STEP_RESULT_BYTES, 8, 12]
    assert got[6:13] == [ctypes.sizeof(R), R.D.offset, R.n_empty.offset, R.ms.offset, O.trace_C.offset,
                         O.trace_cap.offset, O.test_expire_wait.offset]
    assert got[13:] == [O.grad_scale_dev.offset, O.tc_group.offset]


def test_tc_group_option_is_checked(lib):
    """tc_group accepts 0, 2, 4 and 8; any other value is LBG_ERR_ARG before any device
    work (the pointers are never dereferenced)."""
    from paper_0910_4711_gb300 import _binding
    fake = ctypes.c_void_p(0x1000)
    D = ctypes.c_double(0.0)
    for g, bad in ((3, True), (16, True), (-2, True), (4, False), (0, False)):
        o = _binding.Opts()
        lib.lbg_opts_init(ctypes.byref(o))
        assert o.tc_group == 0
        o.tc_group = g
        o.precision = 1
        rc = lib.vq_encode(fake, 8, 4, fake, 2, fake, None, ctypes.byref(D), ctypes.byref(o))
        assert (rc == -1) == bad, (g, rc)


def test_async_calls_reject_host_outs(lib):
    """An asynchronous step / encode (result_dev set) refuses host outputs before
    any device work."""
    from paper_0910_4711_gb300 import _binding
    o = _binding.Opts()
    lib.lbg_opts_init(ctypes.byref(o))
    assert not o.result_dev
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: the call returns first
    o.result_dev = fake
    D = ctypes.c_double(0.0)
    assert lib.lbg_lloyd_step(fake, 8, 4, 2, fake, fake, None, ctypes.byref(D), ctypes.byref(o)) == -1
    assert lib.vq_encode(fake, 8, 4, fake, 2, fake, None, ctypes.byref(D), ctypes.byref(o)) == -1
    n = ctypes.c_int32(0)
    o.n_exact = ctypes.pointer(n)
    assert lib.lbg_lloyd_step(fake, 8, 4, 2, fake, fake, None, None, ctypes.byref(o)) == -1


def test_binding_rejects_bad_arrays(lib):
    """The binding only marshals: a wrong dtype, a non-contiguous array or an
    unknown precision is refused before the library is called."""
    import torch
    X = np.zeros((8, 4), np.float32)
    with pytest.raises(TypeError):
        lbgvq.lbg_train(X.astype(np.float64), 4)
    with pytest.raises(TypeError):
        lbgvq.vq_encode(np.asfortranarray(np.zeros((8, 4), np.float32)), X[:2])
    with pytest.raises(TypeError):
        lbgvq.vq_encode(torch.zeros((8, 4), dtype=torch.float64), torch.zeros((2, 4)))
    with pytest.raises(ValueError):
        lbgvq.vq_encode(torch.zeros((4, 8)).t(), torch.zeros((2, 4)))
    with pytest.raises(ValueError):
        lbgvq.lbg_lloyd_step(X, X[:2], precision="fp16")


@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")])
def test_header_compiles_cleanly(tmp_path, compiler, std, ext):
    """include/lbgvq.h is usable from plain C and from C++ without warnings
    (extern "C" linkage, no C++-only or compiler-specific constructs)."""
    import subprocess
    src = tmp_path / f"use.{ext}"
    src.write_text('#include "lbgvq.h"\n'
                   "int main(void) {\n"
                   "  lbg_opts o;\n"
                   "  lbg_opts_init(&o);\n"
                   "  return (int)o.precision + (int)sizeof(lbg_step_result) - 16;\n"
                   "}\n")
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True)


def test_plain_c_program_links_and_calls(lib, tmp_path):
    """A C program links liblbgvq directly (no Python) and calls the ABI: the
    version, a status string, and calls that the library rejects before any
    device work (N not a power of 2, a null codebook)."""
    import subprocess
    libdir = os.path.dirname(lbgvq.LIB_PATH)
    src = tmp_path / "client.c"
    src.write_text(
        '#include <stdio.h>\n#include <string.h>\n#include "lbgvq.h"\n'
        "int main(void) {\n"
        "  float X[8 * 4] = {0}, C[3 * 4];\n"
        "  int32_t idx[8];\n"
        "  if (lbg_version() != 2) return 1;\n"
        '  if (strcmp(lbg_status_string(LBG_ERR_NOT_POW2), "codebook size is not a power of 2")) return 2;\n'
        "  if (lbg_train(X, 8, 4, 3, 0.01, 1e-3, C, 0, NULL, NULL, NULL) != LBG_ERR_NOT_POW2) return 3;\n"
        "  if (vq_encode(X, 8, 4, NULL, 2, idx, NULL, NULL, NULL) != LBG_ERR_ARG) return 4;\n"
        '  printf("ok\\n");\n'
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-llbgvq", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stderr)
