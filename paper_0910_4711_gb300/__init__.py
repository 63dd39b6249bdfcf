"""GB300-native LBG vector-quantizer design (Annaji & Rao, Sec. 2.2 and Algorithm 1).

The computation runs in the CUDA library ``_lib/liblbgvq.so`` (C ABI in
``include/lbgvq.h``, kernels in ``csrc/``); this package only marshals
arguments to it.  Build it with :func:`paper_0910_4711_gb300.build.build`.
"""
from ._binding import (EXPORTS, LBGError, LIB_PATH, distortion_backward, launch_count, lbg_lloyd_step,
                       lbg_train, lbg_train_batched, lib, measure_fp32_peak, read_step_result,
                       release_workspace, set_workspace_limit, step_result_buffer, version, vq_encode,
                       vq_encode_noalloc)

__all__ = ["lbg_train", "lbg_train_batched", "lbg_lloyd_step", "vq_encode", "vq_encode_noalloc",
           "distortion_backward", "release_workspace", "set_workspace_limit", "launch_count",
           "measure_fp32_peak", "step_result_buffer", "read_step_result",
           "version", "lib", "LBGError", "LIB_PATH", "EXPORTS"]
