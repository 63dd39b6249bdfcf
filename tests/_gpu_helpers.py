"""Shared helpers of the GPU parity tests (comparison rules of the parity contract)."""
import numpy as np

import oracle

GAP_TOL = 1e-5      # near-tie exemption: rows whose two best FP64 distances differ <= 1e-5 relative
C_TOL = 1e-4        # codebook: max_n ||c_gpu - c_ref||_inf / max(||c_ref||_inf, 1)
D_TOL = 1e-5        # total distortion, relative


def check_assign(X, C, a_gpu, a_ref, e_ref, gap_ref):
    """Index-for-index equality outside near-ties; on an exempt row the GPU's
    choice must itself be within GAP_TOL of the minimum distance."""
    a_gpu = np.asarray(a_gpu)
    mism = a_gpu != a_ref
    exempt = gap_ref <= GAP_TOL
    bad = np.flatnonzero(mism & ~exempt)
    assert bad.size == 0, f"{bad.size} non-exempt mismatches, e.g. rows {bad[:5]}"
    alt = np.flatnonzero(mism)
    if alt.size:
        Xd = np.asarray(X, np.float64)[alt]
        d = ((Xd - np.asarray(C, np.float64)[a_gpu[alt]]) ** 2).sum(1)
        assert np.all(d <= e_ref[alt] * (1 + GAP_TOL) + 1e-30)
    return int(alt.size)


def check_codebook(C_gpu, C_ref):
    C_gpu = np.asarray(C_gpu, np.float64)
    C_ref = np.asarray(C_ref, np.float64)
    num = np.abs(C_gpu - C_ref).max(1)
    den = np.maximum(np.abs(C_ref).max(1), 1.0)
    worst = float((num / den).max()) if len(num) else 0.0
    assert worst <= C_TOL, f"codebook rel error {worst}"
    return worst


def check_D(D_gpu, D_ref):
    if D_ref == 0:
        assert D_gpu == 0
        return 0.0
    rel = abs(D_gpu - D_ref) / abs(D_ref)
    assert rel <= D_TOL, f"D rel error {rel} ({D_gpu} vs {D_ref})"
    return rel
