"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle tests.

This module holds no arithmetic of the LBG method: it only draws training
data.  The paper trains on image data that it does not name (Sec. 5 uses
2000 vectors of dimension 2..10); these generators stand in for it:

* :func:`make_image` -- an 8-bit grayscale image: a smooth periodic Gaussian
  random field (white noise blurred with a Gaussian of ``sigma_f`` pixels in
  the Fourier domain, normalised to mean 0 / std 1), scaled to
  ``128 + amp * field``, plus uniform noise in ``[-noise, noise)``, rounded
  half-to-even and clipped to 0..255.
* :func:`blocks` -- non-overlapping b x b blocks in raster order, each
  flattened row-major into a float32 vector of length L = b*b.
* :func:`image_blocks` -- blocks of several seeded images stacked.
* :func:`gmm` -- isotropic Gaussian mixture vectors.
* :func:`batched_sets` -- the recipe of many independent ragged training sets.

All draws use ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import hashlib

import numpy as np

SIGMA_F = 6.0
AMP = 48.0
NOISE = 16.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def make_image(seed: int, H: int = 512, W: int = 512, sigma_f: float = SIGMA_F,
               amp: float = AMP, noise: float = NOISE) -> np.ndarray:
    """Seeded uint8 [H, W] image (smooth random field + uniform noise)."""
    rng = _rng(seed)
    white = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    gain = np.exp(-2.0 * np.pi ** 2 * sigma_f ** 2 * (fx ** 2 + fy ** 2))
    field = np.fft.irfft2(np.fft.rfft2(white) * gain, s=(H, W))
    field = (field - field.mean()) / field.std()
    u = rng.uniform(-noise, noise, size=(H, W))
    img = np.rint(128.0 + amp * field + u)
    return np.clip(img, 0, 255).astype(np.uint8)


def blocks(img: np.ndarray, b: int) -> np.ndarray:
    """[ (H/b)*(W/b), b*b ] float32: b x b blocks in raster order, row-major inside."""
    H, W = img.shape
    if H % b or W % b:
        raise ValueError("image size must be a multiple of the block size")
    t = img.reshape(H // b, b, W // b, b).transpose(0, 2, 1, 3)
    return np.ascontiguousarray(t.reshape(-1, b * b), dtype=np.float32)


def image_blocks(seeds, H: int, W: int, b: int) -> np.ndarray:
    """Blocks of the images drawn from ``seeds``, stacked in seed order."""
    return np.concatenate([blocks(make_image(s, H, W), b) for s in seeds], axis=0)


def gmm(seed: int, M: int, L: int = 32, K: int = 512, sigma: float = 0.1):
    """M vectors of a K-component isotropic mixture: means ~ U[0,1]^L, component
    uniform, x = mean + sigma * N(0, I).  Returns (X float32 [M, L], means, z)."""
    rng = _rng(seed)
    means = rng.uniform(0.0, 1.0, size=(K, L))
    z = rng.integers(0, K, size=M)
    X = means[z] + sigma * rng.standard_normal((M, L))
    return X.astype(np.float32), means, z


def batched_sets(master_seed: int = 3000, count: int = 64, m_lo: int = 4096,
                 m_hi: int = 262144, n_choices=(64, 128, 256, 512, 1024)):
    """Sizes of ``count`` independent sets: M_s log-uniform in [m_lo, m_hi],
    N_s uniform over ``n_choices``; the data of set s are the first M_s 4x4
    blocks of its own 2048x2048 image drawn with seed master_seed + 1 + s.
    Returns a list of (image_seed, M_s, N_s)."""
    rng = _rng(master_seed)
    out = []
    for s in range(count):
        M = int(round(float(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))))
        N = int(n_choices[int(rng.integers(0, len(n_choices)))])
        out.append((master_seed + 1 + s, M, N))
    return out


def digest(a: np.ndarray) -> str:
    """SHA-256 of an array's bytes (recorded beside bench results)."""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# Named workloads (sizes of the paper-style image-block experiments).
WORKLOADS = {
    # one 512x512 image, 4x4 blocks: M=16384, L=16, N=256
    "img512_b4_n256": dict(seeds=[1], H=512, W=512, b=4, N=256),
    # eight 2048x2048 images, 8x8 blocks: M=524288, L=64, N=4096
    "img2048x8_b8_n4096": dict(seeds=list(range(2001, 2009)), H=2048, W=2048, b=8, N=4096),
    # 64 2048x2048 images, 4x4 blocks: M=16777216, L=16, N=4096
    "img2048x64_b4_n4096": dict(seeds=list(range(5001, 5065)), H=2048, W=2048, b=4, N=4096),
}


def workload(name: str):
    """(X float32 [M, L], N) of a named workload."""
    w = WORKLOADS[name]
    return image_blocks(w["seeds"], w["H"], w["W"], w["b"]), w["N"]
