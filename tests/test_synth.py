"""The seeded synthetic inputs follow their stated recipe.

The image-block workloads stand in for the paper's unnamed image data; these
tests pin what the recipe says about them: seeded and reproducible, 8-bit,
a smooth field (sigma_f = 6 px) at 128 + 48 * field plus uniform noise,
blocks in raster order flattened row-major, and the sizes of the named
workloads, the Gaussian mixture and the batched sets.
"""
import math

import numpy as np
import pytest

from paper_0910_4711_gb300 import synth


def test_image_is_seeded_and_8bit():
    a = synth.make_image(7, 256, 192)
    assert a.dtype == np.uint8 and a.shape == (256, 192)
    assert np.array_equal(a, synth.make_image(7, 256, 192))
    assert not np.array_equal(a, synth.make_image(8, 256, 192))
    assert synth.digest(a) == synth.digest(synth.make_image(7, 256, 192))


def test_image_statistics_match_the_recipe():
    """Mean 128; variance amp^2 + noise^2 / 3 (+ 1/12 for the rounding), little
    clipping at 2.6 sigma; neighbouring pixels correlated as a Gaussian blur of
    sigma_f = 6 px predicts: field correlation exp(-1 / (4 sigma_f^2)) at lag 1,
    diluted by the independent noise."""
    img = synth.make_image(3, 1024, 1024).astype(np.float64)
    assert abs(img.mean() - 128.0) < 1.5
    var = synth.AMP ** 2 + synth.NOISE ** 2 / 3 + 1 / 12
    assert img.std() == pytest.approx(math.sqrt(var), rel=0.03)
    c = img - img.mean()
    lag1 = (c[:, 1:] * c[:, :-1]).mean() / c.var()
    rho = math.exp(-1.0 / (4 * synth.SIGMA_F ** 2))
    expect = synth.AMP ** 2 * rho / var
    assert lag1 == pytest.approx(expect, abs=0.01)
    far = (c[:, 40:] * c[:, :-40]).mean() / c.var()     # lag 40 px: the field has decorrelated
    assert abs(far) < 0.05


def test_blocks_raster_order_row_major():
    H, W, b = 8, 12, 4
    img = np.arange(H * W, dtype=np.uint8).reshape(H, W)
    X = synth.blocks(img, b)
    assert X.dtype == np.float32 and X.shape == ((H // b) * (W // b), b * b)
    for k in range(X.shape[0]):
        by, bx = divmod(k, W // b)
        for i in range(b):
            for j in range(b):
                assert X[k, i * b + j] == img[by * b + i, bx * b + j]
    with pytest.raises(ValueError):
        synth.blocks(np.zeros((10, 12), np.uint8), 4)


def test_image_blocks_stack_in_seed_order():
    X = synth.image_blocks([5, 6], 64, 64, 4)
    assert X.shape == (2 * 256, 16)
    np.testing.assert_array_equal(X[:256], synth.blocks(synth.make_image(5, 64, 64), 4))
    np.testing.assert_array_equal(X[256:], synth.blocks(synth.make_image(6, 64, 64), 4))


def test_named_workload_sizes():
    sizes = {name: (len(w["seeds"]) * (w["H"] // w["b"]) * (w["W"] // w["b"]), w["b"] ** 2, w["N"])
             for name, w in synth.WORKLOADS.items()}
    assert sizes["img512_b4_n256"] == (16384, 16, 256)
    assert sizes["img2048x8_b8_n4096"] == (524288, 64, 4096)
    assert sizes["img2048x64_b4_n4096"] == (16777216, 16, 4096)
    X, N = synth.workload("img512_b4_n256")
    assert X.shape == (16384, 16) and N == 256


def test_gaussian_mixture_recipe():
    X, means, z = synth.gmm(4, 20000, L=32, K=512, sigma=0.1)
    assert X.dtype == np.float32 and X.shape == (20000, 32)
    assert means.shape == (512, 32) and means.min() >= 0.0 and means.max() < 1.0
    assert z.min() >= 0 and z.max() < 512
    resid = X.astype(np.float64) - means[z]
    assert resid.std() == pytest.approx(0.1, rel=0.02)
    assert abs(resid.mean()) < 0.002
    X2, _, _ = synth.gmm(4, 20000, L=32, K=512, sigma=0.1)
    assert np.array_equal(X, X2)


def test_batched_sets_recipe():
    sets = synth.batched_sets()
    assert len(sets) == 64 and sets == synth.batched_sets()
    seeds = [s for s, _, _ in sets]
    assert seeds == list(range(3001, 3065))
    Ms = np.array([m for _, m, _ in sets])
    assert Ms.min() >= 4096 and Ms.max() <= 262144
    assert {n for _, _, n in sets} <= {64, 128, 256, 512, 1024}
    # log-uniform: the median of log M sits near the middle of [log 4096, log 262144]
    assert abs(np.median(np.log(Ms)) - 0.5 * (np.log(4096) + np.log(262144))) < 0.8
