"""Pins for the ground-truth and image-quality oracles (CPU only).

The closed-form Marschner-Lobb signal (Sec. V-A.1, Eq. 1): values at points where the
formula reduces by hand (rho = 1, 0, -1), its extremes, agreement with the input
generator's independent implementation, the analytic gradient against central finite
differences (including next to the axis r = 0, where the x / r factor is continued), and
the render of the signal through a one-sample ray whose colour is the signal itself.

MSE / PSNR / SSIM (Table II's metrics): equal images, constant offsets (closed-form MSE
and PSNR), constant images (SSIM reduces to the luminance term), a ramp and its shifted
copy (window means of a linear image are its centre values) and a ramp and its scaled
copy (window variances of a ramp are a^2 times the 1-D Gaussian's second moment), and the
clamp to the display range.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import quality

FM, ALPHA = 6.0, 0.25
DEN = 2 * (1 + ALPHA)


def _uvw(x, y, z):
    return [(x + 1) / 2, (y + 1) / 2, (z + 1) / 2]


def test_ml_closed_form_points():
    # centre: r = 0, cos(pi r / 2) = 1, rho = cos(12 pi) = 1; z = 0
    assert oracle.ml_eval(_uvw(0, 0, 0))[0] == pytest.approx((1 + 2 * ALPHA) / DEN, abs=1e-15)
    # r = 1: cos(pi / 2) = 0, rho = 1
    assert oracle.ml_eval(_uvw(1, 0, 0))[0] == pytest.approx((1 + 2 * ALPHA) / DEN, abs=1e-14)
    # cos(pi r / 2) = 1 / (4 f_M): rho = cos(pi / 2) = 0
    r0 = 2 / math.pi * math.acos(1 / (4 * FM))
    assert oracle.ml_eval(_uvw(r0 / math.sqrt(2), r0 / math.sqrt(2), 0.5))[0] == pytest.approx(
        (1 - math.sin(math.pi / 4) + ALPHA) / DEN, abs=1e-13)
    # cos(pi r / 2) = 1 / (2 f_M): rho = cos(pi) = -1; at z = 1 the global minimum 0
    r1 = 2 / math.pi * math.acos(1 / (2 * FM))
    assert oracle.ml_eval(_uvw(0, r1, 1))[0] == pytest.approx(0.0, abs=1e-14)
    # z = -1 with rho = 1: the global maximum 1
    assert oracle.ml_eval(_uvw(0, 0, -1))[0] == pytest.approx(1.0, abs=1e-15)


def test_ml_matches_input_generator():
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (200, 3))
    ref = synth.MarschnerLobb().at(pts)
    got = np.array([oracle.ml_eval(p)[0] for p in pts])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_ml_gradient_finite_differences():
    rng = np.random.default_rng(4)
    pts = list(rng.uniform(0.02, 0.98, (40, 3)))
    pts += [np.array([0.5 + 1e-7, 0.5, 0.3]), np.array([0.5, 0.5 - 3e-6, 0.8]), np.array([0.5, 0.5, 0.5])]
    h = 1e-6
    for p in pts:
        g = oracle.ml_eval(p)[1:]
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (oracle.ml_eval(p + e)[0] - oracle.ml_eval(p - e)[0]) / (2 * h)
            assert abs(g[a] - fd) <= 2e-7 * max(1.0, abs(fd)), (p, a, g[a], fd)


def test_ml_render_one_sample_is_the_signal():
    # An orthographic camera looking down -z: pixel (col, row) sees the vertical line
    # through its centre; one sample per ray sits at the middle of the unit box, w = 1/2.
    # With a grey ramp table of constant alpha a and no shading, the pixel is a (F, F, F, 1).
    cam = synth.camera_ortho((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 1.0)
    a = 0.4
    tf = np.array([[0, 0, 0, a], [1, 1, 1, a]], dtype=np.float32)
    W = H = 9
    img, ns = oracle.render_ml(cam, tf, W, H, 1, f_m=FM, alpha=ALPHA)   # value range defaults to [0, 1]
    assert ns == W * H
    for row in range(H):
        for col in range(W):
            o, d = oracle.ray(cam, W, H, col, row)
            hit, t0, t1 = oracle.clip_unit_box(o, d)
            assert hit
            x = o + 0.5 * (t0 + t1) * d
            assert x[2] == pytest.approx(0.5, abs=1e-12)
            F = synth.MarschnerLobb().at(x[None, :])[0]
            np.testing.assert_allclose(img[row, col], [a * F, a * F, a * F, a], rtol=0, atol=1e-7)


def _img(rgb):
    rgb = np.asarray(rgb, dtype=np.float64)
    return np.concatenate([rgb, np.ones(rgb.shape[:2] + (1,))], axis=-1)


def test_metrics_equal_images():
    x = _img(np.random.default_rng(0).uniform(0, 1, (20, 23, 3)))
    q = quality.compare(x, x)
    assert q["mse"] == 0.0 and q["psnr_db"] == math.inf
    assert q["ssim"] == pytest.approx(1.0, abs=1e-12)


def test_metrics_constant_offset():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 0.8, (16, 16, 3))
    delta = 7.0   # display units
    y = x + delta / 255.0
    assert quality.mse(_img(x), _img(y)) == pytest.approx(delta * delta, rel=1e-12)
    assert quality.psnr(_img(x), _img(y)) == pytest.approx(10 * math.log10(255.0 ** 2 / delta ** 2), rel=1e-12)


def test_ssim_constant_images():
    mx, my = 40.0, 90.0
    x = np.full((15, 17, 3), mx / 255.0)
    y = np.full((15, 17, 3), my / 255.0)
    expect = (2 * mx * my + quality.C1) / (mx * mx + my * my + quality.C1)
    assert quality.ssim(_img(x), _img(y)) == pytest.approx(expect, rel=1e-12)
    assert quality.C1 == pytest.approx(6.5025) and quality.C2 == pytest.approx(58.5225)


def _gauss_second_moment():
    k = np.arange(-5, 6, dtype=np.float64)
    g = np.exp(-k * k / (2 * 1.5 * 1.5))
    return float((g * k * k).sum() / g.sum())


def test_ssim_shifted_ramp():
    H, W, a, b, delta = 19, 30, 4.0, 3.0, 25.0
    row, col = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    x = a * col + b * row
    y = x + delta
    rgb = lambda v: np.repeat((v / 255.0)[..., None], 3, axis=-1)
    mu = x[5:H - 5, 5:W - 5]                  # window centres of the fully inside positions
    per_pos = (2 * mu * (mu + delta) + quality.C1) / (mu * mu + (mu + delta) ** 2 + quality.C1)
    assert quality.ssim(_img(rgb(x)), _img(rgb(y))) == pytest.approx(per_pos.mean(), rel=1e-11)


def test_ssim_scaled_ramp():
    H, W, a, s = 12, 27, 4.0, 1.7
    col = np.arange(W, dtype=np.float64)
    x = np.broadcast_to(a * col, (H, W))
    y = s * x
    rgb = lambda v: np.repeat((v / 255.0)[..., None], 3, axis=-1)
    V = _gauss_second_moment()
    mu = a * col[5:W - 5]
    C1, C2 = quality.C1, quality.C2
    per_col = ((2 * s * mu * mu + C1) * (2 * s * a * a * V + C2)) / (
        ((1 + s * s) * mu * mu + C1) * ((1 + s * s) * a * a * V + C2))
    assert quality.ssim(_img(rgb(x)), _img(rgb(y))) == pytest.approx(per_col.mean(), rel=1e-10)


def test_metrics_clamp_to_display_range():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (13, 13, 3))
    y = x.copy()
    y[2:5, 3:7] = 1.5          # over-range values display as 1
    x[2:5, 3:7] = 1.0
    y[8, 8] = -0.3             # below-range as 0
    x[8, 8] = 0.0
    assert quality.mse(_img(x), _img(y)) == 0.0
    with pytest.raises(ValueError):
        quality.ssim(_img(x[:10]), _img(y[:10]))
