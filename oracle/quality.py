"""Oracle for image-quality metrics -- TEST INFRASTRUCTURE ONLY (tests, the smoke check and
the benchmark's CPU baseline may load it; the GPU library never does).

The paper scores renders against the ground-truth image by MSE, PSNR and SSIM (Table II,
Sec. V-D.3) without defining them further.  Readings, written out here in plain FP64
NumPy:
  * the images are premultiplied RGBA renders over a black background; the metrics use the
    R, G, B channels, each clamped to [0, 1] and scaled by 255 (the 8-bit display range,
    without rounding to integers), alpha ignored;
  * MSE = mean over pixels and the three channels of (a - b)^2;
  * PSNR = 10 log10(255^2 / MSE) dB (infinite for equal images);
  * SSIM is the structural similarity of Wang, Bovik, Sheikh and Simoncelli (IEEE TIP 2004)
    with their standard constants: an 11 x 11 Gaussian window of standard deviation 1.5
    normalised to sum 1, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = 255; at every window
    position lying fully inside the image,
        SSIM = (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)),
    mu the window-weighted means, s_a^2, s_b^2, s_ab the weighted (co)variances
    E_w[a^2] - mu_a^2, E_w[b^2] - mu_b^2, E_w[ab] - mu_a mu_b; the score is the mean over
    positions and channels.
"""
import math

import numpy as np

WINDOW = 11
SIGMA = 1.5
L = 255.0
C1 = (0.01 * L) ** 2
C2 = (0.03 * L) ** 2


def display(rgba) -> np.ndarray:
    """(H, W, 3) FP64: RGB clamped to [0, 1] and scaled to [0, 255]."""
    x = np.asarray(rgba, dtype=np.float64)[..., :3]
    return 255.0 * np.clip(x, 0.0, 1.0)


def gaussian_window() -> np.ndarray:
    k = np.arange(WINDOW, dtype=np.float64) - (WINDOW - 1) / 2
    g = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def mse(a, b) -> float:
    x, y = display(a), display(b)
    return float(np.mean((x - y) ** 2))


def psnr(a, b) -> float:
    e = mse(a, b)
    return math.inf if e == 0.0 else 10.0 * math.log10(L * L / e)


def _window_mean(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{dy, dx} w[dy, dx] img[y + dy, x + dx] at every position whose window fits."""
    H, W = img.shape
    out = np.zeros((H - WINDOW + 1, W - WINDOW + 1))
    for dy in range(WINDOW):
        for dx in range(WINDOW):
            out += w[dy, dx] * img[dy:dy + H - WINDOW + 1, dx:dx + W - WINDOW + 1]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM at every full window position of two single-channel images (display scale)."""
    w = gaussian_window()
    mx, my = _window_mean(x, w), _window_mean(y, w)
    sxx = _window_mean(x * x, w) - mx * mx
    syy = _window_mean(y * y, w) - my * my
    sxy = _window_mean(x * y, w) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(a, b) -> float:
    x, y = display(a), display(b)
    if x.shape[0] < WINDOW or x.shape[1] < WINDOW:
        raise ValueError("SSIM needs images of at least 11 x 11 pixels")
    return float(np.mean([ssim_map(x[..., c], y[..., c]).mean() for c in range(3)]))


def compare(a, b) -> dict:
    return {"mse": mse(a, b), "psnr_db": psnr(a, b), "ssim": ssim(a, b)}
