"""Error measures the parity tests apply (all computed in FP64 on the host).

value:    e_v = max |f_gpu - f_ref| / max |P|          (sup norm over the convex-hull bound)
gradient: e_g = max_i |g_gpu_i - g_ref_i|_2 / max_i |g_ref_i|_2
image:    per-channel RMSE over all compared pixels, values in [0,1]
Gates for FP32 arithmetic: e_v <= 1e-5, e_g <= 1e-4, RMSE <= 1e-3 per channel.
"""
import numpy as np

VALUE_TOL = 1e-5
GRAD_TOL = 1e-4
IMAGE_RMSE_TOL = 1e-3
SERVED_RMSE_TOL = 2e-3


def value_error(f_gpu, f_ref, ctrl) -> float:
    scale = float(np.max(np.abs(ctrl)))
    return float(np.max(np.abs(np.asarray(f_gpu, np.float64) - f_ref))) / max(scale, 1e-300)


def grad_error(g_gpu, g_ref) -> float:
    d = np.linalg.norm(np.asarray(g_gpu, np.float64) - g_ref, axis=-1)
    return float(d.max()) / max(float(np.linalg.norm(g_ref, axis=-1).max()), 1e-300)


def image_rmse(img_gpu, img_ref) -> np.ndarray:
    d = np.asarray(img_gpu, np.float64).reshape(-1, 4) - np.asarray(img_ref, np.float64).reshape(-1, 4)
    return np.sqrt(np.mean(d * d, axis=0))
