"""The Marschner-Lobb input signal (CPU only): closed-form values at the centre, on the
z faces and at a corner, its range, and the Greville-sampled model's shape."""
import math

import numpy as np

import synth


def _F(x, y, z, fm=6.0, a=0.25):
    r = math.hypot(x, y)
    rho = math.cos(2 * math.pi * fm * math.cos(math.pi * r / 2))
    return (1 - math.sin(math.pi * z / 2) + a * (1 + rho)) / (2 * (1 + a))


def test_closed_form_values():
    f = synth.MarschnerLobb()
    pts = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 1.0], [0.5, 0.5, 0.0], [1.0, 1.0, 0.25], [0.2, 0.9, 0.7]])
    got = f.at(pts)
    assert abs(got[0] - 0.6) < 1e-15                 # (1 + 2 alpha) / (2 (1 + alpha))
    assert abs(got[1] - 0.2) < 1e-15                 # z = 1: (2 alpha) / (2 (1 + alpha))
    assert abs(got[2] - 1.0) < 1e-15                 # z = -1: (2 + 2 alpha) / (2 (1 + alpha))
    for p, g in zip(pts[3:], got[3:]):
        assert abs(g - _F(*(2 * p - 1))) < 1e-14


def test_range_and_model():
    f = synth.MarschnerLobb()
    rng = np.random.default_rng(0)
    v = f.at(rng.uniform(0, 1, (20000, 3)))
    assert v.min() >= 0.0 and v.max() <= 1.0
    spec = synth.marschner_lobb_model(20, 2)
    assert spec.ctrl.shape == (20, 20, 20) and spec.degree == (2, 2, 2)
    g = synth.greville(spec.knots[0], 2)
    np.testing.assert_allclose(spec.ctrl[3, 5, 7], f.at(np.array([[g[7], g[5], g[3]]]))[0], rtol=1e-6)


def test_device_grid_matches_host_grid():
    torch = __import__("pytest").importorskip("torch")
    f = synth.MarschnerLobb()
    m = 17
    u = np.arange(m, dtype=np.float64) / (m - 1)
    ref = f.grid(u, u, u)
    got = f.grid_device(m, device="cpu").numpy()
    assert got.shape == (m, m, m) and got.dtype == np.float32
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7)
