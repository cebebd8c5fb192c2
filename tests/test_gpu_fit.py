"""GPU: MFA encoding (mfa_fit_ctrl, mfa_model_fit, mfa_model_encode) against the encoding
oracle (NumPy least squares per axis and the same adaptive loop)."""
import numpy as np
import pytest

import synth
from oracle import fit as of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("degree,nctrl,m", [((3, 3, 3), (9, 7, 8), (40, 31, 35)), ((2, 4, 1), (12, 8, 5), (50, 41, 12)),
                                            ((4, 2, 3), (7, 10, 6), (29, 44, 23))])
def test_fit_matches_oracle(mfa, degree, nctrl, m):
    rng = np.random.default_rng(sum(nctrl) + sum(m))
    knots = [synth.knots_nonuniform(nctrl[a], degree[a], rng, 2.0) for a in range(3)]
    D = rng.standard_normal((m[2], m[1], m[0])).astype(np.float32)
    ref = of.fit(degree, knots, D.astype(np.float64))
    got = mfa.fit_ctrl(degree, nctrl, knots, _cuda(D)).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_fit_recovers_a_spline(mfa):
    rng = np.random.default_rng(7)
    degree, nctrl, m = (3, 3, 3), (10, 9, 11), (41, 37, 45)
    knots = [synth.knots_uniform(nctrl[a], 3) for a in range(3)]
    P = rng.standard_normal((nctrl[2], nctrl[1], nctrl[0]))
    D = of.evaluate_grid(degree, knots, P, (m[2], m[1], m[0]))
    got = mfa.fit_ctrl(degree, nctrl, None, _cuda(D)).cpu().numpy()
    assert np.abs(got - P).max() <= 1e-5 * np.abs(P).max()      # the data are FP32-rounded
    model, err = mfa.model_fit(degree, nctrl, None, _cuda(D))
    assert err <= 1e-5 * np.abs(D).max()
    assert model.info()["cardinal"] and model.nctrl == nctrl


def test_model_fit_error_matches_oracle(mfa):
    rng = np.random.default_rng(8)
    f = synth.GaussianSum.draw(rng, 5)
    m = (48, 40, 36)
    D = f.grid(of.grid_params(m[0]), of.grid_params(m[1]), of.grid_params(m[2])).astype(np.float32)
    degree, nctrl = (3, 3, 3), (12, 10, 9)
    knots = [synth.knots_uniform(nctrl[a], 3) for a in range(3)]
    P = of.fit(degree, knots, D.astype(np.float64))
    ref_err = np.abs(of.evaluate_grid(degree, knots, P, D.shape) - D.astype(np.float64)).max()
    model, err = mfa.model_fit(degree, nctrl, None, _cuda(D))
    assert err == pytest.approx(ref_err, rel=1e-3, abs=1e-6 * np.abs(D).max())


def test_adaptive_encoding_matches_oracle(mfa):
    rng = np.random.default_rng(9)
    f = synth.GaussianSum.draw(rng, 4)
    m = (45, 39, 33)
    D = f.grid(of.grid_params(m[0]), of.grid_params(m[1]), of.grid_params(m[2])).astype(np.float32)
    err_max = 3e-3 * float(np.abs(D).max())
    knots, P, hist = of.encode((3, 3, 3), D.astype(np.float64), err_max, max_ctrl=(24, 24, 24))
    model, res = mfa.model_encode((3, 3, 3), _cuda(D), err_max, max_ctrl=(24, 24, 24))
    assert res["nctrl"] == hist[-1][1]
    assert res["iterations"] == len(hist)
    assert res["max_err"] <= err_max * (1 + 1e-4)
    assert res["max_err"] == pytest.approx(hist[-1][0], rel=1e-3)
    assert model.nctrl == hist[-1][1]


def test_fit_rejects_undetermined_data(mfa):
    rng = np.random.default_rng(10)
    D = _cuda(rng.standard_normal((6, 7, 8)))
    with pytest.raises(mfa.MfaError):
        mfa.fit_ctrl((3, 3, 3), (9, 5, 5), None, D)                   # more control points than data on x
    # degree 1 on x: the hat function on [0.4, 0.5] holds none of the parameters 0, 1/4, ..., 1
    U = np.array([0, 0, 0.4, 0.45, 0.5, 1, 1.0])
    D = _cuda(rng.standard_normal((4, 4, 5)))
    with pytest.raises(mfa.MfaError, match="determine"):
        mfa.fit_ctrl((1, 1, 1), (5, 3, 3), [U, None, None], D)
    mfa.fit_ctrl((1, 1, 1), (5, 3, 3), None, D)                       # uniform knots: determined


def test_wide_x_error_projection_matches_oracle(mfa):
    """More than 8192 data points along x: the error pass folds the x-projection with global
    atomics instead of its per-block shared-memory table; the error and the adaptive loop's
    knot decisions (which read the x-projection) still match the oracle's."""
    rng = np.random.default_rng(10)
    m = (8500, 6, 5)
    x = of.grid_params(m[0])
    fx = np.sin(9.0 * x) + 0.5 * np.exp(-((x - 0.3) / 0.05) ** 2)
    D = (fx[None, None, :] * (1.0 + 0.1 * of.grid_params(m[1])[None, :, None])
         + 0.05 * of.grid_params(m[2])[:, None, None]).astype(np.float32)
    degree, nctrl = (2, 1, 1), (40, 4, 3)
    knots = [synth.knots_uniform(nctrl[a], degree[a]) for a in range(3)]
    P = of.fit(degree, knots, D.astype(np.float64))
    ref_err = np.abs(of.evaluate_grid(degree, knots, P, D.shape) - D.astype(np.float64)).max()
    model, err = mfa.model_fit(degree, nctrl, None, _cuda(D))
    assert err == pytest.approx(ref_err, rel=1e-3, abs=1e-6 * np.abs(D).max())
    err_max = 2e-3 * float(np.abs(D).max())
    knots_ref, _, hist = of.encode(degree, D.astype(np.float64), err_max, max_ctrl=(96, 6, 5))
    model, res = mfa.model_encode(degree, _cuda(D), err_max, max_ctrl=(96, 6, 5))
    assert res["nctrl"] == hist[-1][1] and res["iterations"] == len(hist)
    assert res["max_err"] == pytest.approx(hist[-1][0], rel=1e-3)
