"""GPU: the render-quality comparison (Sec. V-D.3, Table II) through the C ABI.

mfa_render_ml (the closed-form Marschner-Lobb signal rendered directly) against the
oracle's FP64 render of the same signal: full small images (perspective and orthographic,
with and without shading, f_M and alpha other than the paper's) and the paper's 768^2,
1024-sample shape on seeded pixels.  mfa_image_compare against the oracle's MSE / PSNR /
SSIM on random images, on the MFA render of a Greville-sampled model against the signal's
render, at the minimum size and on non-multiple-of-tile sizes; its degenerate and invalid
inputs.  Last, the property the comparison exists to show: a finer MFA model of the
signal renders closer to the ground truth.
"""
import math

import numpy as np
import pytest

import synth
from metrics import IMAGE_RMSE_TOL, image_rmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


@pytest.fixture(scope="module")
def quality():
    from oracle import quality as q
    return q


ML_CASES = [
    # camera, W, H, ns, shading, f_m, alpha, tf alpha
    (synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0), 64, 48, 256, True, 6.0, 0.25, 0.06),
    (synth.orbit_camera((0.5, 0.5, 0.5), 2.0, 2.1, -0.5, 45.0), 53, 37, 200, False, 6.0, 0.25, 0.1),
    (synth.camera_ortho((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 1.3), 41, 45, 128, True, 3.0, 0.6, 0.08),
    (synth.orbit_camera((0.5, 0.5, 0.5), 1.9, -0.8, 0.9, 50.0), 33, 29, 97, True, 8.5, 0.0, 0.2),
]


@pytest.mark.parametrize("case", range(len(ML_CASES)))
def test_render_ml_matches_oracle(mfa, orc, case):
    import torch
    cam, W, H, ns, shading, fm, alpha, a = ML_CASES[case]
    table = synth.ramp_tf(256, a)
    tf = mfa.transfer_fn(table, shading=shading)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    g = mfa.render_ml(cam, tf, W, H, ns, f_m=fm, alpha=alpha, samples_out=cnt).cpu().numpy()
    r, rc = orc.render_ml(cam, table, W, H, ns, f_m=fm, alpha=alpha, shading=shading)
    assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL), image_rmse(g, r)
    assert np.abs(g - r).max() <= 5e-2
    assert r[..., 3].max() > 0.3 and (r[..., 3] == 0).any() == (g[..., 3] == 0).any()
    assert abs(int(cnt.item()) - rc) <= max(2, 1e-3 * rc)


def test_render_ml_paper_shape_sampled(mfa, orc):
    """The scalability shape (768^2, 1024 samples per ray) on 2048 seeded pixels."""
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    table = synth.ramp_tf(256, 0.06)
    W = H = 768
    g = mfa.render_ml(cam, mfa.transfer_fn(table, shading=True), W, H, 1024).cpu().numpy().reshape(-1, 4)
    pix = np.random.default_rng(768).choice(W * H, 2048, replace=False)
    r, _ = orc.render_ml(cam, table, W, H, 1024, shading=True, pixels=pix)
    assert np.all(image_rmse(g[pix], r) <= IMAGE_RMSE_TOL), image_rmse(g[pix], r)
    assert r[:, 3].max() > 0.5


def test_render_ml_errors(mfa):
    import torch
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    tf = mfa.transfer_fn(synth.ramp_tf(16, 0.1))
    for fm, alpha in ((-1.0, 0.25), (6.0, -0.5), (math.nan, 0.25), (6.0, math.inf)):
        with pytest.raises(mfa.MfaError):
            mfa.render_ml(cam, tf, 8, 8, 8, f_m=fm, alpha=alpha)
    with pytest.raises(mfa.MfaError):
        mfa.render_ml(cam, tf, 8, 8, 0)
    out = mfa.render_ml(cam, tf, 1, 1, 1)      # one pixel, one sample
    assert torch.isfinite(out).all()


def _dev(img):
    import torch
    return torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()


@pytest.mark.parametrize("H,W", [(11, 11), (37, 53), (128, 96), (300, 211)])
def test_image_compare_matches_oracle(mfa, quality, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    base = rng.uniform(-0.1, 1.1, (H, W, 4)).astype(np.float32)           # includes out-of-range values
    noisy = (base + rng.normal(0, 0.05, base.shape)).astype(np.float32)
    smooth = np.cumsum(rng.uniform(0, 1, (H, W, 4)), axis=1).astype(np.float32) / W
    for a, b in ((base, noisy), (smooth, base), (noisy, noisy * 0.5)):
        got = mfa.image_compare(_dev(a), _dev(b))
        ref = quality.compare(a, b)
        assert got["mse"] == pytest.approx(ref["mse"], rel=1e-12)
        assert got["psnr_db"] == pytest.approx(ref["psnr_db"], rel=1e-12)
        assert got["ssim"] == pytest.approx(ref["ssim"], rel=1e-11, abs=1e-13)
        sym = mfa.image_compare(_dev(b), _dev(a))
        assert sym["ssim"] == pytest.approx(got["ssim"], rel=1e-13) and sym["mse"] == pytest.approx(got["mse"], rel=1e-13)


def test_image_compare_degenerate_and_invalid(mfa):
    import torch
    img = _dev(np.random.default_rng(5).uniform(0, 1, (20, 30, 4)))
    q = mfa.image_compare(img, img)
    assert q["mse"] == 0.0 and q["psnr_db"] == math.inf and q["ssim"] == pytest.approx(1.0, abs=1e-14)
    with pytest.raises(mfa.MfaError):
        mfa.image_compare(img[:10].contiguous(), img[:10].contiguous())       # below the 11 x 11 window
    flat = torch.zeros(20 * 30 * 4 + 1, device="cuda")
    mis = flat[1:].view(20, 30, 4)                                            # 4-byte offset: not 16-byte aligned
    with pytest.raises(mfa.MfaError):
        mfa.image_compare(mis, img)
    with pytest.raises(ValueError):
        mfa.image_compare(img, img[:, :29].contiguous())


def test_mfa_render_against_ground_truth(mfa, orc, quality):
    """Greville-sampled degree-2 models of the signal: the metrics of the MFA render against
    the ground-truth render agree with the oracle's on the same two GPU images, and a finer
    model scores closer (lower MSE, higher PSNR and SSIM)."""
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    table = synth.ramp_tf(256, 0.06)
    tf = mfa.transfer_fn(table, shading=True, vmin=0.0, vmax=1.0)
    W = H = 160
    truth = mfa.render_ml(cam, tf, W, H, 512)
    scores = []
    for n in (24, 48, 96):
        spec = synth.marschner_lobb_model(n, 2)
        model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
        img = mfa.render(model, cam, tf, W, H, 512)
        got = mfa.image_compare(img, truth)
        ref = quality.compare(img.cpu().numpy(), truth.cpu().numpy())
        assert got["mse"] == pytest.approx(ref["mse"], rel=1e-12)
        assert got["ssim"] == pytest.approx(ref["ssim"], rel=1e-11)
        scores.append(got)
        model.close()
    assert scores[0]["mse"] > scores[1]["mse"] > scores[2]["mse"]
    assert scores[0]["ssim"] < scores[1]["ssim"] < scores[2]["ssim"]
    assert math.isfinite(scores[2]["psnr_db"]) and scores[2]["psnr_db"] > 20.0
