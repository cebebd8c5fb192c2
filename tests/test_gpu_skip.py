"""GPU: empty-space skipping (render variant 7).  Where a knot-span cell's value bound maps
only to transfer-function rows of zero opacity its samples are skipped; the image equals variant 6's to FP32 rounding (a zero-opacity sample
composites to exactly nothing; the two kernels may fuse the remaining arithmetic
differently), fewer samples are evaluated, and the image matches the oracle.  Edge cases: no transparent row
(nothing skipped), every row transparent (nothing evaluated), a one-row table; on
non-uniform models variant 7 skips within variant 4's march."""
import zlib

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


def _table(kind):
    t = synth.ramp_tf(128, 0.2).copy()
    if kind == "window":          # transparent below 45 % and above 85 % of the range
        x = np.linspace(0.0, 1.0, len(t))
        t[(x < 0.45) | (x > 0.85), 3] = 0.0
    elif kind == "opaque":        # no transparent row
        t[:, 3] = 0.05 + 0.1 * np.linspace(0.0, 1.0, len(t))
    elif kind == "clear":         # every row transparent
        t[:, 3] = 0.0
    elif kind == "one_row":
        t = np.array([[0.8, 0.6, 0.2, 0.0]], dtype=np.float32)
    return np.ascontiguousarray(t, dtype=np.float32)


def _render(mfa, m, cam, table, variant, W=64, H=48, ns=160):
    import torch
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render(m, cam, mfa.transfer_fn(table, shading=True), W, H, ns, variant=variant, samples_out=cnt)
    return img.cpu().numpy(), int(cnt.item())


CASES = [((3, 3, 3), (26, 22, 24), 1), ((2, 2, 2), (30, 28, 26), 1), ((3, 3, 3), (20, 24, 22), 2)]


@pytest.mark.parametrize("degree,nctrl,storage", CASES)
def test_skip_equals_variant6_and_matches_oracle(mfa, orc, degree, nctrl, storage):
    rng = np.random.default_rng(zlib.crc32(repr((degree, nctrl, storage)).encode()))
    knots = [synth.knots_uniform(nctrl[a], degree[a]) for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, degree, rng, 0.01)
    m = mfa.Model(degree, nctrl, knots, P, storage=storage)
    assert m.info()["cardinal"]
    d = synth.random_direction(rng)
    cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.2 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 40.0)
    table = _table("window")
    i6, c6 = _render(mfa, m, cam, table, 6)
    i7, c7 = _render(mfa, m, cam, table, 7)
    np.testing.assert_allclose(i7, i6, rtol=0, atol=1e-5)   # a skipped visible sample would move >= 1e-2
    assert 0 < c7 < c6
    stored = np.asarray(P, np.float64).astype(np.float32).astype(np.float64) if storage == 1 else orc.round_to_f16(P)
    ref = orc.Model(degree, nctrl, knots, stored)
    r, _ = orc.render(ref, cam, table, 64, 48, 160, shading=True)
    assert np.all(image_rmse(i7, r) <= IMAGE_RMSE_TOL), image_rmse(i7, r)
    assert r[..., 3].max() > 0.05


def test_skip_edge_tables_and_fallback(mfa):
    rng = np.random.default_rng(5)
    nctrl = (18, 20, 16)
    knots = [synth.knots_uniform(n, 3) for n in nctrl]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, (3, 3, 3), rng, 0.01)
    m = mfa.Model((3, 3, 3), nctrl, knots, P)
    cam = synth.camera_persp((1.8, 1.4, 2.1), (0.5, 0.5, 0.5), (0, 1, 0), 36.0)
    i6, c6 = _render(mfa, m, cam, _table("opaque"), 6)
    i7, c7 = _render(mfa, m, cam, _table("opaque"), 7)
    np.testing.assert_allclose(i7, i6, rtol=0, atol=1e-5)
    assert c7 == c6
    i7, c7 = _render(mfa, m, cam, _table("clear"), 7)
    assert c7 == 0 and not i7.any()
    i6, _ = _render(mfa, m, cam, _table("one_row"), 6)
    i7, c7 = _render(mfa, m, cam, _table("one_row"), 7)
    assert c7 == 0 and not i7.any() and not i6.any()
    for storage in (1, 3):        # off the cardinal path, variant 7 skips within variant 4
        nu = [synth.knots_nonuniform(n, 3, rng) for n in nctrl]
        mn = mfa.Model((3, 3, 3), nctrl, nu, P, storage=storage)
        assert not mn.info()["cardinal"]
        i4, c4 = _render(mfa, mn, cam, _table("window"), 4)
        i7, c7 = _render(mfa, mn, cam, _table("window"), 7)
        np.testing.assert_allclose(i7, i4, rtol=0, atol=1e-5)
        assert 0 < c7 < c4


def test_skip_full_size_sampled(mfa, orc):
    """The bench's empty-space row at full size -- the 128^3 model, 1024^2, 1024 samples, a
    transfer function transparent below the median control point -- on 2048 seeded pixels
    against the oracle, and against variant 6 on the whole image."""
    import torch
    wl = synth.config2(with_points=False)
    spec, job = wl.model, wl.render
    m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model.from_spec(spec)
    lo, hi = float(spec.ctrl.min()), float(spec.ctrl.max())
    table = synth.ramp_tf(256, 0.05).copy()
    table[np.linspace(0.0, 1.0, len(table)) < (float(np.median(spec.ctrl)) - lo) / (hi - lo), 3] = 0.0
    W, H, ns = job.width, job.height, job.n_samples
    i6, c6 = _render(mfa, m, job.camera, table, 6, W, H, ns)
    i7, c7 = _render(mfa, m, job.camera, table, 7, W, H, ns)
    # alpha sums that differ in the last bit may cross the 0.99 termination threshold one
    # sample apart: such a pixel moves by at most (1 - 0.99) x the table's largest alpha
    d = np.abs(i7 - i6).max(axis=-1)
    assert d.max() <= 0.01 * 0.05 * 1.2 and (d > 1e-5).mean() < 1e-3, (d.max(), (d > 1e-5).mean())
    assert c7 < 0.5 * c6
    pix = np.random.default_rng(77).choice(W * H, 2048, replace=False)
    r, _ = orc.render(ref, job.camera, table, W, H, ns, shading=True, pixels=pix)
    assert np.all(image_rmse(i7.reshape(-1, 4)[pix], r) <= IMAGE_RMSE_TOL)
    assert r[:, 3].max() > 0.1
