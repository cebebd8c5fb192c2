"""GPU: the render with the object-space decomposition (mfa_render_segments) against the
oracle's decomposition on the same stored control points; one block is the single-pass
render bit for bit; without early termination any block grid gives the single-pass image
up to FP32 rounding order and exactly the same samples."""
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


def _seed(*key):
    return zlib.crc32(repr(key).encode())


def _stored(P, storage, orc):
    if storage == 1:
        return np.asarray(P, np.float64).astype(np.float32).astype(np.float64)
    return orc.round_to_f16(P) if storage == 2 else orc.round_to_bf16(P)


def _make(mfa, orc, seed, degree, nctrl, uniform, storage=1):
    rng = np.random.default_rng(seed)
    knots = [synth.knots_uniform(nctrl[a], degree[a]) if uniform else synth.knots_nonuniform(nctrl[a], degree[a], rng)
             for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, degree, rng, 0.01)
    return mfa.Model(degree, nctrl, knots, P, storage=storage), orc.Model(degree, nctrl, knots, _stored(P, storage, orc)), rng


MODELS = [((3, 3, 3), (20, 18, 22), True, 1), ((3, 3, 3), (17, 19, 15), False, 1), ((2, 2, 2), (14, 12, 16), True, 2),
          ((2, 3, 4), (11, 13, 12), False, 3)]


@pytest.mark.parametrize("degree,nctrl,uniform,storage", MODELS)
def test_one_block_is_the_single_pass_render(mfa, orc, degree, nctrl, uniform, storage):
    import torch
    m, _, rng = _make(mfa, orc, _seed("one", degree, nctrl), degree, nctrl, uniform, storage)
    d = synth.random_direction(rng)
    cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.3 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 35.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.2), shading=True)
    for variant in (0, 4):
        c1 = torch.zeros(1, dtype=torch.int64, device="cuda")
        c2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        a = mfa.render(m, cam, tf, 45, 31, 120, samples_out=c1, variant=variant)
        b = mfa.render_segments(m, cam, tf, 45, 31, 120, (1, 1, 1), samples_out=c2, variant=variant)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert int(c1.item()) == int(c2.item())


@pytest.mark.parametrize("blocks", [(2, 2, 2), (3, 1, 2), (1, 4, 1), (4, 4, 4)])
@pytest.mark.parametrize("degree,nctrl,uniform,storage", MODELS)
def test_segments_match_oracle(mfa, orc, degree, nctrl, uniform, storage, blocks):
    import torch
    m, ref, rng = _make(mfa, orc, _seed("seg", degree, nctrl, blocks), degree, nctrl, uniform, storage)
    d = synth.random_direction(rng)
    cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.2 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 38.0)
    table = synth.ramp_tf(256, 0.3)
    tf = mfa.transfer_fn(table, shading=True)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render_segments(m, cam, tf, 40, 28, 150, blocks, samples_out=cnt).cpu().numpy()
    r, rc = orc.render_segments(ref, cam, table, 40, 28, 150, blocks, shading=True)
    assert np.all(image_rmse(img, r) <= IMAGE_RMSE_TOL), image_rmse(img, r)
    assert abs(int(cnt.item()) - rc) <= max(2, 1e-3 * rc)
    assert r[..., 3].max() > 0.5


@pytest.mark.parametrize("blocks", [(2, 2, 2), (1, 3, 5)])
def test_without_termination_equals_single_pass(mfa, orc, blocks):
    import torch
    m, _, rng = _make(mfa, orc, _seed("noert", blocks), (3, 3, 3), (24, 20, 26), True, 1)
    cam = synth.camera_persp((1.8, 1.5, 2.4), (0.5, 0.5, 0.5), (0, 1, 0), 40.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.05), shading=True, ert_alpha=1.0)
    c1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    c2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    a = mfa.render(m, cam, tf, 64, 48, 200, samples_out=c1)
    b = mfa.render_segments(m, cam, tf, 64, 48, 200, blocks, samples_out=c2)
    torch.cuda.synchronize()
    assert float((a - b).abs().max()) <= 1e-5
    assert int(c1.item()) == int(c2.item())


def test_full_size_segments_sampled_pixels(mfa, orc):
    """The 128^3 degree-3 render workload split 2 x 2 x 2: 2048 seeded pixels against the
    oracle's decomposition."""
    import torch
    wl = synth.config2(with_points=False)
    spec, job = wl.model, wl.render
    m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model.from_spec(spec)
    tf = mfa.transfer_fn(job.tf, shading=True)
    img = mfa.render_segments(m, job.camera, tf, job.width, job.height, job.n_samples, (2, 2, 2)).cpu().numpy()
    rng = np.random.default_rng(12)
    pix = rng.choice(job.width * job.height, 2048, replace=False)
    r, _ = orc.render_segments(ref, job.camera, job.tf, job.width, job.height, job.n_samples, (2, 2, 2),
                               shading=True, pixels=pix)
    assert np.all(image_rmse(img.reshape(-1, 4)[pix], r) <= IMAGE_RMSE_TOL)


def test_bad_block_grids_are_rejected(mfa, orc):
    m, _, _ = _make(mfa, orc, 3, (3, 3, 3), (8, 8, 8), True)
    cam = synth.camera_persp((1.8, 1.5, 2.4), (0.5, 0.5, 0.5), (0, 1, 0), 40.0)
    tf = mfa.transfer_fn(synth.ramp_tf(8, 0.1))
    for g in ((0, 1, 1), (8, 8, 2), (65, 1, 1)):
        with pytest.raises(mfa.MfaError):
            mfa.render_segments(m, cam, tf, 8, 8, 8, g)
    with pytest.raises(mfa.MfaError):
        mfa.render_segments(m, cam, tf, 8, 8, 8, (2, 2, 2), variant=5)
