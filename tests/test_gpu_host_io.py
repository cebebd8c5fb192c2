"""GPU: the host-buffer entry points (mfa_decode_host, mfa_render_host) give the same bits as
the device-buffer calls they stage (same kernels, same inputs), across the decode's chunk
boundaries, for page-locked and pageable buffers, and when a render and a decode run at the
same time on two streams."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CHUNK = 1 << 21   # points per pipelined chunk of mfa_decode_host


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


def _model(mfa, uniform, storage, seed):
    rng = np.random.default_rng(seed)
    deg, n = (3, 3, 3), (22, 19, 25)
    knots = [synth.knots_uniform(n[a], 3) if uniform else synth.knots_nonuniform(n[a], 3, rng) for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, deg, rng, 0.01)
    return mfa.Model(deg, n, knots, P, storage=storage)


@pytest.mark.parametrize("uniform,storage", [(True, 1), (False, 2)])
def test_decode_host_equals_device(mfa, uniform, storage):
    import torch
    m = _model(mfa, uniform, storage, 71)
    rng = np.random.default_rng(72)
    for n in (1, 1000, CHUNK - 1, CHUNK, CHUNK + 1, 3 * CHUNK + 17):
        pts = torch.from_numpy(rng.uniform(-0.05, 1.05, (n, 3)).astype(np.float32))
        v_dev, g_dev = mfa.decode(m, pts.cuda())
        for pinned in (True, False):
            p = pts.pin_memory() if pinned else pts.clone()
            v, g = mfa.decode_host(m, p)
            assert torch.equal(v, v_dev.cpu()) and torch.equal(g, g_dev.cpu()), (n, pinned)
    pts = torch.from_numpy(rng.uniform(0, 1, (CHUNK + 3, 3)).astype(np.float32)).pin_memory()
    v, g = mfa.decode_host(m, pts, want_grad=False)
    assert g is None and torch.equal(v, mfa.decode(m, pts.cuda())[0].cpu())
    empty = torch.empty((0, 3), dtype=torch.float32)
    v, g = mfa.decode_host(m, empty)
    assert v.numel() == 0


def test_render_host_equals_device(mfa):
    import torch
    m = _model(mfa, True, 1, 73)
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.4, 0.3, 35.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.08), shading=True)
    for variant, (W, H) in ((0, (97, 61)), (4, (64, 64)), (6, (33, 150))):
        c_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        c_host = torch.zeros(1, dtype=torch.int64, device="cuda")
        img = mfa.render(m, cam, tf, W, H, 120, samples_out=c_dev, variant=variant)
        himg = mfa.render_host(m, cam, tf, W, H, 120, samples_out=c_host, variant=variant)
        assert not himg.is_cuda and torch.equal(himg, img.cpu())
        assert int(c_dev.item()) == int(c_host.item()) > 0
    pageable = torch.empty((40, 30, 4), dtype=torch.float32)
    mfa.render_host(m, cam, tf, 30, 40, 64, out=pageable)
    assert torch.equal(pageable, mfa.render(m, cam, tf, 30, 40, 64).cpu())
    with pytest.raises(mfa.MfaError):
        mfa.render_host(m, cam, tf, 30, 40, 0, out=pageable)          # n_samples = 0


def test_host_calls_overlap_on_two_streams(mfa):
    """A render and a decode enqueued without synchronising, on two streams, give the same
    results as run one after the other."""
    import torch
    m = _model(mfa, True, 1, 74)
    rng = np.random.default_rng(75)
    pts = torch.from_numpy(rng.uniform(0, 1, (2 * CHUNK + 5, 3)).astype(np.float32)).pin_memory()
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 1.1, -0.2, 35.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.08), shading=True)
    ref_img = mfa.render(m, cam, tf, 256, 192, 256).cpu()
    ref_v, ref_g = mfa.decode(m, pts.cuda())
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(sa):
            img = mfa.render_host(m, cam, tf, 256, 192, 256, sync=False)
        with torch.cuda.stream(sb):
            v, g = mfa.decode_host(m, pts, sync=False)
        sa.synchronize()
        sb.synchronize()
        assert torch.equal(img, ref_img)
        assert torch.equal(v, ref_v.cpu()) and torch.equal(g, ref_g.cpu())
