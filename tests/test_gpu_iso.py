"""GPU: isosurface rendering (mfa_render_iso) against the oracle's isosurface on the same
stored control points: the same rays hit, at the same parameter to FP32 resolution, with
the same shaded colour, and every pixel where hit, miss or crossing differ is accounted for
by a near-tie of f - iso at the samples next to the differing crossing (iso_check); a
linear field's plane isosurface at the closed-form parameter."""
import math
import zlib

import numpy as np
import pytest

import iso_check
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


def _stored(P, storage, orc):
    if storage == 1:
        return np.asarray(P, np.float64).astype(np.float32).astype(np.float64)
    return orc.round_to_f16(P) if storage == 2 else orc.round_to_bf16(P)


CASES = [((3, 3, 3), (22, 18, 20), True, 1), ((3, 3, 3), (17, 19, 21), False, 1), ((2, 3, 4), (12, 14, 11), True, 1),
         ((3, 3, 3), (24, 20, 16), True, 2), ((2, 2, 2), (15, 13, 14), False, 3)]


@pytest.mark.parametrize("degree,nctrl,uniform,storage,window",
                         [c + (0,) for c in CASES] + [CASES[0] + (2,), CASES[3] + (2,), CASES[1] + (2,)])
def test_iso_matches_oracle(mfa, orc, degree, nctrl, uniform, storage, window):
    """window 2: compact models, which keep no cell bounds (every sample is queried)."""
    import torch
    rng = np.random.default_rng(zlib.crc32(repr((degree, nctrl, uniform, storage)).encode()))
    knots = [synth.knots_uniform(nctrl[a], degree[a]) if uniform else synth.knots_nonuniform(nctrl[a], degree[a], rng)
             for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, degree, rng, 0.01)
    m = mfa.Model(degree, nctrl, knots, P, storage=storage, window=window)
    stored = _stored(P, storage, orc)
    ref = orc.Model(degree, nctrl, knots, stored)
    iso = float(np.percentile(stored, 65))
    d = synth.random_direction(rng)
    cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.3 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 38.0)
    table = synth.ramp_tf(256, 1.0)
    tf = mfa.transfer_fn(table, shading=True)
    W, H, ns = 48, 36, 64
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img, depth = mfa.render_iso(m, cam, tf, W, H, ns, iso, samples_out=cnt)
    img, depth = img.cpu().numpy(), depth.cpu().numpy()
    r, rd, rq = orc.render_iso(ref, cam, table, W, H, ns, iso, shading=True)
    hg, ho = np.isfinite(depth), np.isfinite(rd)
    assert ho.sum() > 0.1 * W * H                                   # the surface is in view
    bad, ties = iso_check.explain(orc, ref, cam, W, H, ns, iso, depth, rd)
    assert not bad, f"{len(bad)} unexplained disagreements (pixels {bad[:10]}), {ties} near-ties"
    both = hg & ho
    sel = np.zeros_like(both)
    sel[both] = np.abs(depth[both] - rd[both]) <= iso_check.DEPTH_TOL  # the same crossing
    assert sel.sum() >= 0.9 * ho.sum()
    assert np.abs(img[sel] - r[sel]).max() <= 2e-3
    assert np.all(img[~hg] == 0.0) and np.all(img[hg][:, 3] == 1.0)
    assert abs(int(cnt.item()) - rq) <= 0.02 * rq


def test_iso_plane_closed_form(mfa, orc):
    a = np.array([0.7, -0.4, 0.9])
    b = 0.2
    n, deg = (7, 6, 5), (2, 3, 1)
    knots = [synth.knots_uniform(n[i], deg[i]) for i in range(3)]
    g = [synth.greville(knots[i], deg[i]) for i in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    P = a[0] * X + a[1] * Y + a[2] * Z + b
    m = mfa.Model(deg, n, knots, P)
    cam = synth.camera_persp((1.7, 1.2, 2.3), (0.5, 0.5, 0.5), (0, 1, 0), 45.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 1.0), shading=True, vmin=-1.0, vmax=2.0)
    W, H, ns, iso = 40, 30, 50, 0.55
    _, depth = mfa.render_iso(m, cam, tf, W, H, ns, iso)
    depth = depth.cpu().numpy()
    hits = 0
    for row in range(H):
        for col in range(W):
            o, d = orc.ray(cam, W, H, col, row)
            o, d = np.asarray(o), np.asarray(d)
            ok, t0, t1 = orc.clip_unit_box(o, d)
            if not ok:
                assert math.isinf(depth[row, col])
                continue
            dt = (t1 - t0) / ns
            ts = t0 + (np.arange(ns) + 0.5) * dt
            s = np.sign(a @ (o[:, None] + ts[None, :] * d[:, None]) + b - iso)
            crossing = np.any(s[1:] != s[:-1])
            t_star = (iso - b - a @ o) / (a @ d)
            if crossing and min(abs(t_star - ts)) > 1e-5:          # clear of a sample: unambiguous
                hits += 1
                assert abs(depth[row, col] - t_star) <= 2e-5
            elif not crossing and min(abs(t_star - ts[[0, -1]])) > 1e-5:
                assert math.isinf(depth[row, col])
    assert hits > 100


def test_iso_rejects_bad_arguments(mfa):
    m = mfa.Model((3, 3, 3), (8, 8, 8), None, np.zeros((8, 8, 8)))
    cam = synth.camera_persp((1.7, 1.2, 2.3), (0.5, 0.5, 0.5), (0, 1, 0), 45.0)
    tf = mfa.transfer_fn(synth.ramp_tf(8, 1.0))
    with pytest.raises(mfa.MfaError):
        mfa.render_iso(m, cam, tf, 8, 8, 16, float("nan"))
    with pytest.raises(mfa.MfaError):
        mfa.render_iso(m, cam, tf, 8, 8, 0, 0.5)


def test_iso_localised_surface_matches_oracle(mfa, orc):
    """A field that crosses iso only inside one small bump: almost every cell's control
    points lie below iso, so most samples are decided by the cell bounds without a query;
    hits, depths and colours still match the oracle, which queries every sample."""
    import torch
    deg, n = (3, 3, 3), (40, 36, 44)
    knots = [synth.knots_uniform(n[a], deg[a]) for a in range(3)]
    g = [synth.greville(knots[a], deg[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    P = np.exp(-(((X - 0.45) / 0.22) ** 2 + ((Y - 0.55) / 0.2) ** 2 + ((Z - 0.5) / 0.24) ** 2)) - 0.02 * X
    iso = 0.35                                                    # 92 % of the cells lie off iso
    for storage in (1, 2):
        m = mfa.Model(deg, n, knots, P, storage=storage)
        stored = _stored(P, storage, orc)
        ref = orc.Model(deg, n, knots, stored)
        cam = synth.camera_persp((1.6, 1.3, 2.1), (0.5, 0.5, 0.5), (0, 1, 0), 24.0)
        table = synth.ramp_tf(256, 1.0)
        tf = mfa.transfer_fn(table, shading=True, vmin=-0.1, vmax=1.0)
        W, H, ns = 56, 44, 160
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        img, depth = mfa.render_iso(m, cam, tf, W, H, ns, iso, samples_out=cnt)
        img, depth = img.cpu().numpy(), depth.cpu().numpy()
        r, rd, rq = orc.render_iso(ref, cam, table, W, H, ns, iso, shading=True, vmin=-0.1, vmax=1.0)
        hg, ho = np.isfinite(depth), np.isfinite(rd)
        assert 0.05 * W * H < ho.sum() < 0.6 * W * H                 # a small surface in view
        bad, ties = iso_check.explain(orc, ref, cam, W, H, ns, iso, depth, rd)
        assert not bad, f"{len(bad)} unexplained disagreements (pixels {bad[:10]}), {ties} near-ties"
        both = hg & ho
        sel = np.zeros_like(both)
        sel[both] = np.abs(depth[both] - rd[both]) <= iso_check.DEPTH_TOL
        assert sel.sum() >= 0.9 * ho.sum()
        assert np.abs(img[sel] - r[sel]).max() <= 2e-3
        assert abs(int(cnt.item()) - rq) <= 0.02 * rq


def test_iso_full_size_sampled(mfa, orc):
    """The bench's isosurface row at full size -- the 128^3 model, 1024^2, 1024 samples, iso =
    the median control point -- on 2048 seeded pixels against the oracle (which queries every
    sample; the GPU decides most samples by the cell bounds and steps over bounded cells)."""
    import torch
    wl = synth.config2(with_points=False)
    spec, job = wl.model, wl.render
    m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model.from_spec(spec)
    iso = float(np.median(spec.ctrl))
    W, H, ns = job.width, job.height, job.n_samples
    tf = mfa.transfer_fn(job.tf, shading=True)
    img, depth = mfa.render_iso(m, job.camera, tf, W, H, ns, iso)
    img, depth = img.cpu().numpy().reshape(-1, 4), depth.cpu().numpy().reshape(-1)
    pix = np.random.default_rng(1024).choice(W * H, 2048, replace=False)
    r, rd, _ = orc.render_iso(ref, job.camera, job.tf, W, H, ns, iso, shading=True, pixels=pix)
    hg, ho = np.isfinite(depth[pix]), np.isfinite(rd)
    assert ho.mean() > 0.2
    bad, ties = iso_check.explain(orc, ref, job.camera, W, H, ns, iso, depth[pix], rd, pixels=pix)
    print(f"full-size isosurface: {ties} near-tie disagreements of 2048 pixels")
    assert not bad, f"{len(bad)} unexplained disagreements (pixels {pix[bad][:10]}), {ties} near-ties"
    both = hg & ho
    close = np.abs(depth[pix][both] - rd[both]) <= iso_check.DEPTH_TOL
    assert close.mean() >= 0.9
    assert np.abs(img[pix][both][close] - r[both][close]).max() <= 2e-3
