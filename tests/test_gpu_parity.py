"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs.

Gates (FP32 arithmetic): value e_v <= 1e-5, gradient e_g <= 1e-4, image RMSE <= 1e-3 per
channel; knot spans bit-exact.  For FP16 / BF16 storage the gates apply to the KERNEL
error, i.e. against the oracle run on the same rounded control points; the error
against the unrounded FP64 control points is measured and printed, not gated.
"""
import math
import zlib

import numpy as np
import pytest

import synth
from metrics import GRAD_TOL, IMAGE_RMSE_TOL, VALUE_TOL, grad_error, image_rmse, value_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    import torch
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    assert torch.cuda.is_available()
    return m


def _seed(*key) -> int:
    """A seed that is the same in every process (str hashing is randomised)."""
    return zlib.crc32(repr(key).encode())


def _stored(ctrl64, storage, orc):
    """The control-point values a model with this storage type holds, as FP64."""
    if storage == 1:
        return np.asarray(ctrl64, np.float64).astype(np.float32).astype(np.float64)
    if storage == 2:
        return orc.round_to_f16(ctrl64)
    return orc.round_to_bf16(ctrl64)


def _edge_points(knots, rng, n_random):
    """Random points plus corners, the FP32 values nearest every knot (and their FP32
    neighbours), out-of-domain points and a NaN."""
    pts = [rng.uniform(0, 1, (n_random, 3)).astype(np.float32)]
    specials = []
    for a in range(3):
        for kv in np.unique(knots[a]):
            f = np.float32(kv)
            for v in (np.nextafter(f, np.float32(-1)), f, np.nextafter(f, np.float32(2))):
                p = rng.uniform(0, 1, 3).astype(np.float32)
                p[a] = v
                specials.append(p)
    for c in np.array(np.meshgrid([0, 1], [0, 1], [0, 1])).T.reshape(-1, 3):
        specials.append(c.astype(np.float32))
    specials += [np.array([-0.5, 0.3, 1.5], np.float32), np.array([2.0, -1.0, 0.5], np.float32),
                 np.array([np.nan, 0.25, 0.75], np.float32)]
    pts.append(np.stack(specials))
    return np.concatenate(pts)


def _make(mfa, orc, rng, degree, nctrl, uniform, storage=1, field=None, window=0):
    knots = [synth.knots_uniform(nctrl[a], degree[a]) if uniform[a] else synth.knots_nonuniform(nctrl[a], degree[a], rng)
             for a in range(3)]
    if field is None:
        field = synth.GaussianSum.draw(rng, 6)
    P = synth.sample_ctrl(field, knots, degree, rng, 0.01)
    model = mfa.Model(degree, nctrl, knots, P, storage=storage, window=window)
    ref = orc.Model(degree, nctrl, knots, _stored(P, storage, orc))
    return model, ref, P


CASES = [((3, 3, 3), (13, 9, 11), (True, True, True)),
         ((3, 3, 3), (21, 17, 19), (False, False, False)),
         ((1, 1, 1), (7, 5, 6), (True, False, True)),
         ((2, 2, 2), (10, 12, 8), (False, True, False)),
         ((4, 4, 4), (9, 11, 10), (True, False, False)),
         ((2, 3, 4), (8, 9, 12), (False, True, True)),
         ((4, 1, 3), (6, 5, 7), (True, True, False)),
         # uniform knots, one degree: the cardinal path, including models with no interior
         # span (n - p < 2p - 1) and a single span (n = p + 1)
         ((1, 1, 1), (5, 4, 6), (True, True, True)),
         ((2, 2, 2), (3, 7, 12), (True, True, True)),
         ((3, 3, 3), (4, 6, 40), (True, True, True)),
         ((4, 4, 4), (5, 9, 16), (True, True, True))]


@pytest.mark.parametrize("degree,nctrl,uniform", CASES)
@pytest.mark.parametrize("storage", [1, 2, 3], ids=["f32", "f16", "bf16"])
def test_decode_matches_oracle(mfa, orc, degree, nctrl, uniform, storage):
    import torch
    rng = np.random.default_rng(_seed(degree, nctrl, uniform, storage))
    model, ref, P = _make(mfa, orc, rng, degree, nctrl, uniform, storage)
    pts = _edge_points(ref.knots, rng, 5003)
    val, grad = mfa.decode(model, torch.from_numpy(pts).cuda())
    spans = mfa.locate_spans(model, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    v_ref, g_ref, s_ref = ref.decode(pts, spans=True)
    np.testing.assert_array_equal(spans.cpu().numpy(), s_ref)
    ev = value_error(val.cpu().numpy(), v_ref, ref.ctrl)
    eg = grad_error(grad.cpu().numpy(), g_ref)
    assert ev <= VALUE_TOL, ev
    assert eg <= GRAD_TOL, eg
    # values-only call gives the same values
    val2, _ = mfa.decode(model, torch.from_numpy(pts).cuda(), want_grad=False)
    np.testing.assert_array_equal(val2.cpu().numpy(), val.cpu().numpy())


def test_decode_reduced_precision_total_error(mfa, orc):
    """Error of FP16 / BF16 storage against the unrounded FP64 control points (reported)."""
    import torch
    rng = np.random.default_rng(5)
    degree, nctrl = (3, 3, 3), (24, 20, 22)
    knots = [synth.knots_nonuniform(n, 3, rng) for n in nctrl]
    P = synth.sample_ctrl(synth.Turbulence.draw(rng, 64, 1.0, 8.0), knots, degree, rng, 0.0)
    exact = orc.Model(degree, nctrl, knots, P)
    pts = rng.uniform(0, 1, (20000, 3)).astype(np.float32)
    v_ref, g_ref = exact.decode(pts)
    out = {}
    for storage, name in ((1, "f32"), (2, "f16"), (3, "bf16")):
        m = mfa.Model(degree, nctrl, knots, P, storage=storage)
        v, g = mfa.decode(m, torch.from_numpy(pts).cuda())
        out[name] = (value_error(v.cpu().numpy(), v_ref, P), grad_error(g.cpu().numpy(), g_ref))
    print("total error vs FP64 ctrl (value, gradient):", out)
    assert out["f32"][0] <= VALUE_TOL and out["f32"][1] <= GRAD_TOL
    assert out["f32"][0] <= out["f16"][0] <= out["bf16"][0]        # precision ordering


def test_decode_empty_and_ragged(mfa, orc):
    import torch
    rng = np.random.default_rng(6)
    model, ref, _ = _make(mfa, orc, rng, (3, 3, 3), (8, 8, 8), (True, True, True))
    empty = torch.empty((0, 3), device="cuda")
    v, g = mfa.decode(model, empty)
    assert v.numel() == 0 and g.numel() == 0
    for n in (1, 31, 33, 255, 257, 70001):
        pts = rng.uniform(0, 1, (n, 3)).astype(np.float32)
        v, g = mfa.decode(model, torch.from_numpy(pts).cuda())
        vr, gr = ref.decode(pts)
        assert value_error(v.cpu().numpy(), vr, ref.ctrl) <= VALUE_TOL


def test_decode_full_size_128cube_2pow24(mfa, orc):
    """The decode workload at full size: degree 3, 128^3 FP32 control points, 2^24
    uniform points; every point checked against the oracle."""
    import torch
    wl = synth.config2(decode_n=1 << 24)
    spec = wl.model
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model.from_spec(spec)
    pts = wl.decode_points
    v, g = mfa.decode(model, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    vr, gr = ref.decode(pts)
    ev, eg = value_error(v.cpu().numpy(), vr, ref.ctrl), grad_error(g.cpu().numpy(), gr)
    print(f"decode 128^3 2^24: e_v={ev:.3e} e_g={eg:.3e}")
    assert ev <= VALUE_TOL and eg <= GRAD_TOL


def test_cardinal_spans_at_every_knot_128cube(mfa, orc):
    """The bench model (degree 3, 128^3, clamped uniform knots: the cardinal path) at the
    FP32 values nearest every knot and their FP32 neighbours on each axis: the spans the
    decode uses (mfa_locate_spans runs the same device code) equal the oracle's bit for bit,
    and the values and gradients there meet the gates.  The points include cases where the
    rounded product fl32((n - p) u) lands on the wrong side of an integer, so a span taken
    from floor((n - p) u) alone would fail."""
    import torch
    wl = synth.config2(decode_n=1 << 10)
    spec = wl.model
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    assert model.info()["cardinal"]
    ref = orc.Model.from_spec(spec)
    rng = np.random.default_rng(_seed("cardinal-knots-128"))
    pts = _edge_points(ref.knots, rng, 4096)
    spans = mfa.locate_spans(model, torch.from_numpy(pts).cuda())
    v, g = mfa.decode(model, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    vr, gr, sr = ref.decode(pts, spans=True)
    np.testing.assert_array_equal(spans.cpu().numpy(), sr)
    # the rounded product alone misplaces some of these points (so the check has teeth)
    u = np.clip(np.nan_to_num(pts, nan=0.0), 0, 1).astype(np.float32)
    naive = np.empty_like(sr)
    for a in range(3):
        m = spec.nctrl[a] - spec.degree[a]
        naive[:, a] = np.clip(np.floor(u[:, a] * np.float32(m)), 0, m - 1).astype(np.int64) + spec.degree[a]
    assert np.count_nonzero(naive != sr) > 0
    ev, eg = value_error(v.cpu().numpy(), vr, ref.ctrl), grad_error(g.cpu().numpy(), gr)
    assert ev <= VALUE_TOL and eg <= GRAD_TOL, (ev, eg)


# ----------------------------------------------------------------------------------------
# rendering
# ----------------------------------------------------------------------------------------

def _render_both(mfa, orc, model, ref, job, pixels=None, vmin=math.nan, vmax=math.nan):
    import torch
    tf = mfa.transfer_fn(job.tf, shading=job.shading, ka=job.ka, kd=job.kd, ks=job.ks, shininess=job.shininess,
                         ert_alpha=job.ert_alpha, vmin=vmin, vmax=vmax)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render(model, job.camera, tf, job.width, job.height, job.n_samples, samples_out=cnt)
    torch.cuda.synchronize()
    img = img.cpu().numpy().astype(np.float64)
    rimg, rcount = orc.render(ref, job.camera, job.tf, job.width, job.height, job.n_samples, shading=job.shading,
                              ka=job.ka, kd=job.kd, ks=job.ks, shininess=job.shininess, ert_alpha=job.ert_alpha,
                              vmin=vmin, vmax=vmax, pixels=pixels)
    gimg = img.reshape(-1, 4)[pixels] if pixels is not None else img
    return gimg, rimg, int(cnt.item()), rcount


def test_render_small_config_full_image(mfa, orc):
    """Degree 3, 32^3 FP64 control points, ortho 256^2, 128 samples, no shading, ERT
    0.99: every pixel against the oracle."""
    wl = synth.config1()
    spec = wl.model
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64.astype(np.float32).astype(np.float64))
    g, r, gc, rc = _render_both(mfa, orc, model, ref, wl.render)
    rmse = image_rmse(g, r)
    print("config-1 RMSE per channel:", rmse, "max abs:", np.abs(g - r).max(), "samples gpu/oracle:", gc, rc)
    assert np.all(rmse <= IMAGE_RMSE_TOL)
    assert np.abs(g - r).max() <= 5e-3
    assert abs(gc - rc) <= 1e-4 * rc
    assert r[..., 3].max() > 0.5          # the image is not trivially empty


RENDER_CASES = [
    # degree, nctrl, uniform, camera, W, H, ns, shading
    ((3, 3, 3), (16, 12, 14), (True, True, True), "persp", 37, 23, 96, True),
    ((3, 3, 3), (20, 20, 20), (False, False, False), "persp", 64, 48, 200, True),
    ((2, 3, 4), (10, 11, 12), (True, False, True), "ortho_oblique", 33, 41, 64, True),
    ((1, 1, 1), (9, 9, 9), (True, True, True), "persp", 20, 20, 50, False),
    ((4, 4, 4), (12, 10, 11), (False, True, False), "persp_inside", 24, 16, 80, True),
]


def _camera(kind, rng):
    c = (0.5, 0.5, 0.5)
    if kind == "persp":
        d = synth.random_direction(rng)
        return synth.camera_persp(np.array(c) + 2.2 * d, c, synth.view_up_for(d), 35.0)
    if kind == "ortho_oblique":
        return synth.camera_ortho((2.0, 1.4, 2.3), c, (0, 1, 0), 1.6)
    if kind == "ortho_axis":     # rays along -z: two direction components are zero
        return synth.camera_ortho((0.5, 0.5, 2.5), c, (0, 1, 0), 1.2)
    return synth.camera_persp((0.45, 0.55, 0.6), (0.7, 0.2, 0.1), (0, 1, 0), 70.0)   # eye inside the box


@pytest.mark.parametrize("degree,nctrl,uniform,cam,W,H,ns,shading", RENDER_CASES)
def test_render_matches_oracle(mfa, orc, degree, nctrl, uniform, cam, W, H, ns, shading):
    rng = np.random.default_rng(_seed(degree, nctrl, cam))
    model, ref, _ = _make(mfa, orc, rng, degree, nctrl, uniform)
    job = synth.RenderJob(_camera(cam, rng), W, H, ns, synth.ramp_tf(256, 0.08), shading)
    g, r, gc, rc = _render_both(mfa, orc, model, ref, job)
    rmse = image_rmse(g, r)
    assert np.all(rmse <= IMAGE_RMSE_TOL), rmse
    assert abs(gc - rc) <= max(2, 1e-3 * rc)
    assert r[..., 3].max() > 0.05


def test_render_full_size_persp_1024(mfa, orc):
    """The render workload at full size (degree 3, 128^3 FP32, perspective 1024^2, 1024
    samples, Phong): the whole frame on the GPU, 4096 seeded pixels plus two full rows
    through the oracle."""
    wl = synth.config2(with_points=False)
    spec = wl.model
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    ref = orc.Model.from_spec(spec)
    rng = np.random.default_rng(99)
    W, H = wl.render.width, wl.render.height
    pix = np.concatenate([rng.choice(W * H, 4096, replace=False), np.arange(300 * W, 301 * W),
                          np.arange(700 * W, 701 * W)])
    g, r, gc, rc = _render_both(mfa, orc, model, ref, wl.render, pixels=pix)
    rmse = image_rmse(g, r)
    print("1024^2 RMSE per channel:", rmse, "max abs:", np.abs(g - r).max(), "gpu samples:", gc)
    assert np.all(rmse <= IMAGE_RMSE_TOL)
    assert r[:, 3].max() > 0.5


def test_render_constant_density_closed_form(mfa, orc):
    """Constant field and table: A = 1 - (1-a)^n, C = rgb A (no early termination), and
    with termination the stop index k* = ceil(ln(1-alpha_T)/ln(1-a))."""
    import torch
    n = 6
    model = mfa.Model((3, 3, 3), (n, n, n), None, np.full((n, n, n), 0.4))
    cam = synth.camera_ortho((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 1.0)
    rgba = np.float32([0.25, 0.5, 0.75, 0.05]).astype(np.float64)
    for ns, ert in ((64, 1.0), (128, 0.99)):
        tf = mfa.transfer_fn(synth.constant_tf(rgba), ert_alpha=ert)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        img = mfa.render(model, cam, tf, 16, 16, ns, samples_out=cnt).cpu().numpy()
        k = ns if ert >= 1 else math.ceil(math.log(1 - ert) / math.log(1 - rgba[3]))
        A = 1 - (1 - rgba[3]) ** k
        np.testing.assert_allclose(img[..., 3], A, atol=2e-6)
        np.testing.assert_allclose(img[..., :3], np.broadcast_to(rgba[:3] * A, (16, 16, 3)), atol=2e-6)
        assert int(cnt.item()) == 256 * k


def test_render_edge_cases(mfa, orc):
    import torch
    rng = np.random.default_rng(8)
    model, ref, _ = _make(mfa, orc, rng, (3, 3, 3), (10, 10, 10), (True, True, True))
    cam = synth.camera_persp((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 30.0)
    # a camera looking away: every ray misses, nothing is evaluated
    away = synth.camera_persp((0.5, 0.5, 2.5), (0.5, 0.5, 5.0), (0, 1, 0), 30.0)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.1))
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render(model, away, tf, 19, 7, 32, samples_out=cnt)
    assert float(img.abs().max()) == 0.0 and int(cnt.item()) == 0
    # 1x1 image, one sample, one-row table, no termination
    for W, H, ns, table in ((1, 1, 1, synth.ramp_tf(256, 0.1)), (3, 2, 1, synth.constant_tf((1, 0, 0, 0.5), 1)),
                            (5, 3, 7, synth.ramp_tf(2, 0.9))):
        job = synth.RenderJob(cam, W, H, ns, table, True, ert_alpha=1.0)
        g, r, gc, rc = _render_both(mfa, orc, model, ref, job)
        np.testing.assert_allclose(g, r, atol=1e-4)
        assert gc == rc
    # the largest image side and the largest sample count the API accepts
    wide = synth.RenderJob(cam, 32768, 1, 8, synth.ramp_tf(64, 0.3), True)
    g, r, gc, rc = _render_both(mfa, orc, model, ref, wide, pixels=np.arange(0, 32768, 97))
    assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL)
    # (early termination on: with it off, FP32 alpha sums over 2^20 samples of opacity 1e-4
    # lose the increments below half an ulp of the sum -- a limit of FP32 compositing; near
    # the threshold each sample adds ~1e-6, so the FP32 and FP64 sums may cross it a few
    # thousand samples apart, which moves the image by far less than the gate)
    deep = synth.RenderJob(cam, 2, 2, 1 << 20, synth.ramp_tf(64, 1e-4), True)
    g, r, gc, rc = _render_both(mfa, orc, model, ref, deep)
    assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL) and abs(gc - rc) <= 0.05 * rc and rc > 40000
    # rejected arguments leave the output untouched
    out = torch.full((4, 4, 4), 7.0, device="cuda")
    with pytest.raises(mfa.MfaError):
        mfa.render(model, cam, tf, 4, 4, 0, out=out)
    assert float(out.min()) == 7.0


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("degree", [(3, 3, 3), (2, 3, 4), (4, 4, 4)])
def test_render_variants_match_oracle(mfa, orc, variant, degree):
    """Every kernel variant (support cached / records cached / nothing cached) against the
    oracle, on a non-uniform model and a perspective view."""
    import torch
    rng = np.random.default_rng(_seed("variants", degree))
    model, ref, _ = _make(mfa, orc, rng, degree, (14, 12, 13), (False, True, False))
    cam = _camera("persp", rng)
    job = synth.RenderJob(cam, 40, 24, 120, synth.ramp_tf(256, 0.08), True)
    tf = mfa.transfer_fn(job.tf, shading=True)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render(model, cam, tf, job.width, job.height, job.n_samples, samples_out=cnt, variant=variant)
    torch.cuda.synchronize()
    rimg, rc = orc.render(ref, cam, job.tf, job.width, job.height, job.n_samples, shading=True)
    rmse = image_rmse(img.cpu().numpy(), rimg)
    assert np.all(rmse <= IMAGE_RMSE_TOL), rmse
    assert abs(int(cnt.item()) - rc) <= max(2, 1e-3 * rc)
    assert rimg[..., 3].max() > 0.05


CARDINAL_CASES = [
    ((1, 1, 1), (9, 7, 8), "persp"),
    ((2, 2, 2), (3, 7, 12), "ortho_axis"),
    ((3, 3, 3), (4, 6, 40), "persp_inside"),
    ((3, 3, 3), (24, 20, 28), "persp"),
    ((3, 3, 3), (33, 17, 9), "ortho_axis"),
    ((4, 4, 4), (5, 9, 16), "ortho_oblique"),
    ((4, 4, 4), (18, 14, 12), "persp"),
]


@pytest.mark.parametrize("storage", [1, 2, 3], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("degree,nctrl,cam", CARDINAL_CASES)
def test_render_cardinal_matches_oracle(mfa, orc, degree, nctrl, cam, storage):
    """Variant 6 (uniform knots: interior spans on the cardinal basis, the p-1 end spans of
    each axis from their records) against the oracle, including models with no interior
    span, axis-aligned rays whose positions sit on knots, and an eye inside the box; and
    against the record path (variant 4) on the same model."""
    import torch
    rng = np.random.default_rng(_seed("cardinal", degree, nctrl, cam, storage))
    model, ref, _ = _make(mfa, orc, rng, degree, nctrl, (True, True, True), storage)
    assert model.info()["cardinal"]
    camera = _camera(cam, rng)
    job = synth.RenderJob(camera, 40, 28, 150, synth.ramp_tf(256, 0.08), True)
    tf = mfa.transfer_fn(job.tf, shading=True)
    imgs, counts = {}, {}
    for variant in (6, 4, 0):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        imgs[variant] = mfa.render(model, camera, tf, job.width, job.height, job.n_samples, samples_out=cnt,
                                   variant=variant).cpu().numpy()
        counts[variant] = int(cnt.item())
    np.testing.assert_array_equal(imgs[0], imgs[6])          # the default on a cardinal model
    rimg, rc = orc.render(ref, camera, job.tf, job.width, job.height, job.n_samples, shading=True)
    rmse = image_rmse(imgs[6], rimg)
    assert np.all(rmse <= IMAGE_RMSE_TOL), rmse
    assert abs(counts[6] - rc) <= max(2, 1e-3 * rc)
    assert rimg[..., 3].max() > 0.05
    assert np.abs(imgs[6] - imgs[4]).max() <= 2e-3


PATCH_CASES = [
    ((4, 6, 40), "persp_inside", (True, True, True)),   # no interior span on two axes
    ((24, 20, 28), "persp", (True, True, True)),
    ((33, 17, 9), "ortho_axis", (True, True, True)),    # rays along -z, positions on knots
    ((16, 12, 14), "ortho_oblique", (True, True, True)),
    ((22, 18, 20), "persp", (False, False, False)),     # non-uniform knots: spans from the records
    ((15, 19, 13), "persp_inside", (False, True, False)),
]


@pytest.mark.parametrize("storage", [1, 2], ids=["f32", "f16"])
@pytest.mark.parametrize("nctrl,cam,uniform", PATCH_CASES)
def test_render_patches_match_oracle(mfa, orc, nctrl, cam, uniform, storage):
    """Variant 8 (MFA_WINDOW_PATCH: each knot-span cell's tricubic polynomial, evaluated with
    monomials) against the oracle on the stored values, on uniform knots (cardinal spans) and
    non-uniform ones (spans from the records); the patch model's variant 6 equals the same
    stored values' FP32-window model bit for bit (the window is the same; off the cardinal
    path both run variant 4), variant 8 on a model without patches runs the default, and
    the default takes the patches on uniform knots only."""
    import torch
    rng = np.random.default_rng(_seed("patch", nctrl, cam, uniform, storage))
    model, ref, P = _make(mfa, orc, rng, (3, 3, 3), nctrl, uniform, storage, window=mfa.MFA_WINDOW_PATCH)
    plain = mfa.Model((3, 3, 3), nctrl, [np.asarray(k) for k in ref.knots], P, storage=storage,
                      window=mfa.MFA_WINDOW_F32 if storage != 1 else mfa.MFA_WINDOW_AUTO)
    assert model.info()["window"] == mfa.MFA_WINDOW_PATCH and model.info()["cardinal"] == all(uniform)
    assert model.info()["device_bytes"] > plain.info()["device_bytes"] + 250 * np.prod(np.subtract(nctrl, 3))
    camera = _camera(cam, rng)
    job = synth.RenderJob(camera, 40, 28, 150, synth.ramp_tf(256, 0.08), True)
    tf = mfa.transfer_fn(job.tf, shading=True)
    imgs, counts = {}, {}
    for name, m, variant in (("patch", model, 8), ("win", model, 6), ("plain6", plain, 6), ("plain8", plain, 8),
                             ("default", model, 0)):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        imgs[name] = mfa.render(m, camera, tf, job.width, job.height, job.n_samples, samples_out=cnt,
                                variant=variant).cpu().numpy()
        counts[name] = int(cnt.item())
    np.testing.assert_array_equal(imgs["win"], imgs["plain6"])
    np.testing.assert_array_equal(imgs["plain8"], imgs["plain6"])
    # the default takes the patches on the cardinal path only (as the batch kernels do)
    np.testing.assert_array_equal(imgs["default"], imgs["patch" if all(uniform) else "plain6"])
    rimg, rc = orc.render(ref, camera, job.tf, job.width, job.height, job.n_samples, shading=True)
    rmse = image_rmse(imgs["patch"], rimg)
    assert np.all(rmse <= IMAGE_RMSE_TOL), rmse
    assert abs(counts["patch"] - rc) <= max(2, 1e-3 * rc)
    assert rimg[..., 3].max() > 0.05
    assert np.abs(imgs["patch"] - imgs["win"]).max() <= 2e-3


def test_render_patches_full_size_persp_1024(mfa, orc):
    """The render workload at full size with per-cell patches (variant 8): 4096 seeded pixels
    and two full rows against the oracle."""
    import torch
    wl = synth.config2(with_points=False)
    spec = wl.model
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl, window=mfa.MFA_WINDOW_PATCH)
    ref = orc.Model.from_spec(spec)
    rng = np.random.default_rng(98)
    W, H, job = wl.render.width, wl.render.height, wl.render
    pix = np.concatenate([rng.choice(W * H, 4096, replace=False), np.arange(300 * W, 301 * W),
                          np.arange(700 * W, 701 * W)])
    tf = mfa.transfer_fn(job.tf, shading=job.shading, ka=job.ka, kd=job.kd, ks=job.ks, shininess=job.shininess,
                         ert_alpha=job.ert_alpha)
    img = mfa.render(model, job.camera, tf, W, H, job.n_samples, variant=8).cpu().numpy().astype(np.float64)
    r, _ = orc.render(ref, job.camera, job.tf, W, H, job.n_samples, shading=job.shading, ka=job.ka, kd=job.kd,
                      ks=job.ks, shininess=job.shininess, ert_alpha=job.ert_alpha, pixels=pix)
    rmse = image_rmse(img.reshape(-1, 4)[pix], r)
    print("1024^2 patches RMSE per channel:", rmse)
    assert np.all(rmse <= IMAGE_RMSE_TOL)
    assert r[:, 3].max() > 0.5


def test_cardinal_flag(mfa, orc):
    """Which models take the cardinal path: exactly the clamped uniform knots (i/(n-p) in
    FP64) and one degree; knots off by even 1e-13 take the record path."""
    rng = np.random.default_rng(31)
    P = rng.standard_normal((9, 8, 7))
    n = (7, 8, 9)
    uni = [synth.knots_uniform(n[a], 3) for a in range(3)]
    assert mfa.Model((3, 3, 3), n, None, P).info()["cardinal"]
    assert mfa.Model((3, 3, 3), n, uni, P).info()["cardinal"]
    near = [k.copy() for k in uni]
    near[1][5] += 1e-13
    assert not mfa.Model((3, 3, 3), n, near, P).info()["cardinal"]
    off = [k.copy() for k in uni]
    off[1][5] += 1e-7
    assert not mfa.Model((3, 3, 3), n, off, P).info()["cardinal"]
    assert not mfa.Model((2, 3, 3), n, None, P).info()["cardinal"]
    nonu = [synth.knots_nonuniform(n[a], 3, rng) for a in range(3)]
    assert not mfa.Model((3, 3, 3), n, nonu, P).info()["cardinal"]


def _random_config(seed):
    rng = np.random.default_rng(seed)
    degree = tuple(int(d) for d in rng.integers(1, 5, 3)) if rng.random() < 0.5 else (int(rng.integers(1, 5)),) * 3
    nctrl = tuple(int(degree[a] + 1 + rng.integers(0, 36)) for a in range(3))
    uniform = tuple(bool(u) for u in rng.random(3) < 0.6)
    storage = int(rng.integers(1, 4))
    return rng, degree, nctrl, uniform, storage


@pytest.mark.parametrize("seed", range(16))
def test_random_models_against_oracle(mfa, orc, seed):
    """Seeded random models -- degrees 1-4 (mixed per axis or not), 2 to 40 control points
    per axis, uniform and non-uniform knots per axis, every storage type -- decoded at random
    and edge points and rendered from a random perspective view, against the oracle on the
    same stored control points."""
    import torch
    rng, degree, nctrl, uniform, storage = _random_config(1000 + seed)
    model, ref, _ = _make(mfa, orc, rng, degree, nctrl, uniform, storage)
    pts = _edge_points(ref.knots, rng, 3000)
    val, grad = mfa.decode(model, torch.from_numpy(pts).cuda())
    v_ref, g_ref = ref.decode(pts)
    assert value_error(val.cpu().numpy(), v_ref, ref.ctrl) <= VALUE_TOL
    assert grad_error(grad.cpu().numpy(), g_ref) <= GRAD_TOL
    cam = _camera("persp", rng)
    job = synth.RenderJob(cam, 29, 21, int(rng.integers(16, 200)), synth.ramp_tf(256, 0.1), bool(seed % 2))
    g, r, gc, rc = _render_both(mfa, orc, model, ref, job)
    assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL), (degree, nctrl, uniform, storage)
    assert abs(gc - rc) <= max(2, 1e-3 * rc)


def test_render_marschner_lobb(mfa, orc):
    """The Marschner-Lobb signal (degree 2, Greville-sampled): a small model's full image,
    and the paper's scalability shape -- 256^3 control points, 768^2, 1024 samples -- on
    2048 seeded pixels, against the oracle."""
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    table = synth.ramp_tf(256, 0.06)
    for n, W, H, ns, pixels in ((40, 64, 48, 256, None), (256, 768, 768, 1024, 2048)):
        spec = synth.marschner_lobb_model(n, 2)
        model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
        ref = orc.Model.from_spec(spec)
        pix = None if pixels is None else np.random.default_rng(n).choice(W * H, pixels, replace=False)
        job = synth.RenderJob(cam, W, H, ns, table, True)
        g, r, gc, rc = _render_both(mfa, orc, model, ref, job, pixels=pix)
        assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL), (n, image_rmse(g, r))
        assert r[..., 3].max() > 0.5
        if pix is None:
            assert abs(gc - rc) <= max(2, 1e-3 * rc)


@pytest.mark.parametrize("storage", [2, 3], ids=["f16", "bf16"])
@pytest.mark.parametrize("uniform", [True, False], ids=["uniform", "nonuniform"])
def test_f32_window_of_a_16bit_model(mfa, orc, storage, uniform):
    """A 16-bit model with FP32 window values (MFA_WINDOW_F32) computes exactly what an FP32
    model of the same (16-bit) control-point values computes: decodes and renders are equal
    bit for bit, and meet the gates against the oracle on the rounded values."""
    import torch
    rng = np.random.default_rng(_seed("f32-window", storage, uniform))
    degree, nctrl = (3, 3, 3), (19, 15, 17)
    knots = [synth.knots_uniform(n, 3) if uniform else synth.knots_nonuniform(n, 3, rng) for n in nctrl]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, degree, rng, 0.01)
    stored = _stored(P, storage, orc)
    m16 = mfa.Model(degree, nctrl, knots, P, storage=storage, window=mfa.MFA_WINDOW_F32)
    m32 = mfa.Model(degree, nctrl, knots, stored, storage=mfa.MFA_F32)
    i16 = m16.info()
    assert i16["storage"] == storage and i16["window"] == mfa.MFA_WINDOW_F32 and i16["cardinal"] == uniform
    ref = orc.Model(degree, nctrl, knots, stored)
    pts = _edge_points(ref.knots, rng, 3001)
    v16, g16 = mfa.decode(m16, torch.from_numpy(pts).cuda())
    v32, g32 = mfa.decode(m32, torch.from_numpy(pts).cuda())
    assert torch.equal(v16, v32) and torch.equal(g16, g32)
    vr, gr = ref.decode(pts)
    assert value_error(v16.cpu().numpy(), vr, stored) <= VALUE_TOL
    assert grad_error(g16.cpu().numpy(), gr) <= GRAD_TOL
    cam = synth.camera_persp((1.9, 1.4, 2.2), (0.5, 0.5, 0.5), (0, 1, 0), 35.0)
    table = synth.ramp_tf(256, 0.1)
    tf = mfa.transfer_fn(table, shading=True)
    a = mfa.render(m16, cam, tf, 41, 29, 90)
    b = mfa.render(m32, cam, tf, 41, 29, 90)
    assert torch.equal(a, b)
    o, _ = orc.render(ref, cam, table, 41, 29, 90, shading=True)
    assert np.all(image_rmse(a.cpu().numpy(), o) <= IMAGE_RMSE_TOL)
    assert np.array_equal(m16.ctrl(), m16.ctrl()) and m16.ctrl().dtype == (np.float16 if storage == 2 else np.uint16)


# ----------------------------------------------------------------------------------------
# the compact layout (MFA_WINDOW_COMPACT): the plain array for FP32 (two loads per support
# row); entries of eight control points every 8 - degree positions of a row for 16-bit
# types (1.6x the plain array at degree 3, one load per support row)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("degree,nctrl,uniform", CASES)
@pytest.mark.parametrize("storage", [1, 2, 3], ids=["f32", "f16", "bf16"])
def test_compact_decode_matches_oracle(mfa, orc, degree, nctrl, uniform, storage):
    """Decodes of a compact model against the oracle on the stored values (spans bit-exact,
    value and gradient gates); 16-bit compact models equal the 16-bit layer-pair window's
    results bit for bit (the same values enter the same sums), and every model reads back
    its stored control points."""
    import torch
    rng = np.random.default_rng(_seed("compact", degree, nctrl, uniform, storage))
    model, ref, P = _make(mfa, orc, rng, degree, nctrl, uniform, storage, window=mfa.MFA_WINDOW_COMPACT)
    assert model.info()["window"] == mfa.MFA_WINDOW_COMPACT
    pts = _edge_points(ref.knots, rng, 3001)
    val, grad = mfa.decode(model, torch.from_numpy(pts).cuda())
    spans = mfa.locate_spans(model, torch.from_numpy(pts).cuda())
    v_ref, g_ref, s_ref = ref.decode(pts, spans=True)
    np.testing.assert_array_equal(spans.cpu().numpy(), s_ref)
    assert value_error(val.cpu().numpy(), v_ref, ref.ctrl) <= VALUE_TOL
    assert grad_error(grad.cpu().numpy(), g_ref) <= GRAD_TOL
    pairs = mfa.Model(degree, nctrl, [np.asarray(k) for k in ref.knots], P, storage=storage)
    if storage != 1:
        v2, g2 = mfa.decode(pairs, torch.from_numpy(pts).cuda())
        assert torch.equal(v2, val) and torch.equal(g2, grad)
    assert np.array_equal(model.ctrl(), pairs.ctrl())


@pytest.mark.parametrize("degree,nctrl,uniform,cam,W,H,ns,shading", RENDER_CASES)
@pytest.mark.parametrize("storage", [1, 2], ids=["f32", "f16"])
def test_compact_render_matches_oracle(mfa, orc, degree, nctrl, uniform, cam, W, H, ns, shading, storage):
    rng = np.random.default_rng(_seed("compact-render", degree, nctrl, cam, storage))
    model, ref, _ = _make(mfa, orc, rng, degree, nctrl, uniform, storage, window=mfa.MFA_WINDOW_COMPACT)
    if storage != 1:
        ref = orc.Model(ref.degree, ref.nctrl, ref.knots, _stored(ref.ctrl, storage, orc))
    job = synth.RenderJob(_camera(cam, rng), W, H, ns, synth.ramp_tf(256, 0.08), shading)
    g, r, gc, rc = _render_both(mfa, orc, model, ref, job)
    assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL)
    assert abs(gc - rc) <= max(2, 1e-3 * rc)


def test_compact_fp16_device_bytes(mfa):
    """A compact FP16 model holds at most 2.5x its plain FP16 bytes on the device (its entries
    of eight values, 1.6x the padded array at degree 3, and the per-axis tables), against
    about 8x for its layer-pair window."""
    rng = np.random.default_rng(61)
    n = (96, 80, 72)
    P = rng.standard_normal(n[::-1])
    raw = 2 * np.prod(n)
    compact = mfa.Model((3, 3, 3), n, None, P, storage=mfa.MFA_F16, window=mfa.MFA_WINDOW_COMPACT)
    pairs = mfa.Model((3, 3, 3), n, None, P, storage=mfa.MFA_F16)
    print("device bytes / raw FP16 bytes: compact", compact.info()["device_bytes"] / raw, "pairs",
          pairs.info()["device_bytes"] / raw)
    assert compact.info()["device_bytes"] <= 2.5 * raw
    assert pairs.info()["device_bytes"] >= 6 * raw
