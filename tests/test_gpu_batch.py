"""GPU: batched rendering (one graph launch of persistent kernels over many requests).

Each request rendered inside a mixed batch must equal the same request rendered alone
(same per-ray arithmetic, so bitwise equality is the target; the gate is the image
tolerance), and batched images are checked against the FP64 oracle on sampled pixels.
"""
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


def _models(mfa, orc):
    rng = np.random.default_rng(404)
    out = []
    # (degree, nctrl, uniform knots, storage, window): the first model carries per-cell
    # patches (its own kernel group), the second is the same kind on the plain window; the
    # last carries patches on non-uniform knots (the record path's group, as its default)
    specs = [((3, 3, 3), (22, 18, 20), True, 1, 3), ((3, 3, 3), (24, 20, 28), True, 1, 0),
             ((2, 2, 2), (16, 18, 12), False, 1, 0), ((4, 4, 4), (14, 12, 13), True, 1, 0),
             ((3, 3, 3), (30, 26, 22), False, 2, 0), ((2, 3, 4), (12, 15, 18), True, 3, 0),
             ((3, 3, 3), (17, 21, 15), False, 2, 3)]
    for deg, n, uni, storage, window in specs:
        knots = [synth.knots_uniform(n[a], deg[a]) if uni else synth.knots_nonuniform(n[a], deg[a], rng)
                 for a in range(3)]
        P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 8), knots, deg, rng, 0.01)
        m = mfa.Model(deg, n, knots, P, storage=storage, window=window)
        stored = {1: lambda x: x.astype(np.float32).astype(np.float64), 2: orc.round_to_f16,
                  3: orc.round_to_bf16}[storage](P)
        out.append((m, orc.Model(deg, n, knots, stored)))
    return out


def _requests(mfa, models, rng):
    import torch
    reqs, jobs = [], []
    sizes = [(64, 48), (37, 29), (80, 80), (16, 100), (53, 17), (96, 64), (33, 33)]
    for k, (W, H) in enumerate(sizes):
        m, ref = models[k % len(models)]
        d = synth.random_direction(rng)
        cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.3 * d, (0.5, 0.5, 0.5), synth.view_up_for(d),
                                 float(rng.uniform(25, 45)))
        ns = int(rng.integers(40, 160))
        table = synth.ramp_tf(int(rng.choice([2, 64, 256])), float(rng.uniform(0.03, 0.15)))
        tf = mfa.transfer_fn(table, shading=bool(k % 3 != 2))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        reqs.append(mfa.Request(m, cam, tf, W, H, ns, samples_out=cnt))
        jobs.append((m, ref, cam, table, tf, W, H, ns))
    return reqs, jobs


def test_batch_equals_single_renders(mfa, orc):
    import torch
    models = _models(mfa, orc)
    rng = np.random.default_rng(1)
    reqs, jobs = _requests(mfa, models, rng)
    batch = mfa.Batch(16)
    batch.render(reqs)
    torch.cuda.synchronize()
    bitwise = 0
    for q, (m, ref, cam, table, tf, W, H, ns) in zip(reqs, jobs):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        alone = mfa.render(m, cam, tf, W, H, ns, samples_out=cnt)
        torch.cuda.synchronize()
        a, b = alone.cpu().numpy(), q.out.cpu().numpy()
        assert np.all(image_rmse(a, b) <= IMAGE_RMSE_TOL)
        assert np.abs(a - b).max() <= 1e-5
        bitwise += int(np.array_equal(a, b))
        assert int(q.samples_out.item()) == int(cnt.item())
    print(f"{bitwise}/{len(reqs)} requests bitwise identical alone and in the batch")
    assert bitwise == len(reqs)


def test_batch_matches_oracle(mfa, orc):
    import torch
    models = _models(mfa, orc)
    rng = np.random.default_rng(2)
    reqs, jobs = _requests(mfa, models, rng)
    mfa.render_batch(reqs)
    torch.cuda.synchronize()
    for q, (m, ref, cam, table, tf, W, H, ns) in zip(reqs, jobs):
        pix = rng.choice(W * H, min(W * H, 300), replace=False)
        r, _ = orc.render(ref, cam, table, W, H, ns, shading=bool(tf.struct.shading), pixels=pix)
        g = q.out.cpu().numpy().reshape(-1, 4)[pix]
        assert np.all(image_rmse(g, r) <= IMAGE_RMSE_TOL)


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_batch_tile_shapes_and_resubmission(mfa, orc, shape):
    """Every ray-tile shape gives the same images; consecutive submissions through the
    two alternating table slots (and a changed request set) stay correct."""
    import torch
    models = _models(mfa, orc)
    rng = np.random.default_rng(3)
    reqs, jobs = _requests(mfa, models, rng)
    ref_imgs = []
    for (m, ref, cam, table, tf, W, H, ns) in jobs:
        ref_imgs.append(mfa.render(m, cam, tf, W, H, ns).clone())
    batch = mfa.Batch(8)
    batch.configure(tile_shape=shape)
    for rounds in range(3):
        sub = reqs[rounds % 2::1] if rounds < 2 else reqs[:3]
        for q in sub:
            q.out.fill_(-1.0)
        batch.render(sub)
        torch.cuda.synchronize()
        for q in sub:
            k = reqs.index(q)
            assert torch.equal(q.out, ref_imgs[k])


def test_batch_grid_override_and_validation(mfa, orc):
    import torch
    models = _models(mfa, orc)
    rng = np.random.default_rng(4)
    reqs, jobs = _requests(mfa, models, rng)
    batch = mfa.Batch(8)
    batch.configure(tile_shape=0, grid_ctas=7)          # a few CTAs draw all tiles
    batch.render(reqs)
    torch.cuda.synchronize()
    for q, (m, ref, cam, table, tf, W, H, ns) in zip(reqs, jobs):
        assert torch.equal(q.out, mfa.render(m, cam, tf, W, H, ns))
    bad = mfa.Request(reqs[0].model, reqs[0].cam, reqs[0].tf, 8, 8, 0)      # n_samples = 0
    for q in reqs:
        q.out.fill_(3.0)
    with pytest.raises(mfa.MfaError, match="request 2"):
        batch.render(reqs[:2] + [bad])
    torch.cuda.synchronize()
    assert all(float(q.out.min()) == 3.0 for q in reqs[:2])
    with pytest.raises(mfa.MfaError):
        mfa.Batch(8).render(reqs + reqs)                 # more than the capacity


def test_autotuner_render_and_batch(mfa, orc, tmp_path):
    """The tuner measures every variant x tile shape, its choice is looked up by workload
    class (use_tuned), and a tuned render equals the explicit render of that choice."""
    import torch
    models = _models(mfa, orc)
    rng = np.random.default_rng(9)
    reqs, jobs = _requests(mfa, models, rng)
    m, ref, cam, table, tf, W, H, ns = jobs[0]
    best, allr = mfa.tune_render(m, cam, tf, W, H, ns, reps=2)
    n_variants = 6 + int(m.info()["cardinal"]) + int(m.info()["window"] == mfa.MFA_WINDOW_PATCH)
    assert len(allr) == 4 * n_variants and all(r["ms"] > 0 for r in allr)
    assert best["ms"] == min(r["ms"] for r in allr)
    a = mfa.render(m, cam, tf, W, H, ns, use_tuned=True)
    b = mfa.render(m, cam, tf, W, H, ns, variant=best["variant"], tile_shape=best["tile_shape"])
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    path = str(tmp_path / "tune.txt")
    mfa.tune_save(path)
    mfa.tune_load(path)
    batch = mfa.Batch(16)
    bb = mfa.tune_batch(batch, reqs, reps=1)
    assert 0 <= bb["tile_shape"] < 4 and bb["ms"] > 0
    for q in reqs:
        q.out.fill_(-1)
    batch.render(reqs)
    torch.cuda.synchronize()
    for q, (m, ref, cam, table, tf, W, H, ns) in zip(reqs, jobs):
        assert torch.equal(q.out, mfa.render(m, cam, tf, W, H, ns))
