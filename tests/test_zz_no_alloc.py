"""GPU: the allocation-free batched render (mfa_render_batch_static).

Callers that cannot allocate device memory -- a process whose pool already holds the
whole GPU, or a render loop that must not pay cudaMalloc's implicit synchronisation --
use this entry point: its work table sits in a fixed array inside the library instead
of a cudaMalloc'd buffer.  This test calls it through the C ABI twice in a row (the
array keeps the first call's contents, so the second call must rewrite all of it) and
compares every image and sample count with the allocating batched entry point.  It is
collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from metrics import IMAGE_RMSE_TOL, image_rmse

pytestmark = pytest.mark.gpu


def _requests(mfa, rng, n_req):
    import torch
    # (degree, control points, storage, uniform knots): non-uniform knots take the record
    # path, uniform knots with one degree the cardinal path (its own kernels and heads)
    specs = [((3, 3, 3), (20, 18, 22), 1, False), ((2, 2, 2), (14, 16, 12), 2, False),
             ((4, 4, 4), (12, 12, 13), 1, False), ((3, 3, 3), (16, 24, 14), 3, False),
             ((3, 3, 3), (17, 21, 15), 1, True), ((2, 2, 2), (13, 11, 16), 2, True)]
    models = []
    for deg, n, storage, uniform in specs:
        knots = [synth.knots_uniform(n[a], deg[a]) if uniform else synth.knots_nonuniform(n[a], deg[a], rng)
                 for a in range(3)]
        P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 6), knots, deg, rng, 0.01)
        models.append(mfa.Model(deg, n, knots, P, storage=storage))
    reqs = []
    for k in range(n_req):
        d = synth.random_direction(rng)
        cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.4 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 35.0)
        tf = mfa.transfer_fn(synth.ramp_tf(int(rng.choice([16, 256])), 0.1), shading=True)
        W, H = int(rng.integers(8, 70)), int(rng.integers(8, 70))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        reqs.append(mfa.Request(models[k % len(models)], cam, tf, W, H, int(rng.integers(20, 120)), samples_out=cnt))
    return models, reqs


def test_static_batch_matches_allocating_batch_twice():
    import torch
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as mfa
    rng = np.random.default_rng(777)
    for call, n_req in enumerate((13, 7)):          # two calls in a row, the second smaller
        models, reqs = _requests(mfa, rng, n_req)
        assert any(m.info()["cardinal"] for m in models) and not all(m.info()["cardinal"] for m in models)
        arr = mfa._request_array(reqs)
        mfa._bind_stream()
        rc = mfa.lib().mfa_render_batch_static(ctypes.addressof(arr), len(reqs))
        assert rc == 0, mfa.lib().mfa_last_error().decode()
        torch.cuda.synchronize()
        got = [q.out.clone() for q in reqs]
        got_counts = [int(q.samples_out.item()) for q in reqs]
        for q in reqs:
            q.out.fill_(-1.0)
            q.samples_out.zero_()
        mfa.render_batch(reqs)                       # the allocating entry point
        torch.cuda.synchronize()
        for g, q, c in zip(got, reqs, got_counts):
            a, b = g.cpu().numpy(), q.out.cpu().numpy()
            assert np.all(image_rmse(a, b) <= IMAGE_RMSE_TOL), call
            assert np.abs(a - b).max() <= 1e-5, call
            assert c == int(q.samples_out.item()), call


def test_static_batch_rejects_oversize_without_launching():
    import torch
    import paper_2312_15073_gb300 as mfa
    rng = np.random.default_rng(778)
    models, reqs = _requests(mfa, rng, 33)
    for q in reqs:
        q.out.fill_(5.0)
    arr = mfa._request_array(reqs)
    rc = mfa.lib().mfa_render_batch_static(ctypes.addressof(arr), len(reqs))
    assert rc == -1 and "0..32" in mfa.lib().mfa_last_error().decode()
    torch.cuda.synchronize()
    assert all(float(q.out.min()) == 5.0 for q in reqs)


def test_static_batch_refused_under_capture():
    """Under stream capture the call returns MFA_ERR_UNSUPPORTED before enqueueing anything
    (its table copies come from host memory that a replayed graph could not reach), and the
    capture it was called in stays valid: the captured graph replays."""
    import torch
    import paper_2312_15073_gb300 as mfa
    rng = np.random.default_rng(779)
    models, reqs = _requests(mfa, rng, 3)
    for q in reqs:
        q.out.fill_(5.0)
    arr = mfa._request_array(reqs)
    x = torch.zeros(16, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        mfa._bind_stream()
        with torch.cuda.graph(graph, stream=side):
            rc = mfa.lib().mfa_render_batch_static(ctypes.addressof(arr), len(reqs))
            x.add_(1.0)
    torch.cuda.current_stream().wait_stream(side)
    mfa._bind_stream()
    assert rc == -6 and "captured" in mfa.lib().mfa_last_error().decode()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert float(x.min()) == 2.0 and float(x.max()) == 2.0
    assert all(float(q.out.min()) == 5.0 and float(q.out.max()) == 5.0 for q in reqs)
