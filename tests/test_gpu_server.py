"""GPU: the render server (admission by HBM budget, requests joining running work), in both
modes: the device work queue drawn by persistent kernels (mode 0) and one launch per
request on priority streams (mode 1).

Each served result must be the same as the request rendered alone (the same per-ray
arithmetic, so bitwise identity is the target; the gate is the image tolerance).  The
failure paths are driven from the host: an image larger than the budget, a full queue,
a wait that runs out, releasing a request that is still on the GPU, cancelling a
queued one.  Nothing here makes the GPU fault or wait without a bound.
"""
import numpy as np
import pytest

import synth
from metrics import IMAGE_RMSE_TOL, SERVED_RMSE_TOL, image_rmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


@pytest.fixture(scope="module")
def models(mfa, orc):
    specs = synth.config5_models(size_scale=0.125)    # the serving models at 1/8 size
    out = []
    for s in specs:
        m = mfa.Model(s.degree, s.nctrl, s.knots, s.ctrl64, storage=mfa.MFA_F16)
        out.append((m, orc.Model(s.degree, s.nctrl, s.knots, orc.round_to_f16(s.ctrl64))))
    return out


def _stream(n, rng, sides=(16, 48, 96, 160), ns=(32, 160)):
    reqs = []
    for k in range(n):
        ph = rng.uniform(0, 2 * np.pi)
        cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.5, ph, rng.uniform(-0.5, 0.5), 30.0)
        reqs.append(dict(model=int(rng.integers(0, 8)), side=int(rng.choice(sides)),
                         ns=int(rng.integers(ns[0], ns[1] + 1)), cam=cam))
    return reqs


MODES = pytest.mark.parametrize("mode", [0, 1], ids=["queue", "streams"])


@MODES
def test_served_results_equal_alone_and_match_oracle(mfa, orc, models, mode):
    import torch
    rng = np.random.default_rng(55)
    table = synth.ramp_tf(256, 0.05)
    tf = mfa.transfer_fn(table, shading=True)
    srv = mfa.Server(hbm_budget_bytes=64 << 20, max_slots=8, priority_levels=4, mode=mode)
    reqs = _stream(24, rng)
    tickets = [srv.submit(models[r["model"]][0], r["cam"], tf, r["side"], r["side"], r["ns"]) for r in reqs]
    bitwise = 0
    for t, r in zip(tickets, reqs):
        lat = srv.wait(t, 60000.0)
        assert lat > 0
        got = srv.result(t)
        torch.cuda.synchronize()
        srv.release(t)
        m, ref = models[r["model"]]
        alone = mfa.render(m, r["cam"], tf, r["side"], r["side"], r["ns"])
        torch.cuda.synchronize()
        a, b = alone.cpu().numpy(), got.cpu().numpy()
        assert np.all(image_rmse(a, b) <= IMAGE_RMSE_TOL)
        bitwise += int(np.array_equal(a, b))
        pix = rng.choice(r["side"] ** 2, min(64, r["side"] ** 2), replace=False)
        o, _ = orc.render(ref, r["cam"], table, r["side"], r["side"], r["ns"], shading=True, pixels=pix)
        assert np.all(image_rmse(b.reshape(-1, 4)[pix], o) <= SERVED_RMSE_TOL)
    st = srv.stats()
    srv.close()
    print(f"{bitwise}/{len(reqs)} served results bitwise identical to the request alone; stats {st}")
    assert bitwise == len(reqs)
    assert st["completed"] == len(reqs) and st["failed"] == 0


@MODES
def test_admission_respects_the_hbm_budget(mfa, models, mode):
    rng = np.random.default_rng(56)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.05), shading=True)
    budget = 3 * 160 * 160 * 16                    # room for three of the largest images
    srv = mfa.Server(hbm_budget_bytes=budget, max_slots=16, priority_levels=2, mode=mode)
    reqs = _stream(20, rng)
    tickets = [srv.submit(models[r["model"]][0], r["cam"], tf, r["side"], r["side"], r["ns"]) for r in reqs]
    for t in tickets:
        srv.wait(t, 60000.0)
        srv.release(t)                             # frees memory for the ones still queued
    st = srv.stats()
    assert st["completed"] == 20
    assert 0 < st["peak_arena_bytes"] <= budget
    with pytest.raises(mfa.MfaError) as e:         # can never fit: rejected at submit
        srv.submit(models[0][0], reqs[0]["cam"], tf, 400, 400, 10)   # 2.56 MB > budget
    assert e.value.code == -2
    srv.close()


@MODES
def test_full_queue_timeout_release_and_cancel(mfa, models, mode):
    rng = np.random.default_rng(57)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.05), shading=True)
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.5, 0.3, 0.2, 30.0)
    srv = mfa.Server(hbm_budget_bytes=256 << 20, max_slots=1, max_queue=2, priority_levels=1, mode=mode)
    big = srv.submit(models[7][0], cam, tf, 2048, 2048, 2048)     # occupies the only slot for a while
    q1 = srv.submit(models[0][0], cam, tf, 32, 32, 64)
    q2 = srv.submit(models[1][0], cam, tf, 32, 32, 64)
    extra, busy = [], 0
    for _ in range(8):                             # the queue holds two: the rest are refused
        try:
            extra.append(srv.submit(models[2][0], cam, tf, 32, 32, 64))
        except mfa.MfaError as e:
            assert e.code == -5
            busy += 1
    assert busy > 0 and srv.stats()["rejected_busy"] == busy
    with pytest.raises(mfa.MfaError) as e:
        srv.wait(big, 0.001)                       # a wait that runs out
    assert e.value.code == -4
    state, _ = srv.poll(big)
    if state == 1:
        with pytest.raises(mfa.MfaError) as e:
            srv.release(big)                       # still on the GPU
        assert e.value.code == -5
    st2, _ = srv.poll(q2)
    if st2 == 0:
        srv.release(q2)                            # cancel while queued
    srv.wait(big, 60000.0)
    srv.wait(q1, 60000.0)
    for t in extra:
        srv.wait(t, 60000.0)
        srv.release(t)
    srv.release(big)
    srv.release(q1)
    assert srv.stats()["failed"] == 0
    srv.close()


def test_server_rejects_bad_config(mfa):
    with pytest.raises(mfa.MfaError):
        mfa.Server(hbm_budget_bytes=16, max_slots=1)
    with pytest.raises(mfa.MfaError):
        mfa.Server(hbm_budget_bytes=1 << 20, max_slots=0)
    with pytest.raises(mfa.MfaError):
        mfa.Server(hbm_budget_bytes=1 << 20, max_slots=4, mode=2)
    with pytest.raises(mfa.MfaError):                # the device queue's list holds 256 records
        mfa.Server(hbm_budget_bytes=1 << 20, max_slots=257, mode=0)


def test_queue_mixes_kernel_groups_and_reuses_records(mfa, orc):
    """The device work queue with requests of several kernel groups at once (FP32 power rows,
    FP16 rows, compact models and models with per-cell patches in FP32 and FP16, uniform
    knots on the cardinal path and non-uniform on the record path, degrees 2 to 4) and more
    requests than records, so every record is
    republished several times: each result equals the request rendered alone, and matches
    the oracle."""
    import torch
    rng = np.random.default_rng(59)
    specs = [((3, 3, 3), (20, 18, 22), 1, True, 0), ((3, 3, 3), (17, 21, 15), 2, True, 0),
             ((2, 2, 2), (14, 16, 12), 1, False, 0), ((4, 4, 4), (12, 12, 13), 3, False, 0),
             ((2, 3, 4), (13, 11, 16), 1, True, 0), ((3, 3, 3), (15, 19, 17), 2, True, 2),
             ((3, 3, 3), (16, 14, 18), 1, False, 2), ((3, 3, 3), (18, 16, 20), 1, True, 3),
             ((3, 3, 3), (14, 17, 15), 2, True, 3)]
    models = []
    for deg, n, storage, uniform, window in specs:
        knots = [synth.knots_uniform(n[a], deg[a]) if uniform else synth.knots_nonuniform(n[a], deg[a], rng)
                 for a in range(3)]
        P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, deg, rng, 0.01)
        m = mfa.Model(deg, n, knots, P, storage=storage, window=window)
        stored = np.asarray(P, np.float64).astype(np.float32).astype(np.float64) if storage == 1 else (
            orc.round_to_f16(P) if storage == 2 else orc.round_to_bf16(P))
        models.append((m, orc.Model(deg, n, knots, stored)))
    table = synth.ramp_tf(64, 0.08)
    tf = mfa.transfer_fn(table, shading=True)
    srv = mfa.Server(hbm_budget_bytes=64 << 20, max_slots=3, mode=0)
    reqs = []
    for k in range(21):
        d = synth.random_direction(rng)
        cam = synth.camera_persp(np.array([0.5, 0.5, 0.5]) + 2.3 * d, (0.5, 0.5, 0.5), synth.view_up_for(d), 35.0)
        reqs.append((k % len(models), cam, int(rng.integers(9, 70)), int(rng.integers(9, 70)), int(rng.integers(16, 96))))
    tickets = [srv.submit(models[i][0], cam, tf, w, h, ns) for i, cam, w, h, ns in reqs]
    for t, (i, cam, w, h, ns) in zip(tickets, reqs):
        srv.wait(t, 60000.0)
        got = srv.result(t).cpu().numpy()
        srv.release(t)
        alone = mfa.render(models[i][0], cam, tf, w, h, ns).cpu().numpy()
        assert np.array_equal(got, alone), (i, w, h, ns)
        pix = rng.choice(w * h, min(48, w * h), replace=False)
        o, _ = orc.render(models[i][1], cam, table, w, h, ns, shading=True, pixels=pix)
        assert np.all(image_rmse(got.reshape(-1, 4)[pix], o) <= IMAGE_RMSE_TOL)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["peak_in_flight"] <= 3


def test_served_full_size_fp16_against_fp64_oracle(mfa, orc):
    """The served FP16 path at full serving size -- a 512x512x256 degree-3 turbulence model
    stored as FP16, a 2048^2 view with 2048 samples per ray -- against the FP64 oracle on the
    unrounded control points: image RMSE <= 2e-3 on 1024 seeded pixels (the served-path
    gate), and the served image equals the same request rendered alone."""
    import torch
    rng = np.random.default_rng(58)
    n = (512, 512, 256)
    knots = [synth.knots_uniform(n[a], 3) for a in range(3)]
    spec = synth.turbulence_model(rng, (3, 3, 3), n, knots, 64, 0.0)
    m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64, storage=mfa.MFA_F16)
    table = synth.ramp_tf(256, 0.05)
    tf = mfa.transfer_fn(table, shading=True)
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.5, 0.9, 0.25, 30.0)
    srv = mfa.Server(hbm_budget_bytes=256 << 20, max_slots=4, priority_levels=2, mode=0)
    t = srv.submit(m, cam, tf, 2048, 2048, 2048)
    srv.wait(t, 120000.0)
    got = srv.result(t).cpu().numpy()
    srv.release(t)
    srv.close()
    alone = mfa.render(m, cam, tf, 2048, 2048, 2048).cpu().numpy()
    assert np.array_equal(got, alone)
    pix = rng.choice(2048 * 2048, 1024, replace=False)
    ref = orc.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64)
    o, _ = orc.render(ref, cam, table, 2048, 2048, 2048, shading=True, vmin=float(m.info()["vmin"]),
                      vmax=float(m.info()["vmax"]), pixels=pix)
    rmse = image_rmse(got.reshape(-1, 4)[pix], o)
    print("served FP16 512x512x256 2048^2 RMSE vs FP64 oracle:", rmse)
    assert np.all(rmse <= SERVED_RMSE_TOL), rmse
    assert o[:, 3].max() > 0.05
