"""Pins of the oracle's isosurface rendering (CPU only).

A linear field (exactly reproduced from Greville-point control points) has a plane as its
isosurface: every ray whose samples straddle the plane hits it at the closed-form
parameter, Newton on a linear g lands on it in one step, and the shaded colour follows from
the plane's normal in closed form; rays whose samples stay on one side miss.  On a random
field, brute force over the samples confirms the first-crossing rule, and the refined point
lies in its bracket with g within rounding of 0.
"""
import math

import numpy as np
import pytest

import synth
from synth import camera_persp, greville, knots_uniform

CAM = camera_persp((1.7, 1.2, 2.3), (0.5, 0.5, 0.5), (0, 1, 0), 45.0)


def _linear(orc, coef, degree=(2, 3, 1), n=(7, 6, 5), uniform=(True, False, True), seed=1):
    rng = np.random.default_rng(seed)
    knots = [knots_uniform(n[a], degree[a]) if uniform[a] else synth.knots_nonuniform(n[a], degree[a], rng)
             for a in range(3)]
    g = [greville(knots[a], degree[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    P = coef[0] * X + coef[1] * Y + coef[2] * Z + coef[3]
    return orc.Model(degree, n, knots, P)


def _ray(orc, W, H, col, row):
    o, d = orc.ray(CAM, W, H, col, row)
    return np.asarray(o), np.asarray(d)


def test_plane_isosurface_closed_form(orc):
    a = np.array([0.7, -0.4, 0.9])
    b = 0.2
    m = _linear(orc, (a[0], a[1], a[2], b))
    iso = 0.55
    W, H, ns = 23, 17, 40
    tf = synth.ramp_tf(256, 1.0)
    rgba, depth, _ = orc.render_iso(m, CAM, tf, W, H, ns, iso, shading=True, vmin=-1.0, vmax=2.0)
    hits = 0
    for row in range(H):
        for col in range(W):
            o, d = _ray(orc, W, H, col, row)
            ok, t0, t1 = orc.clip_unit_box(o, d)
            if not ok:
                assert math.isinf(depth[row, col]) and rgba[row, col].max() == 0.0
                continue
            dt = (t1 - t0) / ns
            g = lambda t: a @ (o + t * d) + b - iso
            ts = t0 + (np.arange(ns) + 0.5) * dt
            s = np.sign([g(t) for t in ts])
            crossing = np.any(s[1:] != s[:-1])
            if not crossing:
                assert math.isinf(depth[row, col]) and rgba[row, col].max() == 0.0
                continue
            hits += 1
            t_star = (iso - b - a @ o) / (a @ d)
            assert abs(depth[row, col] - t_star) <= 1e-12
            n = a / np.linalg.norm(a)
            ndl = abs(n @ -d)
            rv = 2 * ndl * ndl - 1
            spec = max(rv, 0.0) ** 32.0 if rv > 0 else 0.0
            c = np.array([np.interp((iso + 1.0) / 3.0, np.linspace(0, 1, 256), tf[:, ch].astype(np.float64))
                          for ch in range(3)])
            want = np.clip(c * (0.3 + 0.6 * ndl) + 0.3 * spec, 0, 1)
            np.testing.assert_allclose(rgba[row, col, :3], want, atol=1e-12)
            assert rgba[row, col, 3] == 1.0
    assert hits > 20


def test_first_crossing_and_refinement_on_a_random_field(orc):
    rng = np.random.default_rng(7)
    n, deg = (9, 8, 10), (3, 3, 3)
    knots = [knots_uniform(n[a], 3) for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, deg, rng, 0.0)
    m = orc.Model(deg, n, knots, P)
    iso = float(np.percentile(P, 60))
    W, H, ns = 15, 13, 50
    rgba, depth, nq = orc.render_iso(m, CAM, synth.ramp_tf(64, 1.0), W, H, ns, iso)
    hits = 0
    for row in range(H):
        for col in range(W):
            o, d = _ray(orc, W, H, col, row)
            ok, t0, t1 = orc.clip_unit_box(o, d)
            if not ok:
                continue
            dt = (t1 - t0) / ns
            ts = t0 + (np.arange(ns) + 0.5) * dt
            f = m.decode((o + ts[:, None] * d).astype(np.float64), grad=False)[0] - iso
            sgn = f < 0
            change = np.nonzero(sgn[1:] != sgn[:-1])[0]
            if len(change) == 0 and not np.any(f == 0):
                assert math.isinf(depth[row, col])
                continue
            hits += 1
            k = change[0] + 1
            t = depth[row, col]
            assert ts[k - 1] <= t <= ts[k]                      # inside the first bracket
            g = m.eval(o + t * d)[0] - iso
            assert abs(g) <= 1e-9 * (P.max() - P.min())          # converged
    assert hits > 10 and nq > 0


def test_plane_seen_from_behind_uses_the_two_sided_normal(orc):
    """The same plane as the level set of the negated field: the gradient now faces away
    from the eye, and two-sided shading must give the same colours."""
    a = np.array([0.7, -0.4, 0.9])
    b = 0.2
    iso = 0.55
    W, H, ns = 21, 15, 40
    tf = synth.ramp_tf(256, 1.0)
    up = _linear(orc, (a[0], a[1], a[2], b))
    down = _linear(orc, (-a[0], -a[1], -a[2], -b))
    r1, d1, _ = orc.render_iso(up, CAM, tf, W, H, ns, iso, vmin=-1.0, vmax=2.0)
    r2, d2, _ = orc.render_iso(down, CAM, tf, W, H, ns, -iso, vmin=-2.1, vmax=0.9)   # same table position
    hit = np.isfinite(d1)
    assert hit.sum() > 20
    np.testing.assert_array_equal(np.isfinite(d2), hit)
    np.testing.assert_allclose(d2[hit], d1[hit], atol=1e-12)
    np.testing.assert_allclose(r2[hit][:, :3], r1[hit][:, :3], atol=1e-12)


def test_refinement_converges_through_a_sharp_step(orc):
    """A smooth step in x (control points 0 then 1) crossed by coarsely sampled rays: from
    the first bracket's midpoint on the step's shoulder a Newton step leaves the bracket;
    the bracketed refinement still lands on the crossing within its eight steps."""
    n, deg = (24, 4, 4), (3, 3, 3)
    knots = [knots_uniform(n[a], 3) for a in range(3)]
    P = np.zeros((n[2], n[1], n[0]))
    P[:, :, n[0] // 2:] = 1.0
    m = orc.Model(deg, n, knots, P)
    cam = camera_persp((-1.5, 0.55, 0.45), (1.0, 0.5, 0.5), (0, 1, 0), 25.0)
    W, H = 9, 7
    # 12 samples: converged to rounding; 5 samples (a bracket about 0.2 wide): the eight
    # bracketed steps still bring g below 1e-2
    for ns, tol in ((12, 1e-9), (5, 1e-2)):
        rgba, depth, _ = orc.render_iso(m, cam, synth.ramp_tf(8, 1.0), W, H, ns, 0.5)
        hit = np.isfinite(depth)
        assert hit.sum() > 10
        for row in range(H):
            for col in range(W):
                if not hit[row, col]:
                    continue
                o, d = orc.ray(cam, W, H, col, row)
                assert abs(m.eval(np.asarray(o) + depth[row, col] * np.asarray(d))[0] - 0.5) <= tol


def test_iso_check_accounts_only_for_near_ties(orc):
    """The checker the GPU isosurface tests use (tests/iso_check.py): the oracle against
    itself has nothing to explain; planted disagreements far from any near-tie -- a hit
    turned into a miss, a hit moved to another bracket, a miss turned into a hit -- are all
    reported; a disagreement at a crossing whose sample sits on iso is explained."""
    import iso_check
    rng = np.random.default_rng(23)
    deg, n = (3, 3, 3), (12, 11, 13)
    knots = [knots_uniform(n[a], deg[a]) for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, deg, rng, 0.01)
    m = orc.Model(deg, n, knots, P)
    W, H, ns = 20, 16, 40
    iso = float(np.percentile(P, 60))
    table = synth.ramp_tf(16, 1.0)
    _, depth, _ = orc.render_iso(m, CAM, table, W, H, ns, iso)
    depth = depth.reshape(-1)
    bad, ties = iso_check.explain(orc, m, CAM, W, H, ns, iso, depth, depth)
    assert bad == [] and ties == 0

    # pixels whose every sample is far from iso (no near-tie anywhere on the ray)
    pmax = float(np.abs(P).max())
    clear_hit, clear_miss = [], []
    for p in range(W * H):
        s = iso_check._samples(orc, m, CAM, W, H, ns, iso, p)
        if s is None or np.min(np.abs(s[5])) < 1e-3 * pmax:
            continue
        (clear_hit if np.isfinite(depth[p]) else clear_miss).append(p)
    assert len(clear_hit) >= 3 and len(clear_miss) >= 1
    planted = depth.copy()
    planted[clear_hit[0]] = np.inf                                      # hit -> miss
    o, d = orc.ray(CAM, W, H, clear_hit[1] % W, clear_hit[1] // W)
    _, t0, t1 = orc.clip_unit_box(o, d)
    planted[clear_hit[1]] = t1 - 0.25 * (t1 - t0) / ns                  # hit -> last bracket
    o, d = orc.ray(CAM, W, H, clear_miss[0] % W, clear_miss[0] // W)
    _, t0, t1 = orc.clip_unit_box(o, d)
    planted[clear_miss[0]] = 0.5 * (t0 + t1)                            # miss -> hit
    bad, ties = iso_check.explain(orc, m, CAM, W, H, ns, iso, planted, depth)
    assert sorted(bad) == sorted([clear_hit[0], clear_hit[1], clear_miss[0]]) and ties == 0

    # iso placed exactly on one sample's value: that crossing is a near-tie
    p = clear_hit[2]
    s = iso_check._samples(orc, m, CAM, W, H, ns, iso, p)
    k = int(np.flatnonzero(np.sign(s[5][1:]) != np.sign(s[5][:-1]))[0]) + 1
    iso2 = iso + s[5][k]
    _, depth2, _ = orc.render_iso(m, CAM, table, W, H, ns, iso2)
    depth2 = depth2.reshape(-1)
    assert np.isfinite(depth2[p])
    missed = depth2.copy()
    missed[p] = np.inf
    bad, ties = iso_check.explain(orc, m, CAM, W, H, ns, iso2, missed, depth2)
    assert bad == [] and ties == 1
