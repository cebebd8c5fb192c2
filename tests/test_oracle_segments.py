"""Pins of the oracle's object-space decomposition (CPU only): the volume split into
blocks, each block compositing its segment of every ray, the partial images merged with
over nearest segment first.

The pins: one block is the single-pass render; without early termination any split gives
the single-pass image (associativity of over) and the same samples; with early termination
the image moves by at most 1 - alpha_T per channel and never evaluates fewer samples; the
blocks' sample ranges partition every ray and hold exactly the samples inside the block's
box (brute force); a constant slab split in blocks keeps A = 1 - (1-a)^n.
"""
import numpy as np
import pytest

import synth
from synth import camera_ortho, camera_persp, constant_tf, knots_uniform

CAM = camera_persp((1.9, 1.3, 2.2), (0.5, 0.45, 0.55), (0, 1, 0), 40.0)


def _model(orc, seed, degree=(3, 3, 3), n=(9, 8, 10), uniform=True):
    rng = np.random.default_rng(seed)
    knots = [knots_uniform(n[a], degree[a]) if uniform else synth.knots_nonuniform(n[a], degree[a], rng)
             for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, degree, rng, 0.01)
    return orc.Model(degree, n, knots, P)


def test_one_block_is_the_single_pass_render(orc):
    m = _model(orc, 1)
    tf = synth.ramp_tf(64, 0.2)
    a, na = orc.render(m, CAM, tf, 21, 17, 60, shading=True)
    b, nb = orc.render_segments(m, CAM, tf, 21, 17, 60, (1, 1, 1), shading=True)
    np.testing.assert_array_equal(a, b)
    assert na == nb


@pytest.mark.parametrize("blocks", [(2, 3, 2), (4, 1, 1), (1, 1, 5), (3, 3, 3)])
def test_split_without_termination_equals_single_pass(orc, blocks):
    m = _model(orc, 2, uniform=False)
    tf = synth.ramp_tf(64, 0.15)
    a, na = orc.render(m, CAM, tf, 19, 15, 50, shading=True, ert_alpha=1.0)
    b, nb = orc.render_segments(m, CAM, tf, 19, 15, 50, blocks, shading=True, ert_alpha=1.0)
    assert np.abs(a - b).max() <= 1e-12
    assert na == nb


def test_termination_moves_the_image_by_at_most_one_minus_alpha(orc):
    m = _model(orc, 3)
    tf = synth.ramp_tf(64, 0.6)          # opaque enough that most rays terminate
    a, na = orc.render(m, CAM, tf, 23, 19, 80, shading=False, ert_alpha=0.99)
    b, nb = orc.render_segments(m, CAM, tf, 23, 19, 80, (2, 2, 2), shading=False, ert_alpha=0.99)
    assert a[..., 3].max() >= 0.99                      # termination does happen
    assert np.abs(a - b).max() <= 0.01 + 1e-12
    assert nb >= na


def test_block_ranges_partition_the_ray_and_match_the_boxes(orc):
    rng = np.random.default_rng(4)
    for _ in range(200):
        g = tuple(int(x) for x in rng.integers(1, 5, 3))
        o = rng.uniform(-1.0, 2.0, 3)
        d = synth.random_direction(rng)
        if rng.random() < 0.2:
            d[int(rng.integers(0, 3))] = 0.0             # a ray parallel to one axis's planes
            d = d / np.linalg.norm(d)
            o = rng.uniform(0.0, 1.0, 3)
        t = []
        for a in range(3):
            if d[a] != 0:
                t += [(0 - o[a]) / d[a], (1 - o[a]) / d[a]]
        lo = max(0.0, max(min(t[2 * i], t[2 * i + 1]) for i in range(len(t) // 2)))
        hi = min(max(t[2 * i], t[2 * i + 1]) for i in range(len(t) // 2))
        if not lo < hi or any(d[a] == 0 and not 0 <= o[a] <= 1 for a in range(3)):
            continue
        ns = int(rng.integers(1, 300))
        dt = (hi - lo) / ns
        owner = -np.ones(ns, dtype=int)
        for b in range(g[0] * g[1] * g[2]):
            bi = (b % g[0], (b // g[0]) % g[1], b // (g[0] * g[1]))
            kb, ke = orc.block_range(g, bi, o, d, lo, dt, ns)
            assert 0 <= kb and ke <= ns
            for k in range(kb, ke):
                assert owner[k] < 0                      # no sample in two blocks
                owner[k] = b
                x = o + (lo + (k + 0.5) * dt) * d
                for a in range(3):                       # the sample is in the block's box
                    assert bi[a] / g[a] - 1e-9 <= x[a] <= (bi[a] + 1) / g[a] + 1e-9
        assert (owner >= 0).all()                        # every sample in some block


def test_constant_slab_in_blocks(orc):
    n = 6
    m = orc.Model((3, 3, 3), (n, n, n), [knots_uniform(n, 3)] * 3, np.full((n, n, n), 0.4))
    cam = camera_ortho((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 1.0)
    rgba = np.float32([0.25, 0.5, 0.75, 0.05]).astype(np.float64)
    for ns in (37, 64):
        img, cnt = orc.render_segments(m, cam, constant_tf(rgba), 8, 8, ns, (3, 1, 2), ert_alpha=1.0)
        A = 1 - (1 - rgba[3]) ** ns
        np.testing.assert_allclose(img[..., 3], A, rtol=0, atol=1e-13)
        np.testing.assert_allclose(img[..., :3], np.broadcast_to(rgba[:3] * A, (8, 8, 3)), rtol=0, atol=1e-13)
        assert cnt == 64 * ns


def test_bad_block_grid_is_rejected(orc):
    m = _model(orc, 5)
    with pytest.raises(ValueError):
        orc.render_segments(m, CAM, synth.ramp_tf(4, 0.1), 4, 4, 8, (0, 1, 1))
    with pytest.raises(ValueError):
        orc.render_segments(m, CAM, synth.ramp_tf(4, 0.1), 4, 4, 8, (9, 8, 8))
