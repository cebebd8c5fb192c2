"""Pins of the encoding oracle (CPU only): a fit reproduces the control points of data that
are a spline of the same space, reproduces polynomials of the degree, leaves a residual
orthogonal to every basis function (the normal equations), and the adaptive loop never
lets the error grow while it inserts knots and stops within err_max."""
import numpy as np
import pytest

import synth
from oracle import fit as of


def _spline_data(rng, degree, nctrl, m, uniform=False):
    knots = [synth.knots_uniform(nctrl[a], degree[a]) if uniform else synth.knots_nonuniform(nctrl[a], degree[a], rng, 2.0)
             for a in range(3)]
    P = rng.standard_normal((nctrl[2], nctrl[1], nctrl[0]))
    D = of.evaluate_grid(degree, knots, P, (m[2], m[1], m[0]))
    return knots, P, D


@pytest.mark.parametrize("degree,nctrl,m", [((2, 3, 1), (7, 6, 5), (31, 29, 23)), ((3, 3, 3), (6, 5, 7), (25, 21, 33)),
                                            ((4, 1, 2), (8, 3, 4), (41, 9, 17))])
def test_fit_recovers_the_control_points_of_a_spline(degree, nctrl, m):
    rng = np.random.default_rng(sum(nctrl))
    knots, P, D = _spline_data(rng, degree, nctrl, m)
    Q = of.fit(degree, knots, D)
    assert np.abs(Q - P).max() <= 1e-9 * np.abs(P).max()


def test_fit_reproduces_polynomials_of_the_degree():
    degree, nctrl, m = (2, 3, 1), (6, 7, 4), (19, 23, 11)
    rng = np.random.default_rng(3)
    knots = [synth.knots_nonuniform(nctrl[a], degree[a], rng) for a in range(3)]
    w, v, u = np.meshgrid(of.grid_params(m[2]), of.grid_params(m[1]), of.grid_params(m[0]), indexing="ij")
    D = 0.3 + u * u - 0.7 * u * v ** 3 + 1.5 * w * v * v - 0.2 * w
    Q = of.fit(degree, knots, D)
    F = of.evaluate_grid(degree, knots, Q, D.shape)
    assert np.abs(F - D).max() <= 1e-12


def test_fit_residual_satisfies_the_normal_equations():
    degree, nctrl, m = (3, 2, 3), (8, 6, 7), (30, 20, 26)
    rng = np.random.default_rng(4)
    knots = [synth.knots_nonuniform(nctrl[a], degree[a], rng) for a in range(3)]
    D = rng.standard_normal((m[2], m[1], m[0]))
    Q = of.fit(degree, knots, D)
    r = of.evaluate_grid(degree, knots, Q, D.shape) - D
    g = r
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        A = of.collocation(knots[a], degree[a], of.grid_params(D.shape[axis]))
        g = of._apply(A.T, g, axis)                       # (A_z (x) A_y (x) A_x)^T r
    assert np.abs(g).max() <= 1e-10 * np.abs(D).max()
    assert np.abs(r).max() > 0.1                          # a real least-squares residual


def test_adaptive_encoding_error_never_grows_and_meets_the_bound():
    rng = np.random.default_rng(5)
    f = synth.GaussianSum.draw(rng, 4)
    m = (33, 29, 25)
    D = f.grid(of.grid_params(m[0]), of.grid_params(m[1]), of.grid_params(m[2]))
    err = 2e-3 * np.abs(D).max()
    knots, P, hist = of.encode((3, 3, 3), D, err, max_ctrl=(20, 20, 20))
    errs = [h[0] for h in hist]
    assert all(b <= a * (1 + 1e-9) + 1e-15 for a, b in zip(errs, errs[1:]))   # nested spaces
    assert errs[-1] <= err
    assert hist[0][1] == (4, 4, 4) and all(n <= 20 for n in hist[-1][1])
    F = of.evaluate_grid((3, 3, 3), knots, P, D.shape)
    assert np.abs(F - D).max() == pytest.approx(errs[-1])


def test_adaptive_encoding_respects_the_control_point_limit():
    rng = np.random.default_rng(6)
    D = rng.standard_normal((12, 10, 14))                  # noise: never within a tight bound
    knots, P, hist = of.encode((2, 2, 2), D, 1e-6, max_ctrl=(6, 5, 7))
    assert hist[-1][1] == (6, 5, 7)
    assert P.shape == (7, 5, 6)


def test_data_parameters_and_collocation_rows():
    np.testing.assert_array_equal(of.grid_params(5), [0.0, 0.25, 0.5, 0.75, 1.0])
    U = synth.knots_uniform(6, 2)
    A = of.collocation(U, 2, of.grid_params(9))
    np.testing.assert_allclose(A.sum(axis=1), 1.0, atol=1e-15)        # partition of unity per row
    assert A[0, 0] == 1.0 and A[-1, -1] == 1.0                         # clamped ends interpolate
    assert (np.count_nonzero(A, axis=1) <= 3).all()                    # p + 1 functions per row


def test_clamped_uniform_knots():
    # the textbook clamped uniform vector: p + 1 zeros, interior knots i / (n - p), p + 1 ones
    np.testing.assert_array_equal(of.clamped_uniform(7, 3), [0, 0, 0, 0, 0.25, 0.5, 0.75, 1, 1, 1, 1])
    np.testing.assert_array_equal(of.clamped_uniform(3, 2), [0, 0, 0, 1, 1, 1])


def test_adaptive_inserts_only_where_the_error_exceeds_the_bound():
    # f(x) = (1/4 - x)^3 left of 1/4, 0 right of it: C2 at 1/4, so a cubic spline with knots
    # {1/4, 1/2} reproduces it exactly.  The first refinement splits [0, 1] at 1/2; then only
    # the left span exceeds the bound and gets its midpoint 1/4 -- the right span does not.
    m = (65, 5, 4)
    x = of.grid_params(m[0])
    fx = np.where(x < 0.25, (0.25 - x) ** 3, 0.0)
    D = np.broadcast_to(fx[None, None, :], (m[2], m[1], m[0])).copy()
    knots, P, hist = of.encode((3, 1, 1), D, 1e-3)
    kx = knots[0]
    np.testing.assert_allclose(kx[(kx > 0) & (kx < 1)], [0.25, 0.5])
    assert hist[-1][0] <= 1e-12


def test_adaptive_stops_at_the_first_fit_within_the_bound():
    m = (96, 5, 4)
    x = of.grid_params(m[0])
    D = np.broadcast_to(np.exp(-((x - 0.2) / 0.04) ** 2)[None, None, :], (m[2], m[1], m[0])).copy()
    err_max = 0.025
    _, _, hist = of.encode((3, 1, 1), D, err_max)
    assert all(h[0] > err_max for h in hist[:-1]) and hist[-1][0] <= err_max
    assert len(hist) >= 4
