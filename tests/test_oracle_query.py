"""Pins of the oracle's value + gradient query (CPU only).

Checks: degree-1 reduces to textbook trilinear interpolation; exact reproduction of
linear fields from Greville control points (value and gradient); the convex-hull
bound; central finite differences; the derivative-as-lower-degree-spline identity;
the span-local sum against the full sum over every control point on tiny models with
unequal sizes and degrees per axis (a transposed index fails it); clamping and
threading invariance of decode; per span a polynomial of degree p along each axis, with
C^(p-1) continuity and a jump of the p-th derivative at each simple interior knot.
"""
import numpy as np
import pytest

from synth import greville, knots_nonuniform, knots_uniform


def _model(orc, rng, degree, nctrl, uniform=(True, True, True)):
    knots = [knots_uniform(nctrl[a], degree[a]) if uniform[a] else knots_nonuniform(nctrl[a], degree[a], rng)
             for a in range(3)]
    P = rng.normal(size=(nctrl[2], nctrl[1], nctrl[0]))
    return orc.Model(degree, nctrl, knots, P)


def test_degree1_is_trilinear_interpolation(orc):
    rng = np.random.default_rng(21)
    n = (5, 4, 6)
    knots = [knots_uniform(n[a], 1) for a in range(3)]
    P = rng.normal(size=(n[2], n[1], n[0]))
    m = orc.Model((1, 1, 1), n, knots, P)
    for _ in range(200):
        x = rng.uniform(0, 1, 3)
        # textbook trilinear interpolation of the grid with nodes at i/(n-1)
        g = x * (np.array(n) - 1)
        i0 = np.minimum(np.floor(g).astype(int), np.array(n) - 2)
        w = g - i0
        f = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    wt = (w[0] if dx else 1 - w[0]) * (w[1] if dy else 1 - w[1]) * (w[2] if dz else 1 - w[2])
                    f += wt * P[i0[2] + dz, i0[1] + dy, i0[0] + dx]
        val, grad, _ = m.eval(x)
        assert abs(val - f) <= 1e-13


@pytest.mark.parametrize("deg", [(1, 1, 1), (2, 3, 4), (3, 3, 3), (4, 2, 1)])
@pytest.mark.parametrize("uniform", [True, False])
def test_linear_precision_from_greville_points(orc, deg, uniform):
    """P_ijk = a + b xi_i + c eta_j + d zeta_k at Greville abscissae reproduces
    f = a + b x + c y + d z and grad f = (b, c, d) exactly (up to FP64 rounding)."""
    rng = np.random.default_rng(22)
    n = (9, 7, 8)
    knots = [knots_uniform(n[a], deg[a]) if uniform else knots_nonuniform(n[a], deg[a], rng) for a in range(3)]
    xi, eta, zeta = (greville(knots[a], deg[a]) for a in range(3))
    a0, b, c, d = 0.3, 1.7, -2.2, 0.9
    P = a0 + b * xi[None, None, :] + c * eta[None, :, None] + d * zeta[:, None, None]
    m = orc.Model(deg, n, knots, P)
    pts = np.concatenate([rng.uniform(0, 1, (300, 3)), [[0, 0, 0], [1, 1, 1], [1, 0, 0.5]]])
    for x in pts:
        val, grad, _ = m.eval(x)
        assert abs(val - (a0 + b * x[0] + c * x[1] + d * x[2])) <= 1e-13
        np.testing.assert_allclose(grad, [b, c, d], rtol=0, atol=1e-11)


def test_convex_hull_bound(orc):
    rng = np.random.default_rng(23)
    for deg in [(1, 2, 3), (3, 3, 3), (4, 4, 2)]:
        m = _model(orc, rng, deg, (8, 9, 10), (True, False, True))
        lo, hi = m.ctrl.min(), m.ctrl.max()
        pts = rng.uniform(0, 1, (500, 3)).astype(np.float32)
        val, _ = m.decode(pts)
        assert np.all(val >= lo - 1e-13) and np.all(val <= hi + 1e-13)


def test_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(24)
    h = 1e-5
    for deg in [(2, 2, 2), (3, 3, 3), (4, 3, 2)]:
        m = _model(orc, rng, deg, (10, 11, 12), (False, True, False))
        for _ in range(100):
            x = rng.uniform(0.01, 0.99, 3)
            _, g, _ = m.eval(x)
            fd = np.zeros(3)
            for a in range(3):
                e = np.zeros(3)
                e[a] = h
                fd[a] = (m.eval(x + e)[0] - m.eval(x - e)[0]) / (2 * h)
            scale = max(1.0, np.abs(g).max())
            assert np.abs(fd - g).max() <= 1e-6 * scale, (deg, x, g, fd)


def test_derivative_is_lower_degree_spline(orc):
    """d/dx of a degree-p spline in x is the degree-(p-1) spline on U[1:-1] with control
    points p (P_{i+1} - P_i) / (U_{i+p+1} - U_{i+1}); same in y and z."""
    rng = np.random.default_rng(25)
    deg = (3, 2, 4)
    n = (8, 7, 9)
    knots = [knots_nonuniform(n[a], deg[a], rng) for a in range(3)]
    P = rng.normal(size=(n[2], n[1], n[0]))
    m = orc.Model(deg, n, knots, P)
    axes_np = {0: 2, 1: 1, 2: 0}  # model axis -> numpy axis of P[z][y][x]
    for a in range(3):
        p, U = deg[a], knots[a]
        dU = (U[p + 1:p + n[a]] - U[1:n[a]])            # U_{i+p+1} - U_{i+1}, i = 0..n-2
        diff = np.diff(P, axis=axes_np[a])
        shape = [1, 1, 1]
        shape[axes_np[a]] = n[a] - 1
        Q = p * diff / dU.reshape(shape)
        deg2 = list(deg)
        deg2[a] = p - 1
        n2 = list(n)
        n2[a] = n[a] - 1
        knots2 = list(knots)
        knots2[a] = U[1:-1]
        md = orc.Model(tuple(deg2), tuple(n2), knots2, Q)
        for _ in range(100):
            x = rng.uniform(0, 1, 3)
            _, g, _ = m.eval(x)
            fd, _, _ = md.eval(x)
            assert abs(g[a] - fd) <= 1e-11 * max(1.0, abs(fd)), (a, x)


@pytest.mark.parametrize("deg", [(1, 2, 3), (3, 1, 2), (2, 4, 3), (4, 4, 4)])
def test_span_local_sum_equals_full_sum(orc, deg):
    rng = np.random.default_rng(26)
    n = (deg[0] + 3, deg[1] + 2, deg[2] + 4)
    m = _model(orc, rng, deg, n, (False, True, False))
    pts = list(rng.uniform(0, 1, (60, 3))) + [np.zeros(3), np.ones(3)]
    pts += [np.array([m.knots[0][deg[0] + 1], m.knots[1][deg[1] + 1], 0.5])]
    for x in pts:
        v1, g1, _ = m.eval(x)
        v2, g2 = m.eval_direct(x)
        assert abs(v1 - v2) <= 1e-13
        np.testing.assert_allclose(g1, g2, rtol=1e-12, atol=1e-11)


def test_decode_clamps_and_is_thread_invariant(orc):
    rng = np.random.default_rng(27)
    m = _model(orc, rng, (3, 3, 3), (12, 10, 14), (True, False, True))
    pts = rng.uniform(-0.5, 1.5, (4000, 3)).astype(np.float32)
    pts[0] = [np.nan, 0.5, 0.5]
    v1, g1, s1 = m.decode(pts, spans=True, nthreads=1)
    v4, g4, s4 = m.decode(pts, spans=True, nthreads=5)
    np.testing.assert_array_equal(v1, v4)
    np.testing.assert_array_equal(g1, g4)
    np.testing.assert_array_equal(s1, s4)
    cl = np.clip(np.nan_to_num(pts.astype(np.float64), nan=0.0), 0, 1)
    vc, gc, sc = m.decode(cl.astype(np.float32), spans=True, nthreads=2)
    np.testing.assert_array_equal(v1, vc)
    np.testing.assert_array_equal(s1, sc)
    # spans agree with the basis-level search on each axis
    for i in range(0, 4000, 97):
        for a in range(3):
            assert s1[i, a] == orc.find_span(m.knots[a], m.degree[a], float(cl[i, a]))


@pytest.mark.parametrize("deg,uniform", [((3, 3, 3), True), ((3, 3, 3), False), ((2, 4, 3), False)])
def test_polynomial_per_span_and_knot_continuity(orc, deg, uniform):
    """Along each axis the model is, inside one knot span, a polynomial of degree p in u
    (the per-cell patch view of the model), and at a simple interior knot the polynomials
    of the two neighbouring spans agree in value and in the first p-1 derivatives while
    the p-th derivative jumps (C^(p-1) continuity, no more).  A span boundary placed
    off its knot, or a wrong knot difference in a basis factor, breaks one of the three."""
    from numpy.polynomial import polynomial as npp
    rng = np.random.default_rng(27)
    n = (9, 8, 10)
    knots = [knots_uniform(n[a], deg[a]) if uniform else knots_nonuniform(n[a], deg[a], rng) for a in range(3)]
    P = rng.normal(size=(n[2], n[1], n[0]))
    m = orc.Model(deg, n, knots, P)
    tau = np.linspace(0.05, 0.95, 9)                      # inside the span, off its ends

    def fit(x, a, lo, hi):
        """Degree-p fit of u -> f on [lo, hi] in tau = (u - lo)/(hi - lo); the fit residual."""
        f = []
        for t in tau:
            y = x.copy()
            y[a] = lo + t * (hi - lo)
            f.append(m.eval(y)[0])
        c, (res, *_) = npp.polyfit(tau, f, deg[a], full=True)
        return c, float(np.sqrt(res[0] / len(tau))) if len(res) else 0.0

    for a in range(3):
        p, U = deg[a], knots[a]
        for s in range(p + 1, n[a]):                      # interior knot U_s between spans s-1 and s
            x = rng.uniform(0, 1, 3)
            K, hl, hr = U[s], U[s] - U[s - 1], U[s + 1] - U[s]
            cl, rl = fit(x, a, U[s - 1], K)
            cr, rr = fit(x, a, K, U[s + 1])
            scale = max(1.0, np.abs(cl).max(), np.abs(cr).max())
            assert rl <= 1e-12 * scale and rr <= 1e-12 * scale, (a, s, rl, rr)
            # derivatives in u at the knot: left fit at tau = 1, right fit at tau = 0
            h = min(hl, hr)
            dl, dr = [], []
            for j in range(p + 1):
                dl.append(npp.polyval(1.0, npp.polyder(cl, j)) * (h / hl) ** j)
                dr.append(npp.polyval(0.0, npp.polyder(cr, j)) * (h / hr) ** j)
            for j in range(p):
                assert abs(dl[j] - dr[j]) <= 1e-9 * scale, (a, s, j, dl[j], dr[j])
            assert abs(dl[p] - dr[p]) > 1e-6 * scale, (a, s, dl[p], dr[p])
