"""Pins of the oracle's knot-span search and B-spline basis (CPU only).

Each check is something the mathematics fixes independently of the oracle's code:
partition of unity, the derivative sum, non-negativity and local support, textbook
worked values (tests/golden/basis_textbook.txt), the Bernstein closed form, the
full-recursion definition, and a brute-force linear span scan.
"""
import math
import os

import numpy as np
import pytest

from synth import knots_nonuniform, knots_uniform

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "basis_textbook.txt")


def _cases():
    cases, cur = [], None
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "case":
                cur = {"name": vals[0]}
                cases.append(cur)
            elif key in ("knots", "N", "dN"):
                cur[key] = [float(v) for v in vals]
            elif key in ("degree", "span"):
                cur[key] = int(vals[0])
            elif key == "u":
                cur[key] = float(vals[0])
    return cases


def _knot_vectors():
    rng = np.random.default_rng(7)
    out = []
    for p in range(0, 5):
        for n in (p + 1, p + 2, p + 5, 13):
            out.append((knots_uniform(n, p), p))
            out.append((knots_nonuniform(n, p, rng), p))
    # repeated interior knots (a zero-length span inside the domain)
    out.append((np.array([0, 0, 0, 0, 0.3, 0.3, 0.6, 1, 1, 1, 1.0]), 3))
    out.append((np.array([0, 0, 0, 0.5, 0.5, 1, 1, 1.0]), 2))
    return out


def _probe_points(U, p, rng):
    n = len(U) - p - 1
    lo, hi = U[p], U[n]
    pts = list(rng.uniform(lo, hi, 40)) + list(np.unique(U[p:n + 1])) + [lo, hi]
    pts += [np.nextafter(k, -np.inf) for k in U[p + 1:n]] + [np.nextafter(k, np.inf) for k in U[p + 1:n]]
    return [u for u in pts if lo <= u <= hi]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_textbook_values(orc, case):
    s, N, D = orc.basis(case["knots"], case["degree"], case["u"])
    assert s == case["span"]
    np.testing.assert_allclose(N, case["N"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(D, case["dN"], rtol=0, atol=1e-14)


def test_partition_of_unity_and_derivative_sum(orc):
    rng = np.random.default_rng(11)
    for U, p in _knot_vectors():
        scale = 1.0 / np.min(np.diff(np.unique(U)))
        for u in _probe_points(U, p, rng):
            s, N, D = orc.basis(U, p, u)
            assert abs(N.sum() - 1.0) <= 1e-14, (U, p, u)
            assert np.all(N >= -1e-16), (U, p, u)
            assert abs(D.sum()) <= 1e-13 * max(1.0, scale * p), (U, p, u)


def test_span_matches_brute_force_scan(orc):
    rng = np.random.default_rng(12)
    for U, p in _knot_vectors():
        n = len(U) - p - 1
        for u in _probe_points(U, p, rng) + [U[p] - 0.1, U[n] + 0.1]:
            # the largest s in [p, n-1] with U[s] <= u; u at or past the end -> n-1
            want = p
            for s in range(p, n):
                if U[s] <= u:
                    want = s
            assert orc.find_span(U, p, u) == want, (U, p, u)
            if p <= u <= U[n] and want < n - 1:
                assert U[want] <= u < U[want + 1]


def test_span_local_basis_equals_full_recursion(orc):
    """The p+1 span-local values equal the direct recursion N_{i,p}(u) over the whole
    knot vector, and every function outside the span's support is exactly zero."""
    rng = np.random.default_rng(13)
    for U, p in _knot_vectors():
        n = len(U) - p - 1
        for u in _probe_points(U, p, rng)[:25]:
            s, N, D = orc.basis(U, p, u)
            full = np.array([orc.basis_direct(U, p, i, u) for i in range(n)])
            dfull = np.array([orc.basis_direct_deriv(U, p, i, u) for i in range(n)])
            want = np.zeros(n)
            want[s - p:s + 1] = N
            dwant = np.zeros(n)
            dwant[s - p:s + 1] = D
            np.testing.assert_allclose(full, want, rtol=0, atol=1e-14)
            np.testing.assert_allclose(dfull, dwant, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bezier_case_is_bernstein(orc, p):
    """n = p+1 with knots 0^{p+1} 1^{p+1}: N_{i,p}(u) = C(p,i) u^i (1-u)^{p-i} and
    N'_{i,p} = p (B_{i-1,p-1} - B_{i,p-1})."""
    U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])

    def bern(i, k, u):
        if i < 0 or i > k:
            return 0.0
        return math.comb(k, i) * u ** i * (1 - u) ** (k - i)

    for u in np.linspace(0, 1, 17):
        s, N, D = orc.basis(U, p, u)
        assert s == p
        np.testing.assert_allclose(N, [bern(i, p, u) for i in range(p + 1)], rtol=0, atol=1e-15)
        np.testing.assert_allclose(D, [p * (bern(i - 1, p - 1, u) - bern(i, p - 1, u)) for i in range(p + 1)],
                                   rtol=0, atol=1e-14)


def test_uniform_interior_span_is_translation_invariant(orc):
    """On a uniform knot vector every interior span carries the same local cubic
    polynomials (the cardinal B-spline), so values at the same local offset agree."""
    U = knots_uniform(20, 3)
    h = U[4] - U[3]
    ref = None
    for s in range(6, 17):
        u = U[s] + 0.37 * h
        ss, N, D = orc.basis(U, 3, u)
        assert ss == s
        if ref is None:
            ref = (N, D)
        else:
            np.testing.assert_allclose(N, ref[0], atol=1e-14)
            np.testing.assert_allclose(D, ref[1], atol=1e-11)


def test_rounding_helpers(orc):
    """FP64 -> BF16 / FP16 in one round-to-nearest-even step (no detour via FP32)."""
    e = 2.0 ** -8
    cases = {
        1.0 + e: 1.0,                                # exact tie -> even (mantissa 0)
        1.0 + 3 * e: 1.0 + 4 * e,                     # tie between mantissas 1 and 2 -> 2
        1.0 + e + 2.0 ** -40: 1.0 + 2 * e,            # just above the tie -> up
        1.0 + e + 2.0 ** -30: 1.0 + 2 * e,            # FP32 first would round to the tie and then to 1.0
        -(1.0 + e + 2.0 ** -30): -(1.0 + 2 * e),
        0.0: 0.0,
    }
    x = np.array(list(cases.keys()))
    np.testing.assert_array_equal(orc.round_to_bf16(x), np.array(list(cases.values())))
    h = 2.0 ** -11
    x16 = np.array([1.0 + h, 1.0 + h + 2.0 ** -40, 1.0 + 3 * h])
    np.testing.assert_array_equal(orc.round_to_f16(x16), [1.0, 1.0 + 2 * h, 1.0 + 4 * h])
