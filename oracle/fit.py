"""Oracle for MFA encoding -- TEST INFRASTRUCTURE ONLY (tests, the smoke check and the
benchmark's CPU baseline may load it; the GPU library never does).

The paper builds each MFA model before rendering by fitting a tensor-product B-spline to
the block's regular grid of values and refining its knots where the fit misses a maximum
error (the encoding step, Sec. III-A and Sec. IV-A.2).  Plain FP64 NumPy, written from
those definitions:

  * data D[k][j][i] at the uniform parameters u_i = i / (m_x - 1) (likewise v_j, w_k);
  * the least-squares fit minimises sum (f(u_i, v_j, w_k) - D[k][j][i])^2 over the control
    points.  With collocation matrices A_x[i][c] = N_c(u_i) (and A_y, A_z) of full column
    rank, the minimiser is P = (A_z^+ (x) A_y^+ (x) A_x^+) D, i.e. a least-squares solve
    along x for every line, then along y, then along z (np.linalg.lstsq is the solve);
  * the adaptive encoding starts from the fewest control points (p + 1 per axis), fits,
    and while the largest error exceeds err_max inserts, on every axis, a knot at the
    middle of each knot span whose data (the error projected by its maximum over the other
    two axes) exceed err_max -- leftmost spans first where the axis would pass its
    control-point limit -- then refits, stopping once the error is within err_max, or no
    axis can take another knot (a span holding fewer than two data parameters, or the axis
    at its limit).  Inserting knots only enlarges the spline space, so
    the error never grows from one iteration to the next.
"""
import numpy as np

from . import basis


def grid_params(m: int) -> np.ndarray:
    """The m uniform parameters of a data axis (m >= 2)."""
    return np.arange(m, dtype=np.float64) / (m - 1)


def collocation(U, p: int, u: np.ndarray) -> np.ndarray:
    """A[i][c] = N_c(u_i): the len(u) x n matrix of the basis at the parameters."""
    U = np.asarray(U, dtype=np.float64)
    n = len(U) - p - 1
    A = np.zeros((len(u), n))
    for i, x in enumerate(u):
        s, N, _ = basis(U, p, x)
        A[i, s - p:s + 1] = N
    return A


def _apply(M: np.ndarray, X: np.ndarray, axis: int) -> np.ndarray:
    """M applied along `axis` of X (axis 0 = z, 1 = y, 2 = x)."""
    return np.moveaxis(np.tensordot(M, X, axes=([1], [axis])), 0, axis)


def _solve(A: np.ndarray, X: np.ndarray, axis: int) -> np.ndarray:
    """Least-squares solve A Y = X along `axis` for every line."""
    Xm = np.moveaxis(X, axis, 0)
    shape = Xm.shape
    Y, *_ = np.linalg.lstsq(A, Xm.reshape(shape[0], -1), rcond=None)
    return np.moveaxis(Y.reshape((A.shape[1],) + shape[1:]), 0, axis)


def fit(degree, knots, data) -> np.ndarray:
    """Control points [n_z][n_y][n_x] of the least-squares fit to data[m_z][m_y][m_x]."""
    D = np.asarray(data, dtype=np.float64)
    P = D
    for a, axis in ((0, 2), (1, 1), (2, 0)):   # x, then y, then z
        A = collocation(knots[a], degree[a], grid_params(D.shape[axis]))
        P = _solve(A, P, axis)
    return P


def evaluate_grid(degree, knots, P, shape) -> np.ndarray:
    """The model's values at the data grid of the given (m_z, m_y, m_x) shape."""
    F = np.asarray(P, dtype=np.float64)
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        F = _apply(collocation(knots[a], degree[a], grid_params(shape[axis])), F, axis)
    return F


def clamped_uniform(n: int, p: int) -> np.ndarray:
    interior = np.arange(1, n - p, dtype=np.float64) / (n - p)
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)])


def encode(degree, data, err_max: float, max_ctrl=None, max_iter: int = 64):
    """Adaptive encoding.  Returns (knots[3], P, history) with history a list of
    (max error, (n_x, n_y, n_z)) per fit."""
    D = np.asarray(data, dtype=np.float64)
    m = (D.shape[2], D.shape[1], D.shape[0])                  # data points per axis x, y, z
    limit = tuple(max_ctrl) if max_ctrl is not None else m
    knots = [clamped_uniform(degree[a] + 1, degree[a]) for a in range(3)]
    history = []
    P = None
    for _ in range(max_iter):
        P = fit(degree, knots, D)
        E = np.abs(evaluate_grid(degree, knots, P, D.shape) - D)
        emax = float(E.max())
        history.append((emax, tuple(len(knots[a]) - degree[a] - 1 for a in range(3))))
        if emax <= err_max:
            break
        inserted = False
        for a, axis in ((0, 2), (1, 1), (2, 0)):
            other = tuple(x for x in (0, 1, 2) if x != axis)
            proj = E.max(axis=other)                          # error per data parameter on this axis
            u = grid_params(m[a])
            U = knots[a]
            p = degree[a]
            n = len(U) - p - 1
            new = []
            for s in range(p, n):                             # the axis's knot spans
                lo, hi = U[s], U[s + 1]
                inside = (u >= lo) & ((u < hi) | ((s == n - 1) & (u <= hi)))
                if inside.sum() >= 2 and proj[inside].max() > err_max:
                    new.append(0.5 * (lo + hi))
            room = limit[a] - n
            new = new[:max(room, 0)]
            if new:
                knots[a] = np.sort(np.concatenate([U, new]))
                inserted = True
        if not inserted:
            break
    return knots, P, history
