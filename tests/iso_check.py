"""Accounts for every pixel where a GPU isosurface image and the oracle's disagree.

Both sides march the same n_s midpoint samples along each ray and take the first sample
pair across which f - iso changes sign (Sec. IV-A.4, the isosurface variant of MFA-VV),
then refine the crossing inside that bracket.  The GPU evaluates f in FP32 at FP32 sample
positions, the oracle in FP64 at FP64 positions, so a sample whose value lies within the
GPU's error of iso may fall on the other side of it on the GPU.  Such a near-tie is the
only admissible reason for the two to disagree, and this module checks that it is the
reason for every disagreeing pixel, with the oracle's FP64 values at the samples:

  * a sign change one side sees and the other does not must have a sample next to it with
    |f - iso| <= eps(t) (a near-tie), where
        eps(t) = 1e-5 max|P| + 1e-6 (max|o| + t) |grad f(t)|
    is the FP32 value gate plus the effect of the FP32 sample position (a few ulps of the
    coordinates o + t d) on f;
  * where both find the same bracket but different depths (more than one root inside it),
    the GPU's depth must itself be a root to the same bound, inside the bracket.

A hit at the same crossing (depths within 1e-4) is an agreement; everything else that the
rules above do not cover is returned as unexplained.
"""
import math

import numpy as np

DEPTH_TOL = 1e-4


def _samples(orc, ref, cam, W, H, ns, iso, pixel):
    col, row = pixel % W, pixel // W
    o, d = orc.ray(cam, W, H, col, row)
    ok, t0, t1 = orc.clip_unit_box(o, d)
    if not ok:
        return None
    dt = (t1 - t0) / ns
    ts = t0 + (np.arange(ns) + 0.5) * dt
    g = np.empty(ns)
    gn = np.empty(ns)
    for k, t in enumerate(ts):
        f, grad, _ = ref.eval(o + t * d)
        g[k] = f - iso
        gn[k] = np.linalg.norm(grad)
    return o, d, t0, dt, ts, g, gn


def _eps(pmax, o, t, gnorm):
    return 1e-5 * pmax + 1e-6 * (float(np.max(np.abs(o))) + abs(t)) * gnorm


def explain(orc, ref, cam, W, H, ns, iso, depth_gpu, depth_ref, pixels=None):
    """Indices (into the compared arrays) of disagreeing pixels with no near-tie to explain
    them, and the number of disagreements that were explained.  depth_* hold the hit ray
    parameter or +inf per pixel; pixels maps compared entries to row * W + col (default:
    the whole image)."""
    depth_gpu = np.asarray(depth_gpu, np.float64).reshape(-1)
    depth_ref = np.asarray(depth_ref, np.float64).reshape(-1)
    if pixels is None:
        pixels = np.arange(W * H)
    pmax = float(np.max(np.abs(ref.ctrl)))
    hg, ho = np.isfinite(depth_gpu), np.isfinite(depth_ref)
    gap = np.abs(np.where(hg & ho, depth_gpu, 0.0) - np.where(hg & ho, depth_ref, 0.0))
    differ = (hg != ho) | (hg & ho & ~(gap <= DEPTH_TOL))
    unexplained, explained = [], 0
    for i in np.flatnonzero(differ):
        s = _samples(orc, ref, cam, W, H, ns, iso, int(pixels[i]))
        if s is None:                       # a ray outside the box cannot hit on either side
            unexplained.append(int(i))
            continue
        o, d, t0, dt, ts, g, gn = s
        eps = np.array([_eps(pmax, o, t, n) for t, n in zip(ts, gn)])
        neg = g < 0.0
        # oracle change indices: k >= 1 with a class change between samples k-1 and k, or an
        # exact zero at sample k
        changes = [k for k in range(ns) if g[k] == 0.0 or (k > 0 and neg[k] != neg[k - 1])]

        def near(k):
            lo = max(k - 1, 0)
            return bool(np.any(np.abs(g[lo:k + 1]) <= eps[lo:k + 1]))

        if not hg[i]:                       # GPU miss, oracle hit: every oracle change a near-tie
            ok = all(near(k) for k in changes)
        else:
            tg = depth_gpu[i]
            kr = (tg - t0) / dt - 0.5       # the GPU's bracket: samples ceil(kr) - 1 and ceil(kr)
            cands = sorted({min(max(int(math.ceil(kr + e)), 0), ns - 1) for e in (-1e-3, 0.0, 1e-3)})
            ok = False
            for kg in cands:
                if not ho[i]:               # GPU hit, oracle miss
                    good = near(kg)
                else:
                    ko = changes[0]
                    if kg == ko:            # same bracket, another root inside it
                        f, grad, _ = ref.eval(o + tg * d)
                        inside = ts[max(kg - 1, 0)] - 1e-6 <= tg <= ts[kg] + 1e-6
                        good = inside and abs(f - iso) <= 4.0 * _eps(pmax, o, tg, np.linalg.norm(grad))
                    elif kg < ko:           # the GPU saw an earlier change
                        good = near(kg)
                    else:                   # the GPU passed the oracle's earlier changes
                        good = all(near(k) for k in changes if k < kg) and (kg in changes or near(kg))
                if good:
                    ok = True
                    break
        if ok:
            explained += 1
        else:
            unexplained.append(int(i))
    return unexplained, explained
