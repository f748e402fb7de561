"""Continuous collision detection (oracle side).

The paper guarantees intersection-free trajectories (Sec. 1, Sec. 2) but does
not name its CCD.  Reading: additive CCD (ACCD, from the codimensional
IPC follow-up work), restated here from its definition:

  * subtract the mean displacement of the pair's four points (a common
    translation does not change their distance) and bound the rate at which
    the distance can shrink: l_p = |q_p| + max_i |q_ti| for point-triangle,
    l_p = max(|q_a0|, |q_a1|) + max(|q_b0|, |q_b1|) for edge-edge;
  * advance conservatively: the first advance (1 - s) d0 / l_p keeps the gap
    above s d0; each later advance 0.9 d / l_p cannot close the gap; stop
    before the first advance that would leave the distance below s d0.

It returns a time of impact t in (0, t_max] such that the pair stays apart on
[0, t].  The exact first-contact time (root of the coplanarity cubic with an
inside test) is provided for testing conservativeness.
"""
from __future__ import annotations

import numpy as np

from .distance import pair_distance


def accd_toi(x0: np.ndarray, p: np.ndarray, is_ee: bool, s: float = 0.1,
             t_max: float = 1.0, max_iter: int = 10000) -> float:
    """x0, p: (4, 3) start positions and displacements of one pair."""
    q = p - p.mean(axis=0)
    nq = np.linalg.norm(q, axis=1)
    if is_ee:
        lp = max(nq[0], nq[1]) + max(nq[2], nq[3])
    else:
        lp = nq[0] + max(nq[1], nq[2], nq[3])
    if lp == 0.0:
        return t_max
    flag = np.array([is_ee])
    d0 = float(pair_distance(x0[None], flag)[0])
    g = s * d0
    t = 0.0
    tl = (1.0 - s) * d0 / lp
    for _ in range(max_iter):
        d = float(pair_distance((x0 + (t + tl) * p)[None], flag)[0])
        if t > 0.0 and d < g:
            return t
        t = t + tl
        if t >= t_max:
            return t_max
        tl = 0.9 * d / lp
    return t


def accd_batch(X0: np.ndarray, P: np.ndarray, is_ee: np.ndarray, s=0.1, t_max=1.0, max_iter=10000):
    """Vectorised ACCD over pairs: X0, P (n, 4, 3).  Same iteration per pair."""
    n = X0.shape[0]
    out = np.full(n, t_max)
    if n == 0:
        return out
    Q = P - P.mean(axis=1, keepdims=True)
    nq = np.linalg.norm(Q, axis=2)
    lp = np.where(is_ee, np.maximum(nq[:, 0], nq[:, 1]) + np.maximum(nq[:, 2], nq[:, 3]),
                  nq[:, 0] + np.max(nq[:, 1:], axis=1))
    act = lp > 0.0
    d0 = pair_distance(X0, is_ee)
    g = s * d0
    t = np.zeros(n)
    tl = np.where(act, (1.0 - s) * d0 / np.where(act, lp, 1.0), 0.0)
    live = act.copy()
    for _ in range(max_iter):
        if not np.any(live):
            break
        r = np.nonzero(live)[0]
        d = pair_distance(X0[r] + (t[r] + tl[r])[:, None, None] * P[r], is_ee[r])
        stop = (t[r] > 0.0) & (d < g[r])
        out[r[stop]] = t[r[stop]]
        live[r[stop]] = False
        go = ~stop
        rr = r[go]
        t[rr] = t[rr] + tl[rr]
        done = t[rr] >= t_max
        out[rr[done]] = t_max
        live[rr[done]] = False
        keep = rr[~done]
        tl[keep] = 0.9 * d[go][~done] / lp[keep]
    out[live] = t[live]
    return out


# ----------------------------------------------------------------------------
# exact first contact (testing aid)
# ----------------------------------------------------------------------------
def _coplanar_roots(x0, p):
    """Roots in [0, 1] of det[x1-x0, x2-x0, x3-x0](t) with x_i(t) = x0_i + t p_i."""
    a = [x0[i] - x0[0] for i in (1, 2, 3)]
    b = [p[i] - p[0] for i in (1, 2, 3)]

    def det_at(t):
        return np.linalg.det(np.stack([a[k] + t * b[k] for k in range(3)]))
    # cubic through 4 samples
    ts = np.array([0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0])
    vals = np.array([det_at(t) for t in ts])
    coef = np.polyfit(ts, vals, 3)
    roots = np.roots(coef)
    real = roots[np.abs(roots.imag) < 1e-9].real
    return np.sort(real[(real >= 0.0) & (real <= 1.0)])


def exact_toi(x0: np.ndarray, p: np.ndarray, is_ee: bool, tol: float = 1e-12) -> float:
    """First t in [0, 1] where the pair touches, 1.0 (no contact) otherwise."""
    for t in _coplanar_roots(x0, p):
        x = x0 + t * p
        d = float(pair_distance(x[None], np.array([is_ee]))[0])
        scale = max(np.abs(x).max(), 1e-30)
        if d <= tol * scale:
            return float(t)
    return 1.0
