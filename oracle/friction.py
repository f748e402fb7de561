"""Lagged IPC friction, the frictional term of the step's objective.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

The objective (Sec. 3, Eq. fullspace_ipc) carries h^2 D(x, x^n) with
    D_k(x, x^n) = mu lambda_k^n f0(|u_k|)                       (App. A.3)
    f0(y) = int_{eps_v h}^{y} f1(s) ds + eps_v h
    f1(y) = -y^2 / (eps_v h)^2 + 2 y / (eps_v h)   for 0 < y < eps_v h,   1 beyond,
so f0(y) = -y^3 / (3 (eps_v h)^2) + y^2 / (eps_v h) + eps_v h / 3 below eps_v h and
f0(y) = y above: f0 is C^1 with f0' = f1, and f0(0) = eps_v h / 3.

Readings where the paper is silent (lagged quantities are taken at x^n, the
state at the start of the step, for every pair of the static candidate set
at x^n that is within dhat):
  * u_k = T_k^T (r_k(x) - r_k(x^n)), r_k = sum_i w_i X_i the difference of the
    two closest points (PT: point minus its closest point on the triangle;
    EE: closest point on edge a minus closest point on edge b), with the
    closest-point weights w_i fixed at x^n;
  * T_k (3x2): orthonormal basis of the plane normal to n_k = r_k(x^n) / d_k:
    t1 = the coordinate axis least aligned with n (lowest index on ties),
    made orthogonal to n and normalised; t2 = n x t1;
  * lambda_k^n = kappa A_k c_k |b'(d_k)| at x^n: the normal force of the
    barrier term kappa A_k c_k b(d_k) (c_k the edge-edge mollifier, 1 for
    point-triangle);
  * mu (friction coefficient) and eps_v (velocity threshold) are parameters;
    mu = 0 turns the term off.

In the tangent frame the Hessian of D_k is
    mu lambda [ g(y) I + g'(y) u u^T / y ],   g = f1(y) / y,
whose eigenvalues are g(y) > 0 (across u) and f1'(y) >= 0 (along u), so it is
positive semi-definite as it stands and needs no projection.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# the transition functions
# ----------------------------------------------------------------------------
def f0(y, eh):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y >= eh, y, -y ** 3 / (3.0 * eh * eh) + y * y / eh + eh / 3.0)


def f1(y, eh):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y >= eh, 1.0, -y * y / (eh * eh) + 2.0 * y / eh)


def f1_over_y(y, eh):
    """f1(y) / y, finite at y = 0 (limit 2 / eh)."""
    y = np.asarray(y, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        big = 1.0 / y
    return np.where(y >= eh, big, -y / (eh * eh) + 2.0 / eh)


def dg_over_y(y, eh):
    """g'(y) / y with g = f1 / y (multiplies u u^T, which vanishes as y^2)."""
    y = np.asarray(y, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        big = -1.0 / y ** 3
        small = -1.0 / (eh * eh * y)
    out = np.where(y >= eh, big, small)
    return np.where(y > 0.0, out, 0.0)


# ----------------------------------------------------------------------------
# closest points (brute force over the features of the two primitives)
# ----------------------------------------------------------------------------
def _seg_closest(p, a, b):
    """Parameter t in [0, 1] of the point of segment ab closest to p."""
    e = b - a
    ee = float(e @ e)
    if ee == 0.0:
        return 0.0
    return float(np.clip((p - a) @ e / ee, 0.0, 1.0))


def closest_weights(X: np.ndarray, is_ee: bool) -> np.ndarray:
    """Weights w (4,) with r = sum_i w_i X_i the closest-point difference.

    PT (X = [p, t0, t1, t2]): the closest point on the triangle is the
    orthogonal projection when it falls inside, else the best of the three
    edges' closest points.  EE (X = [a0, a1, b0, b1]): the interior solution
    of the two-parameter least-squares problem when both parameters lie in
    [0, 1], compared with the four endpoint-to-segment candidates."""
    if not is_ee:
        p, t0, t1, t2 = X
        cands = []
        e0, e1 = t1 - t0, t2 - t0
        A = np.array([[e0 @ e0, e0 @ e1], [e0 @ e1, e1 @ e1]])
        if abs(np.linalg.det(A)) > 0.0:
            b1, b2 = np.linalg.solve(A, np.array([e0 @ (p - t0), e1 @ (p - t0)]))
            if b1 >= 0.0 and b2 >= 0.0 and b1 + b2 <= 1.0:
                cands.append(np.array([1.0 - b1 - b2, b1, b2]))
        for i, j in ((0, 1), (1, 2), (2, 0)):
            tri = (t0, t1, t2)
            t = _seg_closest(p, tri[i], tri[j])
            bc = np.zeros(3)
            bc[i] += 1.0 - t
            bc[j] += t
            cands.append(bc)
        best = min(cands, key=lambda bc: float(np.sum((p - bc @ np.stack([t0, t1, t2])) ** 2)))
        return np.concatenate([[1.0], -best])
    a0, a1, b0, b1 = X
    da, db, w0 = a1 - a0, b1 - b0, a0 - b0
    cands = []
    A = np.array([[da @ da, -(da @ db)], [-(da @ db), db @ db]])
    if abs(np.linalg.det(A)) > 1e-30 * max(1.0, float(np.abs(A).max()) ** 2):
        s, t = np.linalg.solve(A, np.array([-(da @ w0), db @ w0]))
        if 0.0 <= s <= 1.0 and 0.0 <= t <= 1.0:
            cands.append((s, t))
    for s in (0.0, 1.0):
        cands.append((s, _seg_closest(a0 + s * da, b0, b1)))
    for t in (0.0, 1.0):
        cands.append((_seg_closest(b0 + t * db, a0, a1), t))

    def dist2(st):
        s, t = st
        r = (a0 + s * da) - (b0 + t * db)
        return float(r @ r)
    s, t = min(cands, key=dist2)
    return np.array([1.0 - s, s, -(1.0 - t), -t])


def tangent_basis(n: np.ndarray) -> np.ndarray:
    """(3, 2) orthonormal basis of the plane normal to the unit vector n."""
    k = int(np.argmin(np.abs(n)))
    a = np.zeros(3)
    a[k] = 1.0
    t1 = a - (a @ n) * n
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    return np.stack([t1, t2], axis=1)


# ----------------------------------------------------------------------------
# lagged data and the per-pair term
# ----------------------------------------------------------------------------
def lagged(Xn: np.ndarray, is_ee: np.ndarray, kappa_area: np.ndarray, eps_x: np.ndarray, dhat: float):
    """Per pair at x^n: weights w (n, 4), basis T (n, 3, 2), normal force
    lambda (n,), closest-point difference r_n (n, 3).  Pairs at or beyond
    dhat get lambda = 0."""
    from .distance import barrier_d1, mollifier_arg
    n = Xn.shape[0]
    W = np.zeros((n, 4))
    T = np.zeros((n, 3, 2))
    lam = np.zeros(n)
    rn = np.zeros((n, 3))
    for k in range(n):
        w = closest_weights(Xn[k], bool(is_ee[k]))
        r = w @ Xn[k]
        d = float(np.linalg.norm(r))
        W[k], rn[k] = w, r
        if d <= 0.0 or d >= dhat:
            continue
        T[k] = tangent_basis(r / d)
        c = 1.0
        if is_ee[k]:
            x = float(mollifier_arg(Xn[k:k + 1], 0)[0][0])
            e = float(eps_x[k])
            c = -x * x / (e * e) + 2.0 * x / e if x < e else 1.0
        lam[k] = kappa_area[k] * c * abs(float(barrier_d1(d, dhat)))
    return W, T, lam, rn


def pair_friction(X: np.ndarray, W, T, lam, rn, mu: float, eh: float, order: int = 2):
    """D_k and its derivatives w.r.t. the 12 coordinates of each pair.

    X (n, 4, 3) current positions.  Returns E (n,), G (n, 12), H (n, 12, 12)."""
    n = X.shape[0]
    s = np.einsum("ni,nic->nc", W, X) - rn                  # r(x) - r(x^n)
    u = np.einsum("ncj,nc->nj", T, s)                       # tangent coordinates
    y = np.linalg.norm(u, axis=1)
    ml = mu * lam
    E = ml * f0(y, eh)
    G = H = None
    if order >= 1:
        gu = (ml * f1_over_y(y, eh))[:, None] * u          # dD/du
        gs = np.einsum("ncj,nj->nc", T, gu)                 # dD/ds
        G = (W[:, :, None] * gs[:, None, :]).reshape(n, 12)
    if order >= 2:
        Huu = (ml * f1_over_y(y, eh))[:, None, None] * np.eye(2)[None] \
            + (ml * dg_over_y(y, eh))[:, None, None] * np.einsum("ni,nj->nij", u, u)
        Hss = np.einsum("nai,nij,nbj->nab", T, Huu, T)      # 3x3
        H = np.einsum("ni,nj,nab->niajb", W, W, Hss).reshape(n, 12, 12)
    return E, G, H
