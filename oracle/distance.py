"""Primitive distances, distance-type classification and the IPC barrier.

Barrier (App. A.3, Eq. ipc_energy):
    b(d) = -(d - dhat)^2 ln(d / dhat)   for 0 < d < dhat,   0 otherwise,
with d the unsquared Euclidean distance (reading: the paper prints d, not d^2).

Pairs (App. A.3): point-triangle (PT) and edge-edge (EE).  The distance of a
pair is the exact minimum over the two primitives; which closed form applies
(point-point, point-edge, point-plane, line-line) is decided by where the
closest points lie.  The squared-distance closed forms are differentiated
symbolically with sympy, so gradients and Hessians here follow from the
definitions with no hand algebra:
    PP: |p - q|^2
    PE: |(p - e0) x (e1 - e0)|^2 / |e1 - e0|^2
    PT: ((p - t0) . n)^2 / |n|^2,        n = (t1 - t0) x (t2 - t0)
    EE: ((a0 - b0) . n)^2 / |n|^2,       n = (a1 - a0) x (b1 - b0)
Edge-edge pairs are multiplied by the IPC mollifier of |(a1-a0) x (b1-b0)|^2
with threshold eps_x = c |a0bar a1bar|^2 |b0bar b1bar|^2 (rest lengths), which
keeps the energy smooth for near-parallel edges (reading: the paper is
silent; the constant c = 1e-3 follows the cited IPC work).
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sp

# distance-type codes (shared meaning with nothing else: oracle-local)
PP, PE, PT_, EE_ = 0, 1, 2, 3


@functools.lru_cache(maxsize=None)
def _sym(kind: str):
    if kind == "PP":
        v = sp.symbols("v0:6", real=True)
        p, q = sp.Matrix(v[0:3]), sp.Matrix(v[3:6])
        D = (p - q).dot(p - q)
    elif kind == "PE":
        v = sp.symbols("v0:9", real=True)
        p, e0, e1 = sp.Matrix(v[0:3]), sp.Matrix(v[3:6]), sp.Matrix(v[6:9])
        c = (p - e0).cross(e1 - e0)
        D = c.dot(c) / (e1 - e0).dot(e1 - e0)
    elif kind == "PT":
        v = sp.symbols("v0:12", real=True)
        p, t0, t1, t2 = (sp.Matrix(v[3 * i:3 * i + 3]) for i in range(4))
        n = (t1 - t0).cross(t2 - t0)
        D = ((p - t0).dot(n)) ** 2 / n.dot(n)
    elif kind == "EE":
        v = sp.symbols("v0:12", real=True)
        a0, a1, b0, b1 = (sp.Matrix(v[3 * i:3 * i + 3]) for i in range(4))
        n = (a1 - a0).cross(b1 - b0)
        D = ((a0 - b0).dot(n)) ** 2 / n.dot(n)
    elif kind == "X":      # mollifier argument |(a1 - a0) x (b1 - b0)|^2
        v = sp.symbols("v0:12", real=True)
        a0, a1, b0, b1 = (sp.Matrix(v[3 * i:3 * i + 3]) for i in range(4))
        n = (a1 - a0).cross(b1 - b0)
        D = n.dot(n)
    else:
        raise KeyError(kind)
    g = [sp.diff(D, s) for s in v]
    H = [[sp.diff(gi, s) for s in v] for gi in g]
    f = sp.lambdify([v], D, "numpy", cse=True)
    fg = sp.lambdify([v], g, "numpy", cse=True)
    fh = sp.lambdify([v], H, "numpy", cse=True)
    return len(v), f, fg, fh


def _eval(kind: str, X: np.ndarray, order: int):
    """X: (n, k) coordinates.  Returns D (n,), grad (n, k), hess (n, k, k)."""
    k, f, fg, fh = _sym(kind)
    n = X.shape[0]
    cols = [X[:, i] for i in range(k)]
    D = np.broadcast_to(np.asarray(f(cols), dtype=np.float64), (n,)).copy()
    if order == 0:
        return D, None, None
    g = np.stack([np.broadcast_to(np.asarray(e, dtype=np.float64), (n,)) for e in fg(cols)], axis=1)
    if order == 1:
        return D, g, None
    Hl = fh(cols)
    H = np.stack([np.stack([np.broadcast_to(np.asarray(e, dtype=np.float64), (n,)) for e in row], axis=1)
                  for row in Hl], axis=1)
    return D, g, H


# ----------------------------------------------------------------------------
# classification: which closed form is the exact minimum distance
# ----------------------------------------------------------------------------
def _point_segment(p, e0, e1):
    e = e1 - e0
    t = np.einsum("ij,ij->i", p - e0, e) / np.einsum("ij,ij->i", e, e)
    tc = np.clip(t, 0.0, 1.0)
    c = e0 + tc[:, None] * e
    d2 = ((p - c) ** 2).sum(axis=1)
    kind = np.where(t <= 0.0, 0, np.where(t >= 1.0, 1, 2))   # 0: PP e0, 1: PP e1, 2: PE
    return d2, kind


def classify_pt(p, t0, t1, t2):
    """Returns (kind, idx) per pair: kind in {PP, PE, PT_} and the local point
    indices (into [p, t0, t1, t2]) of the closed form to use (padded with -1)."""
    n = p.shape[0]
    e0, e1, w = t1 - t0, t2 - t0, p - t0
    a = np.einsum("ij,ij->i", e0, e0)
    b = np.einsum("ij,ij->i", e0, e1)
    c = np.einsum("ij,ij->i", e1, e1)
    d = np.einsum("ij,ij->i", e0, w)
    e = np.einsum("ij,ij->i", e1, w)
    det = a * c - b * b
    b1 = (c * d - b * e) / det
    b2 = (a * e - b * d) / det
    inside = (b1 >= 0.0) & (b2 >= 0.0) & (b1 + b2 <= 1.0)
    kind = np.full(n, PT_, np.int64)
    idx = np.tile(np.array([0, 1, 2, 3]), (n, 1))
    tri = [t0, t1, t2]
    best = np.full(n, np.inf)
    bk = np.zeros(n, np.int64)
    bi = np.full((n, 4), -1, np.int64)
    for (i, j) in ((0, 1), (1, 2), (2, 0)):
        d2, k = _point_segment(p, tri[i], tri[j])
        better = d2 < best
        best = np.where(better, d2, best)
        kk = np.where(k == 2, PE, PP)
        ii = np.where(k[:, None] == 2, np.array([0, 1 + i, 1 + j, -1]),
                      np.where(k[:, None] == 0, np.array([0, 1 + i, -1, -1]), np.array([0, 1 + j, -1, -1])))
        bk = np.where(better, kk, bk)
        bi = np.where(better[:, None], ii, bi)
    kind = np.where(inside, kind, bk)
    idx = np.where(inside[:, None], idx, bi)
    return kind, idx


def classify_ee(a0, a1, b0, b1, parallel_tol=1e-20):
    n = a0.shape[0]
    a, b, w = a1 - a0, b1 - b0, a0 - b0
    aa = np.einsum("ij,ij->i", a, a)
    bb = np.einsum("ij,ij->i", b, b)
    ab = np.einsum("ij,ij->i", a, b)
    aw = np.einsum("ij,ij->i", a, w)
    bw = np.einsum("ij,ij->i", b, w)
    det = aa * bb - ab * ab
    ok = det > parallel_tol * aa * bb
    with np.errstate(invalid="ignore", divide="ignore"):
        s = (ab * bw - bb * aw) / det
        t = (aa * bw - ab * aw) / det
    interior = ok & (s > 0.0) & (s < 1.0) & (t > 0.0) & (t < 1.0)
    pts = [a0, a1, b0, b1]
    best = np.full(n, np.inf)
    bk = np.zeros(n, np.int64)
    bi = np.full((n, 4), -1, np.int64)
    # boundary of the parameter square: each endpoint against the other segment
    for (pi, s0, s1) in ((0, 2, 3), (1, 2, 3), (2, 0, 1), (3, 0, 1)):
        d2, k = _point_segment(pts[pi], pts[s0], pts[s1])
        better = d2 < best
        best = np.where(better, d2, best)
        kk = np.where(k == 2, PE, PP)
        ii = np.where(k[:, None] == 2, np.array([pi, s0, s1, -1]),
                      np.where(k[:, None] == 0, np.array([pi, s0, -1, -1]), np.array([pi, s1, -1, -1])))
        bk = np.where(better, kk, bk)
        bi = np.where(better[:, None], ii, bi)
    kind = np.where(interior, EE_, bk)
    idx = np.where(interior[:, None], np.array([0, 1, 2, 3]), bi)
    return kind, idx


_KNAME = {PP: "PP", PE: "PE", PT_: "PT", EE_: "EE"}
_KPTS = {PP: 2, PE: 3, PT_: 4, EE_: 4}


def pair_sqdist(X12: np.ndarray, kind: np.ndarray, idx: np.ndarray, order: int = 2):
    """Squared distance D of each pair with its gradient/Hessian in the pair's
    12 coordinates.  X12: (n, 4, 3)."""
    n = X12.shape[0]
    D = np.zeros(n)
    G = np.zeros((n, 12)) if order >= 1 else None
    H = np.zeros((n, 12, 12)) if order >= 2 else None
    for k in (PP, PE, PT_, EE_):
        m = kind == k
        if not np.any(m):
            continue
        npts = _KPTS[k]
        # group rows by local index pattern (few distinct patterns)
        pats, inv = np.unique(idx[m][:, :npts], axis=0, return_inverse=True)
        rows = np.nonzero(m)[0]
        for pi, pat in enumerate(pats):
            r = rows[inv.ravel() == pi]
            Xs = X12[r][:, pat, :].reshape(len(r), -1)
            d, g, h = _eval(_KNAME[k], Xs, order)
            D[r] = d
            cidx = (3 * pat[:, None] + np.arange(3)[None]).ravel()
            if order >= 1:
                G[np.ix_(r, cidx)] = g
            if order >= 2:
                H[np.ix_(r, cidx, cidx)] = h
    return D, G, H


def pair_kinds(X12: np.ndarray, is_ee: np.ndarray):
    kind = np.zeros(X12.shape[0], np.int64)
    idx = np.full((X12.shape[0], 4), -1, np.int64)
    pt = ~is_ee
    if np.any(pt):
        k, i = classify_pt(X12[pt, 0], X12[pt, 1], X12[pt, 2], X12[pt, 3])
        kind[pt], idx[pt] = k, i
    if np.any(is_ee):
        k, i = classify_ee(X12[is_ee, 0], X12[is_ee, 1], X12[is_ee, 2], X12[is_ee, 3])
        kind[is_ee], idx[is_ee] = k, i
    return kind, idx


# ----------------------------------------------------------------------------
# barrier
# ----------------------------------------------------------------------------
def barrier(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -(d - dhat) ** 2 * np.log(d / dhat)
    v = np.where(d < dhat, v, 0.0)
    return np.where(d > 0.0, v, np.inf)


def barrier_d1(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -2.0 * (d - dhat) * np.log(d / dhat) - (d - dhat) ** 2 / d
    return np.where(d < dhat, v, 0.0)


def barrier_d2(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -2.0 * np.log(d / dhat) - 4.0 * (d - dhat) / d + (d - dhat) ** 2 / d ** 2
    return np.where(d < dhat, v, 0.0)


def mollifier_arg(X12: np.ndarray, order: int = 2):
    return _eval("X", X12.reshape(X12.shape[0], 12), order)


def pair_barrier(X12, is_ee, weight, eps_x, dhat, order=2, project=True):
    """Weighted barrier energy of pairs: weight * c(x) * b(d) (c = 1 for PT).

    X12 (n, 4, 3); weight (n,) = dt^2 kappa A_k; eps_x (n,) mollifier
    thresholds (ignored for PT).  Returns E (n,), grad (n, 12), hess (n,12,12)
    with the Hessian filtered to PSD per `project` (False: raw; True /
    "clamp": negative eigenvalues set to zero; "abs": replaced by their
    absolute values).
    """
    n = X12.shape[0]
    kind, idx = pair_kinds(X12, is_ee)
    D, gD, hD = pair_sqdist(X12, kind, idx, order)
    d = np.sqrt(D)
    active = d < dhat
    E = np.zeros(n)
    G = np.zeros((n, 12)) if order >= 1 else None
    H = np.zeros((n, 12, 12)) if order >= 2 else None
    if not np.any(active):
        return E, G, H
    a = np.nonzero(active)[0]
    da = d[a]
    b0 = barrier(da, dhat)
    c = np.ones(len(a))
    gc = np.zeros((len(a), 12))
    hc = np.zeros((len(a), 12, 12))
    ee = is_ee[a]
    if np.any(ee):
        r = np.nonzero(ee)[0]
        x, gx, hx = mollifier_arg(X12[a[r]], order)
        eps = eps_x[a[r]]
        m = x < eps
        cval = np.where(m, -x * x / eps ** 2 + 2.0 * x / eps, 1.0)
        c1 = np.where(m, -2.0 * x / eps ** 2 + 2.0 / eps, 0.0)
        c2 = np.where(m, -2.0 / eps ** 2, 0.0)
        c[r] = cval
        if order >= 1:
            gc[r] = c1[:, None] * gx
        if order >= 2:
            hc[r] = c2[:, None, None] * np.einsum("ni,nj->nij", gx, gx) + c1[:, None, None] * hx
    w = weight[a]
    E[a] = w * c * b0
    if order >= 1:
        b1 = barrier_d1(da, dhat)
        gd = gD[a] / (2.0 * da[:, None])
        gb = b1[:, None] * gd
        G[a] = w[:, None] * (c[:, None] * gb + b0[:, None] * gc)
    if order >= 2:
        b2 = barrier_d2(da, dhat)
        hd = hD[a] / (2.0 * da[:, None, None]) - np.einsum("ni,nj->nij", gD[a], gD[a]) / (4.0 * da[:, None, None] ** 3)
        hb = b2[:, None, None] * np.einsum("ni,nj->nij", gd, gd) + b1[:, None, None] * hd
        Hk = (c[:, None, None] * hb + np.einsum("ni,nj->nij", gb, gc) + np.einsum("ni,nj->nij", gc, gb)
              + b0[:, None, None] * hc)
        Hk = w[:, None, None] * Hk
        from .energy import psd_filter
        Hk = psd_filter(Hk, project)
        H[a] = Hk
    return E, G, H


def pair_distance(X12: np.ndarray, is_ee: np.ndarray) -> np.ndarray:
    kind, idx = pair_kinds(X12, is_ee)
    D, _, _ = pair_sqdist(X12, kind, idx, 0)
    return np.sqrt(D)
