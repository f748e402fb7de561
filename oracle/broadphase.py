"""Brute-force candidate pairs (oracle side).

Pairs (App. A.3): point-triangle and edge-edge pairs between surface
primitives.  Readings: primitives of different objects pair up (gel pads and
affine bodies are objects); a pad flagged for self-contact also pairs its own
primitives that share no vertex (a point against a triangle not incident to
it, two edges without a common end point), which is the soft-soft contact of
a gel with itself; an affine body never pairs with itself (it is rigid up to
its affine modes).  Pairs whose four vertices are all fixed are dropped, and
a gel pad never pairs with the body it is attached to.

Candidate test: axis-aligned boxes of the two primitives, each taken over the
primitive's vertices (and, for the swept set, over their positions at both
ends of the step), overlap after widening by dhat:
    lo_a <= hi_b + dhat  and  lo_b <= hi_a + dhat   on every axis
(closed intervals; a pair closer than dhat always passes).

Object pairs that never pair are one set of ordered (a, b) object ids; an
object that does not self-contact appears there as (a, a).
"""
from __future__ import annotations

import numpy as np


def _boxes(X: np.ndarray, prims: np.ndarray, X_end=None):
    P = X[prims]                       # (n, k, 3)
    lo, hi = P.min(axis=1), P.max(axis=1)
    if X_end is not None:
        Q = X_end[prims]
        lo = np.minimum(lo, Q.min(axis=1))
        hi = np.maximum(hi, Q.max(axis=1))
    return lo, hi


def _overlap(loA, hiA, loB, hiB, dhat, chunk=2048):
    """All (i, j) with box i of A and box j of B overlapping after widening."""
    out_i, out_j = [], []
    for s in range(0, loA.shape[0], chunk):
        la, ha = loA[s:s + chunk, None, :], hiA[s:s + chunk, None, :]
        ok = np.all((la <= hiB[None] + dhat) & (loB[None] <= ha + dhat), axis=2)
        i, j = np.nonzero(ok)
        out_i.append(i + s)
        out_j.append(j)
    if not out_i:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(out_i), np.concatenate(out_j)


def excluded_object_pairs(scene) -> set:
    """Object pairs that never pair: (pad, body) when the pad is attached to
    the body, and (o, o) for every object that does not self-contact."""
    n_pads = int(scene.gel_obj.max()) + 1 if scene.n_verts else 0
    ex = set()
    m = scene.attach >= 0
    for pad, b in zip(scene.gel_obj[m], scene.attach[m]):
        o = n_pads + int(b)
        ex.add((int(pad), o))
        ex.add((o, int(pad)))
    selfc = np.zeros(n_pads, bool) if scene.self_contact is None else np.asarray(scene.self_contact, bool)
    for o in range(n_pads + len(scene.bodies)):
        if o >= n_pads or not selfc[o]:
            ex.add((o, o))
    return ex


def candidates(sd, Xc: np.ndarray, dhat: float, excluded: set, Xc_end=None):
    """Returns (pt (n,2) [point cv id, tri index], ee (m,2) [edge, edge]).

    PT pairs: every point against every triangle of another object, and of
    its own object when that object self-contacts and the triangle does not
    contain the point.  EE pairs: edge a of object oa against edge b of
    object ob with oa < ob, or, within a self-contacting object, edges a < b
    with no common vertex.  Rows are sorted lexicographically.
    """
    plo, phi = _boxes(Xc, sd.points[:, None], Xc_end)
    tlo, thi = _boxes(Xc, sd.tris, Xc_end)
    elo, ehi = _boxes(Xc, sd.edges, Xc_end)
    pts, ees = [], []
    objs = range(sd.n_objects)
    for oa in objs:
        pa = np.nonzero(sd.point_obj == oa)[0]
        ea = np.nonzero(sd.edge_obj == oa)[0]
        for ob in objs:
            if (oa, ob) in excluded:
                continue
            tb = np.nonzero(sd.tri_obj == ob)[0]
            if len(pa) and len(tb):
                i, j = _overlap(plo[pa], phi[pa], tlo[tb], thi[tb], dhat)
                p, t = sd.points[pa[i]], tb[j]
                if oa == ob:  # the point must not be a vertex of the triangle
                    keep = np.all(sd.tris[t] != p[:, None], axis=1)
                    p, t = p[keep], t[keep]
                pts.append(np.stack([p, t], axis=1))
            if oa <= ob:
                eb = np.nonzero(sd.edge_obj == ob)[0]
                if len(ea) and len(eb):
                    i, j = _overlap(elo[ea], ehi[ea], elo[eb], ehi[eb], dhat)
                    a, b = ea[i], eb[j]
                    if oa == ob:  # each unordered pair once, no common vertex
                        A, B = sd.edges[a], sd.edges[b]
                        keep = (a < b) & np.all(A[:, :, None] != B[:, None, :], axis=(1, 2))
                        a, b = a[keep], b[keep]
                    ees.append(np.stack([a, b], axis=1))
    pt = np.concatenate(pts) if pts else np.zeros((0, 2), np.int64)
    ee = np.concatenate(ees) if ees else np.zeros((0, 2), np.int64)
    # drop pairs whose four vertices are all fixed
    if len(pt):
        allfix = sd.fixed[pt[:, 0]] & np.all(sd.fixed[sd.tris[pt[:, 1]]], axis=1)
        pt = pt[~allfix]
    if len(ee):
        allfix = np.all(sd.fixed[sd.edges[ee[:, 0]]], axis=1) & np.all(sd.fixed[sd.edges[ee[:, 1]]], axis=1)
        ee = ee[~allfix]
    pt = pt[np.lexsort((pt[:, 1], pt[:, 0]))] if len(pt) else pt
    ee = ee[np.lexsort((ee[:, 1], ee[:, 0]))] if len(ee) else ee
    return pt.astype(np.int64), ee.astype(np.int64)


def canonical(sd, pt: np.ndarray, ee: np.ndarray):
    """Vertex-id form used to compare candidate sets across implementations:
    PT -> (p, sorted triangle vertices), EE -> the two sorted edges, the
    lexicographically smaller first (an EE pair is unordered)."""
    a = np.concatenate([pt[:, :1], np.sort(sd.tris[pt[:, 1]], axis=1)], axis=1) if len(pt) else np.zeros((0, 4), np.int64)
    if len(ee):
        e0, e1 = np.sort(sd.edges[ee[:, 0]], axis=1), np.sort(sd.edges[ee[:, 1]], axis=1)
        swap = (e0[:, 0] > e1[:, 0]) | ((e0[:, 0] == e1[:, 0]) & (e0[:, 1] > e1[:, 1]))
        e0[swap], e1[swap] = e1[swap].copy(), e0[swap].copy()
        b = np.concatenate([e0, e1], axis=1)
    else:
        b = np.zeros((0, 4), np.int64)
    a = a[np.lexsort(a.T[::-1])] if len(a) else a
    b = b[np.lexsort(b.T[::-1])] if len(b) else b
    return a, b
