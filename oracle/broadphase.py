"""Brute-force candidate pairs (oracle side).

Pairs (App. A.3): point-triangle and edge-edge pairs between surface
primitives.  Reading: only primitives of different objects pair up
(gel pads and affine bodies are objects; gel self-contact is not modelled),
pairs whose four vertices are all fixed are dropped, and a gel pad never
pairs with the body it is attached to.

Candidate test: axis-aligned boxes of the two primitives, each taken over the
primitive's vertices (and, for the swept set, over their positions at both
ends of the step), overlap after widening by dhat:
    lo_a <= hi_b + dhat  and  lo_b <= hi_a + dhat   on every axis
(closed intervals; a pair closer than dhat always passes).
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
    """(pad, body-object) pairs excluded because the pad is attached to it."""
    n_pads = int(scene.gel_obj.max()) + 1 if scene.n_verts else 0
    ex = set()
    m = scene.attach >= 0
    for pad, b in zip(scene.gel_obj[m], scene.attach[m]):
        o = n_pads + int(b)
        ex.add((int(pad), o))
        ex.add((o, int(pad)))
    return ex


def candidates(sd, Xc: np.ndarray, dhat: float, excluded: set, Xc_end=None):
    """Returns (pt (n,2) [point cv id, tri index], ee (m,2) [edge, edge]).

    PT pairs: every point against every triangle of another object.
    EE pairs: edge a of object oa against edge b of object ob with oa < ob.
    Rows are sorted lexicographically.
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
            if oa == ob or (oa, ob) in excluded:
                continue
            tb = np.nonzero(sd.tri_obj == ob)[0]
            if len(pa) and len(tb):
                i, j = _overlap(plo[pa], phi[pa], tlo[tb], thi[tb], dhat)
                pts.append(np.stack([sd.points[pa[i]], tb[j]], axis=1))
            if oa < ob:
                eb = np.nonzero(sd.edge_obj == ob)[0]
                if len(ea) and len(eb):
                    i, j = _overlap(elo[ea], ehi[ea], elo[eb], ehi[eb], dhat)
                    ees.append(np.stack([ea[i], eb[j]], axis=1))
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
    PT -> (p, sorted triangle vertices), EE -> (sorted edge a, sorted edge b)
    with the edge of the lower object first."""
    a = np.concatenate([pt[:, :1], np.sort(sd.tris[pt[:, 1]], axis=1)], axis=1) if len(pt) else np.zeros((0, 4), np.int64)
    b = np.concatenate([np.sort(sd.edges[ee[:, 0]], axis=1), np.sort(sd.edges[ee[:, 1]], axis=1)], axis=1) if len(ee) else np.zeros((0, 4), np.int64)
    a = a[np.lexsort(a.T[::-1])] if len(a) else a
    b = b[np.lexsort(b.T[::-1])] if len(b) else b
    return a, b
