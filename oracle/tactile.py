"""Tactile outputs read off the deformed coated surface (Sec. 4.2).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Markers (Sec. 4.2, Markers): a marker sits on a coated-surface triangle at
barycentric coordinates alpha; its position after deformation is
p~ = sum_u alpha_u x~_u and its flow is p~ - p (p: the rest position).

Depth and normal maps (Sec. 4.2, RGB Images and Depth Maps; readings, the
paper gives no sensor model):
  * an orthographic sensor on a gel pad: origin o on the pad's rest contact
    face, in-plane unit axes e_u, e_v, unit normal n pointing out of the
    coated face, pixel pitch; pixel (r, c) has its centre at
    o + (c + 1/2) pitch e_u + (r + 1/2) pitch e_v;
  * the camera looks through the gel from behind, along +n: each pixel shows
    the front-face triangle (a coated triangle of that pad whose rest
    outward normal has n-component > 1/2) hit first along +n, i.e. the one
    with the smallest height h = (x - o).n at the pixel centre;
  * depth = -h at that point (how far the surface is pressed below the rest
    face; 0 at rest), linearly interpolated over the triangle; normal = the
    deformed outward unit normal of that triangle; pixels no triangle covers
    report hit = 0 and depth 0;
  * a pixel centre belongs to a triangle when its barycentric coordinates
    are all >= -1e-12, so a centre on a shared edge is not lost to rounding
    (it then belongs to both; the depth is the same, continuous surface).
This is the brute-force definition: every pixel against every front-face
triangle.
"""
from __future__ import annotations

import numpy as np


def boundary_faces(tets: np.ndarray, x_rest: np.ndarray) -> np.ndarray:
    """Faces of a tet mesh that belong to one tet only, outward oriented."""
    faces = {}
    local = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
    for t in tets:
        for (a, b, c) in local:
            f = (t[a], t[b], t[c])
            key = tuple(sorted(f))
            if key in faces:
                faces[key] = None
            else:
                opp = [v for v in t if v not in f][0]
                faces[key] = (f, opp)
    out = []
    for val in faces.values():
        if val is None:
            continue
        f, opp = val
        p0, p1, p2 = x_rest[f[0]], x_rest[f[1]], x_rest[f[2]]
        nrm = np.cross(p1 - p0, p2 - p0)
        if nrm @ (x_rest[opp] - p0) > 0.0:          # normal must point away from the tet
            f = (f[0], f[2], f[1])
        out.append(f)
    return np.asarray(out, dtype=np.int64)


def front_triangles(tets, x_rest, coated, pad_of_vertex, pad, normal):
    """Coated boundary faces of `pad` whose rest outward normal has an
    n-component above 1/2 (all three vertices coated)."""
    F = boundary_faces(tets, x_rest)
    keep = []
    for f in F:
        if not (coated[f].all() and np.all(pad_of_vertex[f] == pad)):
            continue
        p0, p1, p2 = x_rest[f]
        nrm = np.cross(p1 - p0, p2 - p0)
        nrm /= np.linalg.norm(nrm)
        if nrm @ normal > 0.5:
            keep.append(f)
    return np.asarray(keep, dtype=np.int64).reshape(-1, 3)


def marker_positions(x: np.ndarray, tri: np.ndarray, bary: np.ndarray) -> np.ndarray:
    """p~_k = sum_u alpha_ku x_(tri_ku)."""
    return np.einsum("ku,kuc->kc", bary, x[tri])


def depth_normal_map(x: np.ndarray, tris: np.ndarray, origin, e_u, e_v, n, pitch: float,
                     height: int, width: int):
    """(depth (H, W), normal (H, W, 3), hit (H, W) bool) by brute force."""
    o, eu, ev, nn = (np.asarray(a, dtype=np.float64) for a in (origin, e_u, e_v, n))
    P = x[tris]                                          # (T, 3, 3)
    U = (P - o) @ eu
    V = (P - o) @ ev
    Hh = (P - o) @ nn
    fn = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    depth = np.zeros((height, width))
    normal = np.zeros((height, width, 3))
    hit = np.zeros((height, width), bool)
    for r in range(height):
        for c in range(width):
            pu, pv = (c + 0.5) * pitch, (r + 0.5) * pitch
            best = np.inf
            for t in range(len(tris)):
                (u0, u1, u2), (v0, v1, v2) = U[t], V[t]
                det = (u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0)
                if det == 0.0:
                    continue
                b1 = ((pu - u0) * (v2 - v0) - (u2 - u0) * (pv - v0)) / det
                b2 = ((u1 - u0) * (pv - v0) - (pu - u0) * (v1 - v0)) / det
                b0 = 1.0 - b1 - b2
                if min(b0, b1, b2) < -1e-12:
                    continue
                h = b0 * Hh[t, 0] + b1 * Hh[t, 1] + b2 * Hh[t, 2]
                if h < best:
                    best = h
                    depth[r, c] = -h
                    normal[r, c] = fn[t]
                    hit[r, c] = True
    return depth, normal, hit
