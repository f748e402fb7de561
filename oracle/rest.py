"""Rest-shape precomputation (oracle side).

Gel: rest shape matrix ``D_m`` and its inverse, tet volumes ``V_e``, lumped
vertex masses ``rho V_e / 4`` (the mass matrix ``M`` of Sec. 3.1 read as
lumped-diagonal), Lame parameters from ``(E, nu)`` (App. A.1).

Body: volume, centre of mass and second moments by exact integration over the
closed surface (tetrahedra fanned from a reference point), giving the reduced
mass matrix ``M^y = int rho J^T J dV`` of Sec. 3.3 with
``J_j = [I, xbar_j0 I, xbar_j1 I, xbar_j2 I]``.

Surface: boundary faces of the tet mesh, unique edges, and the contact area
weights (``A_k`` of Eq. fullspace_ipc is not defined in the paper; read as
one third of incident rest triangle areas, see ``surface_data``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GelRest:
    Dm_inv: np.ndarray      # (T, 3, 3)
    vol: np.ndarray         # (T,)
    mass: np.ndarray        # (N,)
    mu: float
    lam: float


@dataclass
class BodyRest:
    com: np.ndarray         # (3,)
    xbar: np.ndarray        # (nv, 3) vertices relative to the centre of mass
    vol: float
    mass: float
    S: np.ndarray           # (3, 3) int rho xbar xbar^T dV
    My: np.ndarray          # (12, 12)


@dataclass
class SurfaceData:
    """Contact surface of one environment in a unified contact-vertex space.

    Contact vertex ids: gel vertices 0..N-1 keep their ids; body b's vertex j
    gets id ``N + body_vert_off[b] + j``.
    """
    n_gel: int
    body_vert_off: np.ndarray     # (n_b + 1,)
    points: np.ndarray            # (P,) contact-vertex ids usable as PT points
    point_obj: np.ndarray         # (P,) object id
    point_area: np.ndarray        # (P,) a_v
    tris: np.ndarray              # (F, 3) contact-vertex ids
    tri_obj: np.ndarray           # (F,)
    edges: np.ndarray             # (Ed, 2)
    edge_obj: np.ndarray          # (Ed,)
    edge_area: np.ndarray         # (Ed,) a_e
    edge_rest_len2: np.ndarray    # (Ed,) squared rest length
    fixed: np.ndarray             # (n_gel + n_bodyverts,) bool: no DoF moves it
    n_objects: int


def lame(E: float, nu: float):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def gel_rest(scene) -> GelRest:
    X = scene.gel_x
    T = scene.gel_tets
    X0 = X[T[:, 0]]
    Dm = np.stack([X[T[:, 1]] - X0, X[T[:, 2]] - X0, X[T[:, 3]] - X0], axis=-1)
    det = np.linalg.det(Dm)
    if np.any(det <= 0.0):
        raise ValueError("gel tetrahedra must be positively oriented")
    vol = det / 6.0
    mass = np.zeros(X.shape[0])
    np.add.at(mass, T.ravel(), np.repeat(scene.rho * vol / 4.0, 4))
    mu, lam = lame(scene.E, scene.nu)
    return GelRest(Dm_inv=np.linalg.inv(Dm), vol=vol, mass=mass, mu=mu, lam=lam)


def body_rest(body) -> BodyRest:
    """Mass properties of a closed outward triangle surface of density rho.

    Each triangle (v0, v1, v2) spans a signed tetrahedron with the vertex mean
    r.  For a tetrahedron with corners q_0..q_3 and volume V:
      int dV = V,  int x dV = V (sum q_i) / 4,
      int x x^T dV = V / 20 (sum q_i q_i^T + s s^T),  s = sum q_i.
    """
    X = body.rest_x
    F = body.tris
    r = X.mean(axis=0)
    Xr = X - r                      # integrate about r to limit cancellation
    q1, q2, q3 = Xr[F[:, 0]], Xr[F[:, 1]], Xr[F[:, 2]]
    V = np.einsum("ij,ij->i", np.cross(q1, q2), q3) / 6.0
    vol = V.sum()
    if vol <= 0.0:
        raise ValueError("body surface must be closed and outward oriented")
    s = q1 + q2 + q3                # the fourth corner is r itself (0 here)
    first = (V[:, None] * s).sum(axis=0) / 4.0
    second = np.zeros((3, 3))
    for q in (q1, q2, q3):
        second += np.einsum("i,ij,ik->jk", V, q, q)
    second += np.einsum("i,ij,ik->jk", V, s, s)
    second /= 20.0
    c = first / vol
    com = r + c
    S = body.rho * (second - vol * np.outer(c, c))
    m = body.rho * vol
    My = np.zeros((12, 12))
    My[0:3, 0:3] = m * np.eye(3)
    for k in range(3):
        for l in range(3):
            My[3 + 3 * k:6 + 3 * k, 3 + 3 * l:6 + 3 * l] = S[k, l] * np.eye(3)
    return BodyRest(com=com, xbar=X - com, vol=vol, mass=m, S=S, My=My)


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one tetrahedron, oriented outward."""
    loc = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    faces = tets[:, loc].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1].astype(np.int64)


def _edges_of(tris: np.ndarray):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def surface_data(scene, bodies: list) -> SurfaceData:
    """Gel boundary + body surfaces, areas and fixed flags (reading: the
    contact area weights come from one third of the incident rest triangle
    areas)."""
    N = scene.n_verts
    nb = len(scene.bodies)
    off = np.zeros(nb + 1, np.int64)
    for b, body in enumerate(scene.bodies):
        off[b + 1] = off[b] + body.rest_x.shape[0]
    n_pads = int(scene.gel_obj.max()) + 1 if N else 0

    # positions at rest in contact-vertex space
    Xc = np.concatenate([scene.gel_x] + [bd.rest_x for bd in scene.bodies]) if nb else scene.gel_x
    gtris = boundary_faces(scene.gel_tets)
    btris = [bd.tris.astype(np.int64) + N + off[b] for b, bd in enumerate(scene.bodies)]
    tris = np.concatenate([gtris] + btris) if nb else gtris
    tri_obj = np.concatenate([scene.gel_obj[gtris[:, 0]]] +
                             [np.full(bd.tris.shape[0], n_pads + b) for b, bd in enumerate(scene.bodies)])

    a = Xc[tris[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(Xc[tris[:, 1]] - a, Xc[tris[:, 2]] - a), axis=1)

    nc = N + int(off[-1])
    vert_area = np.zeros(nc)
    np.add.at(vert_area, tris.ravel(), np.repeat(area / 3.0, 3))
    on_surface = np.zeros(nc, bool)
    on_surface[tris.ravel()] = True
    points = np.nonzero(on_surface)[0]
    obj_of = np.concatenate([scene.gel_obj.astype(np.int64)] +
                            [np.full(bd.rest_x.shape[0], n_pads + b) for b, bd in enumerate(scene.bodies)])

    edges = _edges_of(tris)
    # area of each edge: one third of the adjacent triangle areas
    te = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    te = np.sort(te, axis=1)
    ta = np.concatenate([area, area, area]) / 3.0
    # map each triangle edge to its index in `edges`
    ekey = edges[:, 0] * nc + edges[:, 1]
    tkey = te[:, 0] * nc + te[:, 1]
    idx = np.searchsorted(ekey, tkey)
    edge_area = np.zeros(edges.shape[0])
    np.add.at(edge_area, idx, ta)
    el2 = ((Xc[edges[:, 0]] - Xc[edges[:, 1]]) ** 2).sum(axis=1)

    fixed = np.zeros(nc, bool)
    fixed[:N] = scene.pinned
    return SurfaceData(n_gel=N, body_vert_off=off, points=points,
                       point_obj=obj_of[points], point_area=vert_area[points],
                       tris=tris, tri_obj=tri_obj, edges=edges,
                       edge_obj=obj_of[edges[:, 0]], edge_area=edge_area,
                       edge_rest_len2=el2, fixed=fixed, n_objects=n_pads + nb)
