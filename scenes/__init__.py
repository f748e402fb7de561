"""Seeded synthetic inputs for the batched ABD-IPC step.

This module only builds geometry and seeded scenario parameters: tetrahedral
gel grids, icosphere and box surface meshes, pinned/attached vertex masks and
scripted rigid-translation trajectories for driven bodies.  It holds none of
the solver's arithmetic (no masses, no rest-shape matrices, no energies); the
oracle and the CUDA library each derive those from the raw geometry on their
own.  Both sides may import this module.

Scene layout (all SI units, float64 coordinates):

* The gel pad(s) of one environment form one tetrahedral mesh (``gel_x``,
  ``gel_tets``).  ``gel_obj`` labels each vertex with its pad id (0, 1, ...);
  different pads are different contact objects.  ``pinned`` marks vertices
  held fixed (the bottom face of a pad resting on a table), ``attach`` gives,
  per vertex, the index of the affine body that drives it (``-1`` = free),
  which models the sensor-attached region of a gel pad (Sec. 4.1, "Tactile
  Sensors Modeling").  ``self_contact`` (optional, one flag per pad) lets
  the primitives of a pad that share no vertex touch one another: gel
  self-contact (soft-soft contact within one pad).
* Each affine body is a closed, outward-oriented triangle surface given at its
  rest placement in world coordinates.  Its reduced state is
  ``y = [p, a0, a1, a2]`` where ``p`` is the world position of its centre of
  mass and ``a_k`` the k-th column of the affine matrix ``A``; the rest
  placement is ``p = centre of mass, A = I``.
* Driven bodies follow a scripted trajectory given as a translation ``delta``
  of the body from its rest placement, with ``A = I`` (Sec. 4.1, "Robot
  Actions": targets assembled into ``s^y``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

__all__ = [
    "Body", "Scene", "Scenario", "SolverParams",
    "gel_grid", "icosphere", "box_surface",
    "config0", "config1", "config2", "config3", "config3_batch", "small_contact_scene",
    "self_contact_pad", "pad_and_sphere",
    "free_fall_scene", "spin_scene", "self_contact_scene",
]


# ----------------------------------------------------------------------------
# data containers
# ----------------------------------------------------------------------------
@dataclass
class Body:
    rest_x: np.ndarray          # (nv, 3) float64, rest placement (world)
    tris: np.ndarray            # (nt, 3) int32, outward-oriented, closed
    rho: float                  # density, kg/m^3
    kappa_s: float              # orthogonality stiffness, Pa
    driven: bool                # follows a scripted target when True


@dataclass
class Scene:
    gel_x: np.ndarray           # (N, 3) float64 rest positions
    gel_tets: np.ndarray        # (T, 4) int32, positively oriented
    gel_obj: np.ndarray         # (N,) int32 pad id
    pinned: np.ndarray          # (N,) bool
    attach: np.ndarray          # (N,) int32, body index or -1
    E: float                    # Young's modulus, Pa
    nu: float                   # Poisson ratio
    rho: float                  # gel density, kg/m^3
    bodies: List[Body] = field(default_factory=list)
    name: str = ""
    self_contact: Optional[np.ndarray] = None   # (n_pads,) bool, None = no pad self-contacts

    @property
    def n_verts(self) -> int:
        return int(self.gel_x.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.gel_tets.shape[0])


@dataclass
class SolverParams:
    dt: float = 1e-3
    gravity: tuple = (0.0, 0.0, -9.81)
    dhat: float = 1e-4
    kappa: float = 1e6
    newton_tol: float = 1e-4        # ||p||_inf / dt, m/s
    pcg_rel_tol: float = 1e-4
    newton_max: int = 300           # safety cap; the press steps need up to ~120 iterations
    pcg_max: int = 1000
    ls_max: int = 30
    accd_max: int = 10000
    accd_s: float = 0.1
    al_kappa: float = 1e6           # mass-weighted AL penalty factor
    al_max: int = 10
    ee_mollifier: float = 1e-3
    precision: int = 0              # 0 FP64, 1 mixed (FP32 Hessians / mat-vec)
    max_pairs_per_env: int = 0      # candidate-pair capacity per env (0 = default)
    friction_mu: float = 0.0        # lagged IPC friction coefficient (0 = frictionless)
    friction_eps_v: float = 1e-3    # static/dynamic velocity threshold, m/s
    newton_abs_after: int = 1000000  # Newton iterations that clamp negative eigenvalues; |lambda| after
    rollout_pcg_window: int = 0     # rollout: PCG iterations per loop iteration (0: whole solves)
    pcg_fused: int = 1              # 1 / 2: one persistent kernel per PCG iteration (ready / env order); 0: three
    pcg_iters_per_launch: int = 8   # fused kernel: PCG iterations per launch (> 1: no line-up per iteration)

    def parity(self) -> "SolverParams":
        """Tighter tolerances used when two implementations are compared."""
        p = SolverParams(**self.__dict__)
        p.newton_tol = 1e-7
        p.pcg_rel_tol = 1e-8
        p.pcg_max = 5000
        return p


@dataclass
class Scenario:
    scene: Scene
    params: SolverParams
    n_steps: int
    # delta(step) -> (n_bodies, 3) translation from rest placement at the END
    # of step `step` (0-based) for driven bodies; rows of free bodies ignored.
    delta: Callable[[int], np.ndarray]
    # optional initial velocities
    v0: Optional[np.ndarray] = None         # (N, 3)
    ydot0: Optional[np.ndarray] = None      # (n_bodies, 12)
    precision: int = 0                      # 0 = FP64, 1 = mixed


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def _orient(vx: np.ndarray, tet: list) -> list:
    a, b, c, d = (vx[i] for i in tet)
    if np.dot(np.cross(b - a, c - a), d - a) < 0.0:
        tet = [tet[0], tet[1], tet[3], tet[2]]
    return tet


_GRID_CACHE: dict = {}
_SPHERE_CACHE: dict = {}


def gel_grid(nx: int, ny: int, nz: int, size=(0.02, 0.02, 0.004),
             origin=None, pad_id: int = 0):
    """Cached front of `_gel_grid` (returns fresh copies)."""
    key = (nx, ny, nz, tuple(float(v) for v in size), None if origin is None else tuple(float(v) for v in origin))
    hit = _GRID_CACHE.get(key)
    if hit is None:
        hit = _gel_grid(nx, ny, nz, size, origin)
        _GRID_CACHE[key] = hit
    return tuple(a.copy() for a in hit)


def _gel_grid(nx: int, ny: int, nz: int, size=(0.02, 0.02, 0.004), origin=None):
    """Regular vertex grid, each hexahedron split into 5 tetrahedra.

    The split alternates with the parity of (i + j + k) so that face
    diagonals of neighbouring cells coincide and the mesh is conforming.
    Returns (x (N,3), tets (T,4) int32, bottom mask (N,) bool, top mask).
    Default placement: x, y centred on 0, top face at z = 0.
    """
    sx, sy, sz = size
    if origin is None:
        origin = (-sx / 2, -sy / 2, -sz)
    xs = origin[0] + np.linspace(0.0, sx, nx)
    ys = origin[1] + np.linspace(0.0, sy, ny)
    zs = origin[2] + np.linspace(0.0, sz, nz)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    vx = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * ny + j) * nz + k

    even_central = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    odd_central = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    tets = []
    for i in range(nx - 1):
        for j in range(ny - 1):
            for k in range(nz - 1):
                central = even_central if (i + j + k) % 2 == 0 else odd_central
                corners_out = odd_central if (i + j + k) % 2 == 0 else even_central
                c = lambda t: vid(i + t[0], j + t[1], k + t[2])
                tets.append(_orient(vx, [c(t) for t in central]))
                for o in corners_out:
                    # the three central corners adjacent to o differ in one axis
                    nb = [t for t in central
                          if sum(abs(t[m] - o[m]) for m in range(3)) == 1]
                    tets.append(_orient(vx, [c(o)] + [c(t) for t in nb]))
    tets = np.asarray(tets, dtype=np.int32)
    bottom = np.isclose(vx[:, 2], zs[0])
    top = np.isclose(vx[:, 2], zs[-1])
    return vx, tets, bottom, top


def icosphere(level: int, radius: float, center=(0.0, 0.0, 0.0)):
    """Icosahedron subdivided `level` times, vertices projected to the sphere.

    level 1/2/3/4 -> 42/162/642/2562 vertices.  Triangles are outward.
    The unit sphere of each level is built once and scaled.
    """
    hit = _SPHERE_CACHE.get(level)
    if hit is None:
        hit = _unit_icosphere(level)
        _SPHERE_CACHE[level] = hit
    verts, tris = hit
    return verts * radius + np.asarray(center, dtype=np.float64), tris.copy()


def _unit_icosphere(level: int):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    x = np.asarray(verts)
    tris = np.asarray(faces, dtype=np.int32)
    # make every face outward (centroid direction test)
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return x, tris


def box_surface(lo, hi):
    """Closed axis-aligned box surface: 8 vertices, 12 outward triangles."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x = np.array([[lo[0] if (i & 1) == 0 else hi[0],
                   lo[1] if (i & 2) == 0 else hi[1],
                   lo[2] if (i & 4) == 0 else hi[2]] for i in range(8)])
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4),
             (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    tris = np.asarray(tris, dtype=np.int32)
    ctr = 0.5 * (lo + hi)
    p0, p1, p2 = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", n, (p0 + p1 + p2) / 3.0 - ctr) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return x, tris


def _single_pad_scene(nx, ny, nz, E, nu, rho, bodies, name, size=(0.02, 0.02, 0.004)):
    x, tets, bottom, _ = gel_grid(nx, ny, nz, size=size)
    n = x.shape[0]
    return Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(n, np.int32),
                 pinned=bottom.copy(), attach=-np.ones(n, np.int32),
                 E=E, nu=nu, rho=rho, bodies=bodies, name=name)


def _press_slide(depth: float, slide: float, gap: float, n_press=50, n_slide=50):
    """Translation script: descend to `depth` below the top, then slide in +x."""
    def delta(step: int) -> np.ndarray:
        s = step + 1
        dz = -(gap + depth) * min(s, n_press) / n_press
        dx = slide * max(0, min(s - n_press, n_slide)) / n_slide
        return np.array([[dx, 0.0, dz]])
    return delta


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------
def config0() -> Scenario:
    """Gel 9x9x3 (20x20x4 mm) + 8 mm ABD cube driven down at 5 mm/s, 20 steps."""
    gap = 5e-5
    s = 8e-3
    bx, bt = box_surface((-s / 2, -s / 2, gap), (s / 2, s / 2, gap + s))
    body = Body(rest_x=bx, tris=bt, rho=1200.0, kappa_s=1e8, driven=True)
    scene = _single_pad_scene(9, 9, 3, 3e5, 0.45, 1000.0, [body], "config0")
    params = SolverParams()
    speed = 5e-3

    def delta(step):
        return np.array([[0.0, 0.0, -speed * params.dt * (step + 1)]])
    return Scenario(scene=scene, params=params, n_steps=20, delta=delta)


def config1(env: int, nx=40, ny=40, nz=6, n_steps=100) -> Scenario:
    """Gel 40x40x6 + driven icosphere (level 2, r = 4 mm), seeded press/slide."""
    rng = np.random.default_rng(1000 + env)
    depth = rng.uniform(0.0, 1.5e-3)
    slide = rng.uniform(-2e-3, 2e-3)
    gap = 5e-5
    r = 4e-3
    sx, st = icosphere(2, r)
    sx[:, 2] += gap - sx[:, 2].min()
    body = Body(rest_x=sx, tris=st, rho=1200.0, kappa_s=1e8, driven=True)
    scene = _single_pad_scene(nx, ny, nz, 3e5, 0.45, 1000.0, [body], f"config1[{env}]")
    half = n_steps // 2
    return Scenario(scene=scene, params=SolverParams(), n_steps=n_steps,
                    delta=_press_slide(depth, slide, gap, half, n_steps - half))


def config2(env: int, n_steps=100) -> Scenario:
    """Uneven batch member: gel {16,24,32,48}^2 x {4,6}, E~U(1e5,5e5),
    icosphere level U{1..3}, radius U(3,8) mm, seeded press/slide."""
    rng = np.random.default_rng(2000 + env)
    nxy = int(rng.choice([16, 24, 32, 48]))
    nz = int(rng.choice([4, 6]))
    E = float(rng.uniform(1e5, 5e5))
    level = int(rng.integers(1, 4))
    r = float(rng.uniform(3e-3, 8e-3))
    depth = rng.uniform(0.0, 1.5e-3)
    slide = rng.uniform(-2e-3, 2e-3)
    gap = 5e-5
    sx, st = icosphere(level, r)
    sx[:, 2] += gap - sx[:, 2].min()
    body = Body(rest_x=sx, tris=st, rho=1200.0, kappa_s=1e8, driven=True)
    scene = _single_pad_scene(nxy, nxy, nz, E, 0.45, 1000.0, [body], f"config2[{env}]")
    params = SolverParams()
    half = n_steps // 2
    return Scenario(scene=scene, params=params, n_steps=n_steps,
                    delta=_press_slide(depth, slide, gap, half, n_steps - half),
                    precision=1)


def config4_request(req: int, n_steps=200) -> Scenario:
    """One request of the serving stream: a config-2-style env drawn from
    its own seed (default_rng(5000 + req)) with the same distribution:
    gel {16,24,32,48}^2 x {4,6}, E ~ U(1e5, 5e5), icosphere level U{1..3},
    radius U(3, 8) mm, press U(0, 1.5) mm then slide U(-2, 2) mm."""
    rng = np.random.default_rng(5000 + req)
    nxy = int(rng.choice([16, 24, 32, 48]))
    nz = int(rng.choice([4, 6]))
    E = float(rng.uniform(1e5, 5e5))
    level = int(rng.integers(1, 4))
    r = float(rng.uniform(3e-3, 8e-3))
    depth = rng.uniform(0.0, 1.5e-3)
    slide = rng.uniform(-2e-3, 2e-3)
    gap = 5e-5
    sx, st = icosphere(level, r)
    sx[:, 2] += gap - sx[:, 2].min()
    body = Body(rest_x=sx, tris=st, rho=1200.0, kappa_s=1e8, driven=True)
    scene = _single_pad_scene(nxy, nxy, nz, E, 0.45, 1000.0, [body], f"request[{req}]")
    half = n_steps // 2
    return Scenario(scene=scene, params=SolverParams(), n_steps=n_steps,
                    delta=_press_slide(depth, slide, gap, half, n_steps - half), precision=1)


def config3(env: int, n=32, nz=6, n_steps=200, level=4, gap=None) -> Scenario:
    """Two gel pads on ABD fingers closing at 10 mm/s on a free icosphere.

    Pads are 20x20x4 mm with their contact faces normal to x; each pad's back
    face is attached to a 22x22x4 mm finger box behind it.  The object is a
    free icosphere (r = 10 mm, rho = 800) under gravity.  The initial gap
    between each pad and the sphere is 20 um + U(0, 20) um, or `gap` when
    given: at 10 um per step the pads reach the sphere within 2-4 steps,
    before it has fallen 0.1 mm (a gap of a millimetre would let it fall out
    of the 20 mm pads before they close).
    """
    rng = np.random.default_rng(3000 + env)
    r = 10e-3
    gap0 = 2e-5 + rng.uniform(0.0, 2e-5)
    if gap is not None:
        gap0 = float(gap)
    thick = 4e-3
    xs, ys, zs = [], [], []
    parts_x, parts_t, obj, pinned, attach = [], [], [], [], []
    off = 0
    bodies = []
    for side, sgn in enumerate((-1.0, 1.0)):
        # pad occupies |x| in [r + gap0, r + gap0 + thick]; build in z then rotate
        x, tets, bottom, top = gel_grid(n, n, nz, size=(0.02, 0.02, thick))
        # local z in [-thick, 0] (top at 0).  Map local (u, v, w) -> world
        # contact face (w = 0) at x = sgn * (r + gap0), back face farther out.
        w = x[:, 2]
        X = np.stack([sgn * (r + gap0 - w), x[:, 0], x[:, 1]], axis=1)
        # the map to world coordinates mirrors one pad: re-orient every tet
        tt = []
        for q in tets:
            tt.append(_orient(X, list(q)))
        tt = np.asarray(tt, np.int32)
        parts_x.append(X)
        parts_t.append(tt + off)
        obj.append(np.full(X.shape[0], side, np.int32))
        pinned.append(np.zeros(X.shape[0], bool))
        att = -np.ones(X.shape[0], np.int32)
        att[bottom] = side
        attach.append(att)
        off += X.shape[0]
        # finger box behind the pad
        xb0 = sgn * (r + gap0 + thick)
        lo = (min(xb0, xb0 + sgn * 4e-3), -0.011, -0.011)
        hi = (max(xb0, xb0 + sgn * 4e-3), 0.011, 0.011)
        fx, ft = box_surface(lo, hi)
        bodies.append(Body(rest_x=fx, tris=ft, rho=1200.0, kappa_s=1e8, driven=True))
    ox, ot = icosphere(level, r)
    bodies.append(Body(rest_x=ox, tris=ot, rho=800.0, kappa_s=1e8, driven=False))
    scene = Scene(gel_x=np.concatenate(parts_x), gel_tets=np.concatenate(parts_t),
                  gel_obj=np.concatenate(obj), pinned=np.concatenate(pinned),
                  attach=np.concatenate(attach), E=3e5, nu=0.45, rho=1000.0,
                  bodies=bodies, name=f"config3[{env}]")
    params = SolverParams()
    speed = 10e-3

    def delta(step):
        d = speed * params.dt * (step + 1)
        return np.array([[d, 0.0, 0.0], [-d, 0.0, 0.0], [0.0, 0.0, 0.0]])
    return Scenario(scene=scene, params=params, n_steps=n_steps, delta=delta, precision=1)


# ----------------------------------------------------------------------------
# small scenes used by tests
# ----------------------------------------------------------------------------
def small_contact_scene(nx=5, ny=5, nz=3, body="cube", level=1, radius=2e-3,
                        size=(0.01, 0.01, 0.002), gap=5e-5, driven=True,
                        depth=3e-4, n_steps=6) -> Scenario:
    """A small gel with one driven (or free, falling) body just above it."""
    if body == "cube":
        s = 4e-3
        bx, bt = box_surface((-s / 2 + 3e-4, -s / 2 + 2e-4, gap), (s / 2 + 3e-4, s / 2 + 2e-4, gap + s))
    else:
        bx, bt = icosphere(level, radius)
        bx[:, 2] += gap - bx[:, 2].min()
        bx[:, 0] += 3e-4
        bx[:, 1] += 1e-4
    b = Body(rest_x=bx, tris=bt, rho=1200.0, kappa_s=1e8, driven=driven)
    scene = _single_pad_scene(nx, ny, nz, 3e5, 0.45, 1000.0, [b], "small", size=size)
    params = SolverParams()

    def delta(step):
        return np.array([[0.0, 0.0, -(gap + depth) * min(step + 1, n_steps) / n_steps]])
    return Scenario(scene=scene, params=params, n_steps=n_steps, delta=delta)


def self_contact_scene(nx=5, ny=5, nz=2, nu_xy=4, gap=5e-5, depth=1e-4, n_steps=4,
                       self_contact=True, with_body=True) -> Scenario:
    """Gel self-contact: one pad made of two blocks, a pinned 10x10x2 mm base
    and a free 6x6x2 mm block resting `gap` above it (slightly offset so that
    no vertices line up), pressed onto the base by a driven 3 mm cube.  Both
    blocks are the same pad, so the contact between them exists only as
    self-contact of the pad."""
    xl, tl, bl, _ = gel_grid(nx, ny, nz, size=(0.01, 0.01, 0.002))
    xu, tu, _, _ = gel_grid(nu_xy, nu_xy, nz, size=(0.006, 0.006, 0.002),
                            origin=(-0.003 + 3e-4, -0.003 + 1e-4, gap))
    x = np.concatenate([xl, xu])
    tets = np.concatenate([tl, tu + xl.shape[0]]).astype(np.int32)
    n = x.shape[0]
    pinned = np.concatenate([bl, np.zeros(xu.shape[0], bool)])
    bodies = []
    if with_body:
        s3, z0 = 3e-3, gap + 0.002 + gap
        bx, bt = box_surface((-s3 / 2 + 2e-4, -s3 / 2 + 3e-4, z0), (s3 / 2 + 2e-4, s3 / 2 + 3e-4, z0 + s3))
        bodies.append(Body(rest_x=bx, tris=bt, rho=1200.0, kappa_s=1e8, driven=True))
    scene = Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(n, np.int32), pinned=pinned,
                  attach=-np.ones(n, np.int32), E=3e5, nu=0.45, rho=1000.0, bodies=bodies,
                  name="self_contact", self_contact=np.array([bool(self_contact)]))
    params = SolverParams()

    def delta(step):
        return np.array([[0.0, 0.0, -(2 * gap + depth) * min(step + 1, n_steps) / n_steps]])[:len(bodies)]
    return Scenario(scene=scene, params=params, n_steps=n_steps, delta=delta)


def free_fall_scene(nx=4, ny=4, nz=3, with_body=True, pinned=False, v0=(0.1, -0.2, 0.3)):
    """Gel (optionally unpinned) and a free cube far apart: no contact."""
    x, tets, bottom, _ = gel_grid(nx, ny, nz, size=(0.006, 0.006, 0.002))
    n = x.shape[0]
    bodies = []
    if with_body:
        bx, bt = box_surface((0.02, 0.02, 0.02), (0.024, 0.025, 0.026))
        bodies.append(Body(rest_x=bx, tris=bt, rho=1200.0, kappa_s=1e8, driven=False))
    scene = Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(n, np.int32),
                  pinned=bottom.copy() if pinned else np.zeros(n, bool),
                  attach=-np.ones(n, np.int32), E=3e5, nu=0.45, rho=1000.0,
                  bodies=bodies, name="free_fall")
    params = SolverParams()
    v = np.tile(np.asarray(v0, dtype=np.float64), (n, 1))
    yd = None
    if with_body:
        yd = np.zeros((1, 12))
        yd[0, :3] = v0
    return Scenario(scene=scene, params=params, n_steps=5,
                    delta=lambda s: np.zeros((len(bodies), 3)), v0=v, ydot0=yd)


def spin_scene(omega=(0.0, 0.0, 20.0)):
    """A lone free cube spinning about its centre (no gel contact)."""
    x, tets, bottom, _ = gel_grid(3, 3, 2, size=(0.004, 0.004, 0.002))
    n = x.shape[0]
    bx, bt = box_surface((0.05, 0.05, 0.05), (0.058, 0.058, 0.058))
    body = Body(rest_x=bx, tris=bt, rho=1200.0, kappa_s=1e8, driven=False)
    scene = Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(n, np.int32),
                  pinned=bottom.copy(), attach=-np.ones(n, np.int32),
                  E=3e5, nu=0.45, rho=1000.0, bodies=[body], name="spin")
    params = SolverParams(gravity=(0.0, 0.0, 0.0))
    w = np.asarray(omega, dtype=np.float64)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    yd = np.zeros((1, 12))
    # dA/dt = W A at A = I: columns of W
    yd[0, 3:6] = W[:, 0]
    yd[0, 6:9] = W[:, 1]
    yd[0, 9:12] = W[:, 2]
    return Scenario(scene=scene, params=params, n_steps=10,
                    delta=lambda s: np.zeros((1, 3)), ydot0=yd)


def config3_batch(n_envs: int, n=32, nz=6, n_steps=200, level=4):
    """Config 3 as a batch that shares one scene: the geometry of config3(0)
    at the mean gap, and per env the initial gap of config3(env) applied as
    an opposite rigid shift of each finger with its pad along x (the rest
    shape of a pad does not depend on where it is placed).  Returns (scene,
    params, per-env (shift of pad 0, shift of pad 1) along x, delta)."""
    mean_gap = 3e-5
    base = config3(0, n, nz, n_steps, level, gap=mean_gap)
    shifts = []
    for env in range(n_envs):
        rng = np.random.default_rng(3000 + env)
        g = 2e-5 + rng.uniform(0.0, 2e-5)
        shifts.append((-(g - mean_gap), g - mean_gap))
    return base.scene, base.params, shifts, base.delta


def self_contact_pad(n: int, nz: int = 3) -> Scene:
    """One free-standing n x n x nz gel pad (20 x 20 x 4 mm, bottom pinned)
    flagged for self-contact, no bodies: a candidate-search workload."""
    x, tets, bottom, _ = gel_grid(n, n, nz)
    N = x.shape[0]
    return Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(N, np.int32), pinned=bottom.copy(),
                 attach=-np.ones(N, np.int32), E=3e5, nu=0.45, rho=1000.0, bodies=[],
                 name=f"self_contact_pad[{n}]", self_contact=np.array([True]))


def pad_and_sphere(n: int, nz: int, level: int, r: float = 10e-3) -> Scene:
    """An n x n x nz pad with a free icosphere resting 20 um above its top:
    a candidate-search workload for a large object."""
    x, tets, bottom, _ = gel_grid(n, n, nz)
    N = x.shape[0]
    sx, st = icosphere(level, r)
    sx[:, 2] += 2e-5 - sx[:, 2].min()
    body = Body(rest_x=sx, tris=st, rho=800.0, kappa_s=1e8, driven=False)
    return Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(N, np.int32), pinned=bottom.copy(),
                 attach=-np.ones(N, np.int32), E=3e5, nu=0.45, rho=1000.0, bodies=[body],
                 name=f"pad_and_sphere[{n},{level}]")


def config1_batch(n_envs: int, nx=40, ny=40, nz=6, n_steps=100):
    """Config 1 as a batch: one shared scene (identical geometry in every env)
    and the per-env seeded press/slide scripts of config1(env)."""
    base = config1(0, nx, ny, nz, n_steps)
    deltas = []
    half = n_steps // 2
    for env in range(n_envs):
        rng = np.random.default_rng(1000 + env)
        depth = rng.uniform(0.0, 1.5e-3)
        slide = rng.uniform(-2e-3, 2e-3)
        deltas.append(_press_slide(depth, slide, 5e-5, half, n_steps - half))
    return base.scene, base.params, deltas
