"""Pins of the tactile oracle (Sec. 4.2): boundary extraction against the
box's closed-form surface, depth / normal maps against rest, rigid-sink and
planar-tilt closed forms, markers against affine maps."""
import numpy as np
import pytest

import scenes
from oracle import tactile as tc

PITCH = 0.5e-3


def _gel():
    sc = scenes.config0()
    s = sc.scene
    coated = ~s.pinned & (s.attach < 0)
    return s, coated


def test_boundary_faces_cover_the_box_surface_outward():
    x, tets, _, _ = scenes.gel_grid(5, 4, 3, size=(0.02, 0.01, 0.004))
    F = tc.boundary_faces(tets, x)
    assert len(F) == 2 * 2 * ((5 - 1) * (4 - 1) + (5 - 1) * (3 - 1) + (4 - 1) * (3 - 1))
    a = np.cross(x[F[:, 1]] - x[F[:, 0]], x[F[:, 2]] - x[F[:, 0]])
    area = 0.5 * np.linalg.norm(a, axis=1)
    assert area.sum() == pytest.approx(2 * (0.02 * 0.01 + 0.02 * 0.004 + 0.01 * 0.004), rel=1e-12)
    centre = 0.5 * (x.max(0) + x.min(0))
    cent = x[F].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", a, cent - centre) > 0)        # outward everywhere


def test_front_triangles_tile_the_top_face():
    s, coated = _gel()
    T = tc.front_triangles(s.gel_tets, s.gel_x, coated, s.gel_obj, 0, np.array([0.0, 0.0, 1.0]))
    a = 0.5 * np.linalg.norm(np.cross(s.gel_x[T[:, 1]] - s.gel_x[T[:, 0]], s.gel_x[T[:, 2]] - s.gel_x[T[:, 0]]), axis=1)
    assert a.sum() == pytest.approx(0.02 * 0.02, rel=1e-12)
    assert np.allclose(s.gel_x[T][:, :, 2], 0.0)


def _maps(x, s, coated):
    T = tc.front_triangles(s.gel_tets, s.gel_x, coated, s.gel_obj, 0, np.array([0.0, 0.0, 1.0]))
    n = int(round(0.02 / PITCH))
    return tc.depth_normal_map(x, T, (-0.01, -0.01, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1), PITCH, n, n)


def test_depth_map_at_rest_and_after_a_rigid_sink():
    s, coated = _gel()
    d, nrm, hit = _maps(s.gel_x, s, coated)
    assert hit.all() and np.all(d == 0.0)
    assert np.allclose(nrm, [0.0, 0.0, 1.0], atol=1e-15)
    delta = 3.7e-5
    d2, nrm2, hit2 = _maps(s.gel_x - np.array([0.0, 0.0, delta]), s, coated)
    assert hit2.all() and np.allclose(d2, delta, rtol=0, atol=1e-18)
    assert np.allclose(nrm2, [0.0, 0.0, 1.0], atol=1e-15)


def test_depth_of_a_planar_tilt_is_the_plane_at_every_pixel():
    s, coated = _gel()
    a, b = 1.3e-3, -0.7e-3
    x = s.gel_x.copy()
    top = np.isclose(x[:, 2], 0.0)
    x[top, 2] += a * x[top, 0] + b * x[top, 1]
    d, nrm, hit = _maps(x, s, coated)
    n = d.shape[0]
    cx = -0.01 + (np.arange(n) + 0.5) * PITCH
    X, Y = np.meshgrid(cx, cx)                      # rows follow v (= y), columns u (= x)
    assert hit.all()
    assert np.allclose(d, -(a * X + b * Y), rtol=0, atol=1e-18)
    nz = np.array([-a, -b, 1.0]) / np.linalg.norm([-a, -b, 1.0])
    assert np.allclose(nrm, nz, atol=1e-12)


def test_markers_follow_affine_maps_and_sit_on_vertices_at_corners():
    s, coated = _gel()
    T = tc.front_triangles(s.gel_tets, s.gel_x, coated, s.gel_obj, 0, np.array([0.0, 0.0, 1.0]))
    rng = np.random.default_rng(3)
    k = rng.integers(0, len(T), 50)
    bary = rng.dirichlet([1, 1, 1], 50)
    bary[0] = [1.0, 0.0, 0.0]
    p = tc.marker_positions(s.gel_x, T[k], bary)
    assert np.array_equal(p[0], s.gel_x[T[k[0], 0]])
    A = np.eye(3) + 1e-2 * rng.normal(size=(3, 3))
    t = np.array([1e-4, -2e-4, 3e-5])
    q = tc.marker_positions(s.gel_x @ A.T + t, T[k], bary)
    assert np.allclose(q, p @ A.T + t, rtol=0, atol=1e-15)
