"""Pins of the oracle's coated-surface output (Sec. 4.1, Sec. 4.2): closed-form
counts of grid meshes and a membership test by coordinates that does not go
through the mesh's boundary faces."""
import numpy as np

import scenes
from oracle.output import coated_surface, coated_vertices


def _grid_count(nx, ny, nz):
    # boundary vertices of an nx x ny x nz vertex grid, minus the pinned bottom layer
    return nx * ny * nz - (nx - 2) * (ny - 2) * (nz - 2) - nx * ny


def test_config0_count():
    sc = scenes.config0().scene
    assert sc.n_verts == 243
    assert len(coated_vertices(sc)) == 194 - 81 == _grid_count(9, 9, 3)


def test_config1_count():
    sc = scenes.config1(0).scene
    assert sc.n_verts == 9600
    assert len(coated_vertices(sc)) == 3824 - 1600 == 2224 == _grid_count(40, 40, 6)


def test_membership_by_coordinates_and_order():
    # a box grid: a vertex is on the boundary iff a coordinate sits at the
    # box's min or max; coated iff also not on the pinned bottom face
    for env in (0, 3, 5):
        sc = scenes.config2(env).scene
        x = sc.gel_x
        lo, hi = x.min(axis=0), x.max(axis=0)
        tol = 1e-12
        on_face = np.any((np.abs(x - lo) < tol) | (np.abs(x - hi) < tol), axis=1)
        bottom = np.abs(x[:, 2] - lo[2]) < tol
        assert np.array_equal(bottom, sc.pinned)
        want = np.nonzero(on_face & ~bottom)[0]
        got = coated_vertices(sc)
        assert np.array_equal(got, want)
        assert np.all(np.diff(got) > 0)


def test_attached_vertices_are_not_coated():
    # two-finger grasp: each pad's back face is attached to its finger body
    sc = scenes.config3(0, n=6, nz=3, level=1).scene
    got = set(coated_vertices(sc).tolist())
    att = set(np.nonzero(sc.attach >= 0)[0].tolist())
    assert att and not (got & att)
    # per pad: boundary of a 6x6x3 grid minus one 6x6 face
    assert len(got) == 2 * (6 * 6 * 3 - 4 * 4 * 1 - 6 * 6)


def test_output_is_the_positions_of_those_vertices():
    sc = scenes.config0().scene
    rng = np.random.default_rng(3)
    x = sc.gel_x + rng.normal(scale=1e-6, size=sc.gel_x.shape)
    out = coated_surface(sc, x)
    idx = coated_vertices(sc)
    assert out.shape == (len(idx), 3)
    assert np.array_equal(out, x[idx])
