"""The step's output: the coated surface of the gel (test infrastructure).

Sec. 4.1 ("Tactile Sensors Modeling") splits the boundary of a gel pad into
the part attached to the sensor body and the coated part that touches the
world; the simulator's visible output is the deformed coated surface, on
which Sec. 4.2 places markers and reads depth.  Here the coated surface of an
environment's gel is every boundary vertex of its tetrahedral mesh that is
neither pinned (a pad's face resting on a fixed support) nor attached to a
body, listed in increasing gel vertex id; its output is those vertices'
positions in that order.

Only the tests use this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from .rest import boundary_faces


def coated_vertices(scene) -> np.ndarray:
    """Gel vertex ids of the coated surface, increasing (Sec. 4.1: the gel
    boundary minus its fixed and attached parts)."""
    on_boundary = np.zeros(scene.n_verts, bool)
    on_boundary[boundary_faces(np.asarray(scene.gel_tets)).ravel()] = True
    keep = on_boundary & ~np.asarray(scene.pinned, bool) & (np.asarray(scene.attach) < 0)
    return np.nonzero(keep)[0]


def coated_surface(scene, x: np.ndarray) -> np.ndarray:
    """Positions [n][3] of the coated-surface vertices of gel state x [N][3]."""
    return np.asarray(x, np.float64)[coated_vertices(scene)]
