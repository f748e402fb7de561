"""GPU parity of the step's output, the coated surface (Sec. 4.1, Sec. 4.2):
the library's read-back against the oracle's coated-vertex list and the
oracle's stepped state.

Which vertices are output and in which order is index work: compared exactly
(the read-back rows equal the GPU state's own rows at the oracle's coated ids,
bit for bit).  The positions themselves follow the per-step FP64 bar, 1e-6 of
the scene's bounding-box diagonal, against the oracle stepped from the same
input at the parity tolerances."""
import numpy as np
import pytest

import scenes
from oracle.output import coated_surface, coated_vertices

from gpu_util import bbox_diag, gpu_targets, oracle_states, to_gpu_y

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402

build()


def _check_scene(sc, n_steps):
    prm = sc.params.parity()
    oenv, traj = oracle_states(sc, prm, n_steps)
    idx = coated_vertices(sc.scene)
    # one env alone, then the same scene beside a different one (the rows of
    # the batched read-back are env after env)
    other = scenes.config0().scene
    for batch in ([sc.scene], [other, sc.scene]):
        genv = ipc.Envs(batch, prm)
        e = len(batch) - 1
        assert genv.sizes[e][2] == len(idx)
        for s in range(n_steps):
            x, v, y, yd, sy = traj[s]
            xo, _, yo, _, _ = traj[s + 1]
            assert genv.set_state(e, x, v, to_gpu_y(genv, e, oenv, y), yd) == ipc.IPC_OK
            genv.set_targets(e, gpu_targets(genv, e, oenv, sy))
            status, _ = genv.step([e])
            assert status[0] == ipc.IPC_OK
            xg = genv.get_state(e)[0]
            one = genv.read_gel_surface(e)
            every = genv.read_gel_surface_all()
            off = sum(genv.sizes[k][2] for k in range(e))
            # the output set and order: exactly the oracle's coated vertices
            assert np.array_equal(one, xg[idx])
            assert np.array_equal(every[off:off + len(idx)], one)
            # the positions: the oracle's stepped coated surface
            err = np.abs(one - coated_surface(sc.scene, xo)).max() / bbox_diag(oenv, x, y)
            assert err <= 1e-6, (s, err)
        genv.close()


def test_coated_surface_config0():
    _check_scene(scenes.config0(), 3)


def test_coated_surface_attached_pads():
    # two pads whose back faces are attached to the finger bodies: attached
    # vertices are not part of the output
    _check_scene(scenes.config3(0, n=5, nz=3, level=1, gap=2e-5), 2)
