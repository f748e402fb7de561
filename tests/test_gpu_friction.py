"""Lagged IPC friction on the GPU against the oracle (App. A.3,
D_k = mu lambda_k^n f0(|u_k|)): per-step positions from the same input state
at the parity tolerances, and the sliding-cube closed form."""
import numpy as np
import pytest

import scenes
from oracle import OracleEnv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from gpu_util import all_points, bbox_diag, from_gpu_y, gpu_targets, oracle_states, to_gpu_y  # noqa: E402
from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402

build()


def _press_and_slide():
    """A driven cube pressed 0.1 mm into the gel, then dragged along x."""
    sc = scenes.small_contact_scene(body="cube", gap=2e-5, depth=1e-4, n_steps=3)
    press = sc.delta

    def delta(k):
        dl = press(k).copy()
        dl[0, 0] = 3e-5 * max(0, k - 2)                  # 30 um per step from step 3
        return dl
    sc.delta = delta
    return sc


@pytest.mark.parametrize("mu", [0.5])
def test_friction_step_parity_with_oracle(mu):
    sc = _press_and_slide()
    prm = sc.params.parity()
    prm.friction_mu = mu
    n = 6
    oenv, traj = oracle_states(sc, prm, n)
    genv = ipc.Envs([sc.scene], prm)
    for s in range(n):
        x, v, y, yd, sy = traj[s]
        xo, vo, yo, ydo, _ = traj[s + 1]
        assert genv.set_state(0, x, v, to_gpu_y(genv, 0, oenv, y), yd) == ipc.IPC_OK
        genv.set_targets(0, gpu_targets(genv, 0, oenv, sy))
        status, _ = genv.step()
        assert status[0] == ipc.IPC_OK
        xg, vg, yg, ydg = genv.get_state(0)
        yg = from_gpu_y(genv, 0, oenv, yg)
        err = np.abs(all_points(oenv, xg, yg) - all_points(oenv, xo, yo)).max() / bbox_diag(oenv, x, y)
        assert err <= 1e-6, (s, err)
    # friction acted: the last step without friction ends elsewhere
    p0 = sc.params.parity()
    x, v, y, yd, sy = traj[n - 1]
    x0, _, y0, _, _ = OracleEnv(sc.scene, p0).step(x, v, y, yd, sy)
    moved = np.abs(all_points(oenv, x0, y0) - all_points(oenv, traj[n][0], traj[n][2])).max()
    assert moved > 1e-4 * bbox_diag(oenv, x, y)
    genv.close()


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_gpu_sliding_cube_decelerates_at_mu_g(mu):
    sc = scenes.small_contact_scene(body="cube", driven=False, gap=5e-5)
    sc.scene.E = 1e7
    prm = sc.params
    prm.friction_mu = mu
    prm.newton_tol = 1e-6
    prm.pcg_rel_tol = 1e-8
    prm.pcg_max = 5000
    genv = ipc.Envs([sc.scene], prm)
    for _ in range(15):
        st, _ = genv.step()
        assert st[0] == 0
    x, v, y, yd = genv.get_state(0)
    yd[0, 0] = 0.2
    assert genv.set_state(0, x, v, y, yd) == ipc.IPC_OK
    vs = [0.2]
    for _ in range(8):
        st, _ = genv.step()
        assert st[0] == 0
        vs.append(genv.get_state(0)[3][0, 0])
    a = (vs[-1] - vs[0]) / (8 * prm.dt)
    assert a == pytest.approx(-mu * 9.81, abs=0.1 * 9.81 * max(mu, 0.05))
    genv.close()
