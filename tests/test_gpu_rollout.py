"""ipc_rollout: n steps of every env inside one device loop, each env on its
own schedule.  Per env it runs the same computation as n calls of ipc_step
(App. A.2, one time step after another), so the tests hold it to the
lock-step path: the same end state within the FP64 multi-step bar (1e-6 of
the bbox diagonal per step; contact sums use atomics, so the two orders
differ in the last bits every step), the same statuses, and the same
failure behaviour."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402

build()

K = 4


def _batch():
    # an uneven batch: config-2 envs of different gel and sphere sizes,
    # pressing into contact within the K steps
    return [scenes.config2(e, n_steps=12) for e in (0, 1, 2, 5)]


def _table(genv, scs, k0, n):
    mb = max(genv.max_bodies, 1)
    t = np.zeros((n, len(scs), mb, 12))
    for k in range(n):
        for e, sc in enumerate(scs):
            y = genv.rest_y(e)
            y[:, :3] += np.asarray(sc.delta(k0 + k)).reshape(-1, 3)[: y.shape[0]]
            t[k, e, : y.shape[0]] = y
    return t


def _lockstep(scs, prm, n, stream=None):
    g = ipc.Envs([sc.scene for sc in scs], prm, stream=stream)
    tab = _table(g, scs, 0, n)
    st_all = np.zeros(len(scs), np.int32)
    g.act_pair_iters = 0
    for k in range(n):
        g.set_targets_all(tab[k])
        st, s = g.step()
        g.act_pair_iters += s["act_pair_iters"]
        st_all = np.where(st_all == 0, st, st_all)
    return g, st_all


def _states(g, n):
    return [g.get_state(e) for e in range(n)]


def _assert_close(sa, sb, n_steps, bound=1e-6):
    for e, (a, b) in enumerate(zip(sa, sb)):
        diag = float(np.linalg.norm(a[0].max(0) - a[0].min(0)))
        tol = bound * n_steps * diag
        assert np.abs(a[0] - b[0]).max() <= tol, (e, np.abs(a[0] - b[0]).max() / diag)
        assert np.abs(a[2][:, :3] - b[2][:, :3]).max() <= tol, e


@pytest.mark.parametrize("profiled,window", [(False, 64), (False, 2), (False, 0), (True, 64)])
def test_rollout_matches_lockstep_steps(profiled, window):
    """K steps of an uneven batch: as a rollout (one graph, or the same loop
    as plain launches when profiling) and as K ipc_step calls.  window: PCG
    iterations per loop iteration (solves carried over between loop
    iterations; 2 carries nearly every solve many times, 0 carries none)."""
    scs = _batch()
    prm = scenes.SolverParams().parity()
    prm.rollout_pcg_window = window
    ga, st_a = _lockstep(scs, prm, K)
    assert np.all(st_a == 0)
    gb = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    if profiled:
        gb.profile_enable(True)
    tab = torch.as_tensor(_table(gb, scs, 0, K), device="cuda")
    st, steps, stats = gb.rollout(K, tab)
    assert np.all(st == 0) and np.all(steps == K)
    assert stats["newton_env_iters"] > 0 and stats["pcg_iters"] > 0 and stats["max_pairs"] > 0
    # the contact mat-vec work: active pairs (at most the candidates) per PCG
    # iteration, summed like the lock-step steps' (iteration counts may differ
    # by a few where the atomics' order moves a residual across the tolerance)
    assert 0 < stats["act_pair_iters"] <= stats["pcg_iters"] * stats["max_pairs"]
    assert abs(stats["act_pair_iters"] - ga.act_pair_iters) <= 0.05 * ga.act_pair_iters
    _assert_close(_states(ga, len(scs)), _states(gb, len(scs)), K)
    if profiled:
        prof = gb.profile()
        assert prof["pcg_iter"][0] > 0 or prof["pcg_matvec"][0] > 0
    ga.close()
    gb.close()


def test_rollout_subset_async_and_repeat():
    """A rollout over a subset (enqueued, results read later) leaves the other
    envs untouched; a second rollout continues from where the first ended,
    like two rounds of ipc_step."""
    scs = _batch()
    prm = scenes.SolverParams().parity()
    gb = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    before = _states(gb, len(scs))
    tab = torch.as_tensor(_table(gb, scs, 0, 2), device="cuda")
    assert gb.rollout(2, tab, env_ids=[1, 3], wait=False) is None
    st, steps, stats = gb.rollout_results()
    assert np.all(st == 0) and np.all(steps == 2)
    after = _states(gb, len(scs))
    for e in (0, 2):
        for a, b in zip(before[e], after[e]):
            assert np.array_equal(a, b)
    tab2 = torch.as_tensor(_table(gb, scs, 2, 2), device="cuda")
    st, steps, _ = gb.rollout(2, tab2, env_ids=[1, 3])
    assert np.all(st == 0) and np.all(steps == 2)
    ga, st_a = _lockstep(scs, prm, K)
    la, lb = _states(ga, len(scs)), _states(gb, len(scs))
    _assert_close([la[1], la[3]], [lb[1], lb[3]], K)
    ga.close()
    gb.close()


def test_rollout_stops_an_env_at_its_failing_step():
    """With a Newton cap too small for contact steps every env fails
    (IPC_ENOTCONV) at some step and stops there: its status, its step count
    and its state are those of the lock-step run stopped at the same step."""
    scs = _batch()
    prm = scenes.SolverParams().parity()
    prm.newton_max = 3
    ga = ipc.Envs([sc.scene for sc in scs], prm)
    tab = _table(ga, scs, 0, K)
    first_fail = np.full(len(scs), -1)
    code = np.zeros(len(scs), np.int32)
    snap = {}
    for k in range(K):
        live = [e for e in range(len(scs)) if first_fail[e] < 0]
        if not live:
            break
        ga.set_targets_all(tab[k])
        st, _ = ga.step(live)
        for j, e in enumerate(live):
            if st[j] != 0:
                first_fail[e], code[e] = k, st[j]
                snap[e] = ga.get_state(e)
    assert np.any(first_fail >= 0)                 # the cap bites
    gb = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    st, steps, _ = gb.rollout(K, torch.as_tensor(tab, device="cuda"))
    for e in range(len(scs)):
        if first_fail[e] >= 0:
            assert st[e] == code[e] and steps[e] == first_fail[e] + 1, (e, st[e], steps[e], first_fail[e])
            _assert_close([snap[e]], [gb.get_state(e)], first_fail[e] + 1)
        else:
            assert st[e] == 0 and steps[e] == K
    ga.close()
    gb.close()


def test_rollout_zero_steps_and_bad_table():
    scs = _batch()[:2]
    prm = scenes.SolverParams()
    gb = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    before = _states(gb, 2)
    st, steps, stats = gb.rollout(0, None)
    assert np.all(steps == 0) and stats["newton_env_iters"] == 0
    for a, b in zip(before, _states(gb, 2)):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    with pytest.raises(ValueError):
        gb.rollout(2, torch.zeros((3, 2, 1, 12), dtype=torch.float64, device="cuda"))
    with pytest.raises(ipc.IpcError):   # driven bodies need a table
        gb.rollout(2, None)
    gb.close()


def test_rollout_per_env_step_limits():
    """steps_per_env caps each env's steps: env i ends where i lock-step
    steps end, the envs with more steps go on."""
    scs = _batch()
    prm = scenes.SolverParams().parity()
    gb = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    tab = torch.as_tensor(_table(gb, scs, 0, 3), device="cuda")
    st, steps, _ = gb.rollout(3, tab, steps_per_env=[0, 1, 3, 2])
    assert np.all(st == 0) and list(steps) == [0, 1, 3, 2]
    for e, n in enumerate([0, 1, 3, 2]):
        ga, st_a = _lockstep([scs[e]], prm, n) if n else (ipc.Envs([scs[e].scene], prm), np.zeros(1))
        _assert_close([ga.get_state(0)], [gb.get_state(e)], max(n, 1))
        ga.close()
    with pytest.raises(ipc.IpcError):
        gb.rollout(3, tab, steps_per_env=[1, -1, 0, 0])
    gb.close()
