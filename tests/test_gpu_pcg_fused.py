"""The fused PCG iteration kernel (ipc_params.pcg_fused = 1, the default, or 2):
contact terms, SELL mat-vec and update of every env in one persistent
launch, an env's update waiting for its own products.  It computes what the
three-kernel iteration (pcg_fused = 0) computes (Sec. 3.3's block-Jacobi
PCG, one iteration after another), so the tests hold the two to each other:
the same statuses, the same PCG work within a few iterations, and end
states within the multi-step bar of their precision (1e-6 of the bbox
diagonal per step in FP64 at the parity tolerances; the contact sums use
atomics, so the two orders differ in the last bits every iteration).  The
fused path against the oracle is covered by every other GPU test, which
runs the default."""
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
    # uneven envs pressing into contact within the K steps: several row
    # items and pair groups per env, envs leaving PCG at different iterations
    return [scenes.config2(e, n_steps=12) for e in (0, 1, 2, 5)]


def _table(g, scs, k0, n):
    mb = max(g.max_bodies, 1)
    t = np.zeros((n, len(scs), mb, 12))
    for k in range(n):
        for e, sc in enumerate(scs):
            y = g.rest_y(e)
            y[:, :3] += np.asarray(sc.delta(k0 + k)).reshape(-1, 3)[: y.shape[0]]
            t[k, e, : y.shape[0]] = y
    return t


def _run(prm, fused, rollout, stream=True, ipl=1):
    scs = _batch()
    p = type(prm)(**prm.__dict__)
    p.pcg_fused = fused
    p.pcg_iters_per_launch = ipl
    g = ipc.Envs([sc.scene for sc in scs], p, stream=torch.cuda.Stream() if stream else None)
    tab = _table(g, scs, 0, K)
    pcg = 0
    if rollout:
        st, steps, s = g.rollout(K, torch.as_tensor(tab, device="cuda"))
        assert np.all(steps == K)
        pcg = s["pcg_iters"]
    else:
        st = np.zeros(len(scs), np.int32)
        for k in range(K):
            g.set_targets_all(tab[k])
            s_k, s = g.step()
            st = np.where(st == 0, s_k, st)
            pcg += s["pcg_iters"]
    out = [g.get_state(e) for e in range(len(scs))]
    g.close()
    return np.asarray(st), out, pcg


def _close(sa, sb, bound):
    worst = 0.0
    for a, b in zip(sa, sb):
        diag = float(np.linalg.norm(a[0].max(0) - a[0].min(0)))
        worst = max(worst, np.abs(a[0] - b[0]).max() / diag, np.abs(a[2][:, :3] - b[2][:, :3]).max() / diag)
    assert worst <= bound * K, worst


@pytest.mark.parametrize("fused,rollout,stream,ipl", [(1, False, True, 1), (1, True, True, 1), (1, False, False, 1),
                                                      (2, False, True, 1), (2, True, True, 1),
                                                      (1, False, True, 4), (1, True, True, 4), (1, False, False, 3),
                                                      (1, True, True, 16)])
def test_fused_matches_three_kernels_fp64(fused, rollout, stream, ipl):
    """FP64 at the parity tolerances: lock-step graphs, the rollout graph,
    and host-driven steps (no stream: plain launches); update items in
    ready order (1) and in env order (2); ipl > 1: that many iterations
    per launch (k_pcg_multi, the per-env dataflow across iterations)."""
    prm = scenes.SolverParams().parity()
    st_a, xa, pa = _run(prm, fused, rollout, stream, ipl)
    st_b, xb, pb = _run(prm, 0, rollout, stream)
    assert np.all(st_a == 0) and np.all(st_b == 0)
    assert abs(pa - pb) <= 0.02 * pb, (pa, pb)
    _close(xa, xb, 1e-6)


def test_fused_matches_three_kernels_mixed():
    """Mixed precision (FP32 matrix and mat-vec) at the default tolerances,
    as a rollout.  Here two runs of the same path already differ: the
    contact sums' atomic order moves the FP32 products, the slowly
    converging envs of this batch stop at other points within the Newton
    tolerance (measured: the PCG totals of one step in repeated runs of
    either path spread by up to 40%, the gel's end points by up to 1e-5 m
    within the 4 steps).  So this holds the fused path to the other at that
    spread (statuses, PCG work within a factor 2, end points within 1e-3
    of the diagonal per step); the mixed parity tests against the oracle
    run the fused path by default."""
    prm = scenes.SolverParams()
    prm.precision = 1
    st_a, xa, pa = _run(prm, 1, True, ipl=4)
    st_b, xb, pb = _run(prm, 0, True)
    assert np.all(st_a == 0) and np.all(st_b == 0)
    assert 0.5 * pb <= pa <= 2.0 * pb, (pa, pb)
    _close(xa, xb, 1e-3)


def test_multi_iteration_rollout_window_runs_single_iterations():
    """Inside a rollout window (which counts single iterations) the fused
    kernel runs one iteration per launch whatever pcg_iters_per_launch
    says: the same end states as the three kernels with that window."""
    prm = scenes.SolverParams().parity()
    prm.rollout_pcg_window = 2
    st_a, xa, pa = _run(prm, 1, True, ipl=4)
    st_b, xb, pb = _run(prm, 0, True)
    assert np.all(st_a == 0) and np.all(st_b == 0)
    assert abs(pa - pb) <= 0.02 * pb, (pa, pb)
    _close(xa, xb, 1e-6)


def test_fused_with_friction_matches_three_kernels():
    """Lagged friction (App. A.3) on: the fused kernels take the friction
    record groups among an env's products (d_k of the record points formed
    on the fly, as the pair terms do) and hold to the three-kernel form,
    where the friction kernel reads d_k after the mat-vec; a driven cube
    pressed into the gel and dragged along it, FP64 parity tolerances, as
    lock-step graphs, as a rollout with 8 iterations per launch, and as a
    rollout with a PCG window of 2 (one iteration per launch)."""
    base = scenes.small_contact_scene(body="cube", gap=2e-5, depth=1e-4, n_steps=3)
    press = base.delta

    def delta(k):
        dl = press(k).copy()
        dl[0, 0] = 3e-5 * max(0, k - 2)
        return dl
    n = 6
    for rollout, window in ((False, 0), (True, 0), (True, 2)):
        out = []
        for fused in (1, 0):
            prm = base.params.parity()
            prm.friction_mu = 0.5
            prm.pcg_fused = fused
            prm.rollout_pcg_window = window
            g = ipc.Envs([base.scene], prm, stream=torch.cuda.Stream())
            mb = max(g.max_bodies, 1)
            tab = np.zeros((n, 1, mb, 12))
            for k in range(n):
                y = g.rest_y(0)
                y[:, :3] += np.asarray(delta(k)).reshape(-1, 3)[: y.shape[0]]
                tab[k, 0, : y.shape[0]] = y
            if rollout:
                st, steps, _ = g.rollout(n, torch.as_tensor(tab, device="cuda"))
                assert np.all(steps == n)
            else:
                st = np.zeros(1, np.int32)
                for k in range(n):
                    g.set_targets_all(tab[k])
                    s_k, _ = g.step()
                    st = np.where(st == 0, s_k, st)
            assert np.all(np.asarray(st) == 0)
            out.append(g.get_state(0))
            g.close()
        a, b = out
        diag = float(np.linalg.norm(a[0].max(0) - a[0].min(0)))
        assert np.abs(a[0] - b[0]).max() <= 1e-6 * n * diag
        assert np.abs(a[2][:, :3] - b[2][:, :3]).max() <= 1e-6 * n * diag


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a GPU fault: one env's products are made to
    wait for an update round that nothing completes (ipc_debug_pcg_wait_out).
    The waits give up after about a second, the kernel ends that env's step
    with IPC_ECUDA, and the context goes on: the same env steps normally
    from a set state afterwards, and its result equals a fresh context's."""
    scs = _batch()[:2]
    prm = scenes.SolverParams().parity()
    g = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    tab = _table(g, scs, 0, 2)
    g.set_targets_all(tab[0])
    st, _ = g.step()
    assert np.all(st == 0)
    state = [g.get_state(e) for e in range(2)]
    status, ms = g.debug_pcg_wait_out(0)
    assert status == ipc.IPC_ECUDA
    assert 200.0 < ms < 10000.0, ms                  # the ~1 s limit, not a hang
    # the context is usable: restore the state and take the next step
    for e in range(2):
        assert g.set_state(e, *state[e]) == ipc.IPC_OK
    g.set_targets_all(tab[1])
    st, _ = g.step()
    assert np.all(st == 0)
    after = [g.get_state(e) for e in range(2)]
    g.close()
    h = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    for e in range(2):
        assert h.set_state(e, *state[e]) == ipc.IPC_OK
    h.set_targets_all(tab[1])
    st, _ = h.step()
    assert np.all(st == 0)
    ref = [h.get_state(e) for e in range(2)]
    h.close()
    _close(after, ref, 1e-6 / K)


def test_fused_profile_class():
    """The profiled (host-driven) loop launches the fused kernel once per
    PCG iteration and none of the three separate ones."""
    scs = _batch()
    prm = scenes.SolverParams().parity()
    g = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    g.profile_enable(True)
    g.profile_reset()
    g.set_targets_all(_table(g, scs, 0, 1)[0])
    st, s = g.step()
    prof = g.profile()
    g.close()
    assert np.all(st == 0)
    assert prof["pcg_iter"][0] > 0
    assert prof["pcg_matvec"][0] == 0 and prof["pcg_update"][0] == 0 and prof["pair_matvec"][0] == 0
