"""Continuous batching on the GPU: requests loaded into the env slots of
resident per-class pools (a finished request's slot takes the next request
of its class; pools of different classes step on their own streams) give,
for every request, the same result as that request run alone in its own
context: whole multi-step requests at the FP64 parity tolerances
(1e-6 of the bounding-box diagonal), and single mixed-precision steps from
in-contact states at the mixed bar (1e-4), the per-step form in which the
tolerances are stated.  (At the mixed benchmark tolerances whole trajectories
of the same request can take different Newton paths through contact onset;
one 6-step config-2 request ended 5e-4 of the diagonal apart.)"""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402
from paper_2504_12908_b300.serving import GpuEngine, Request, Server, topology_key  # noqa: E402

build()


def _requests():
    # two classes with several requests each (slots get reused) and two
    # classes with one request; the config-2 pair shares a size class but
    # not material, sphere radius or script
    a, b = _same_class2()
    scs = [scenes.small_contact_scene(body="sphere", level=1, depth=2e-4, n_steps=5),
           scenes.config0(),
           scenes.small_contact_scene(body="sphere", level=1, depth=1e-4, n_steps=4),
           a,
           scenes.small_contact_scene(body="sphere", level=1, depth=3e-4, n_steps=6),
           b,
           scenes.small_contact_scene(body="cube", depth=1e-4, n_steps=4)]
    # (request 4's sixth step ends IPC_ENOTCONV at the parity tolerances in
    # the oracle too: its line search stalls at 57 Newton iterations)
    steps = [5, 6, 4, 5, 5, 4, 4]
    arrival = [0.0, 0.0, 0.02, 0.04, 0.06, 0.08, 0.08]
    reqs = [Request(rid=i, scene=sc.scene, delta=sc.delta, n_steps=steps[i], arrival=arrival[i])
            for i, sc in enumerate(scs)]
    return reqs


def _same_class2():
    a = scenes.config2(0)
    for e in range(1, 400):
        b = scenes.config2(e)
        if topology_key(b.scene) == topology_key(a.scene) and b.scene.E != a.scene.E:
            return a, b
    raise AssertionError("no env of the same class")


def _alone(req, prm):
    g = ipc.Envs([req.scene], prm)
    if req.state is not None:
        assert g.set_state(0, *req.state) == ipc.IPC_OK
    for k in range(req.n_steps):
        t = g.rest_y(0)
        t[:, :3] += np.asarray(req.delta(k)).reshape(-1, 3)[: t.shape[0]]
        g.set_targets(0, t)
        st, _ = g.step()
        assert st[0] == 0
    x, _, y, _ = g.get_state(0)
    g.close()
    return x, y


def _compare(rep, reqs, prm, bound):
    """bound: the per-step bar; a request of n steps may accumulate n of them
    (contact sums use atomics, so the two runs differ in the last bits every
    step)."""
    for r in reqs:
        res = rep.results[r.rid]
        assert res.status == 0 and res.steps == r.n_steps
        xa, ya = _alone(r, prm)
        diag = float(np.linalg.norm(xa.max(0) - xa.min(0)))
        tol = bound * r.n_steps * diag
        assert np.abs(res.final_x - xa).max() <= tol, r.rid
        assert np.abs(res.final_y[:, :3] - ya[:, :3]).max() <= tol, r.rid


@pytest.mark.parametrize("graphs", [True, False])
def test_each_request_is_the_same_alone_and_in_the_mix(graphs):
    """Multi-step requests at the FP64 parity tolerances (where one step's
    result is unique to ~1e-10 m): every request ends where it ends alone,
    within the FP64 bar of 1e-6 of the bbox diagonal per step."""
    prm = scenes.SolverParams().parity()
    reqs = _requests()
    # with graphs the pools advance up to 3 steps per call as rollouts
    srv = Server(GpuEngine(prm, graphs=graphs), slots_per_pool=2, mem_reserve=1 << 30, chunk=3 if graphs else 1)
    rep = srv.run(reqs)
    bad = {rid: (r.status, r.steps, reqs[rid].n_steps, r.slot) for rid, r in rep.results.items()
           if r.status != 0 or r.steps != reqs[rid].n_steps}
    assert rep.completed == len(reqs) and rep.backlog == 0, str(bad)
    assert rep.pools == 4 and rep.slot_reuses >= 1
    assert rep.env_steps == sum(r.n_steps for r in reqs)
    _compare(rep, reqs, prm, 1e-6)


def test_mixed_precision_steps_are_the_same_alone_and_in_the_mix():
    """Mixed precision at the benchmark tolerances, one step per request from
    an in-contact state (the per-step form of the mixed bar, 1e-4 of the
    bbox diagonal): each step in the mix matches the same step alone."""
    prm = scenes.SolverParams()
    prm.precision = 1
    reqs = _requests()
    # advance each scene alone to an in-contact state, then ask for one step
    one = []
    for r in reqs:
        g = ipc.Envs([r.scene], prm)
        for k in range(r.n_steps):
            t = g.rest_y(0)
            t[:, :3] += np.asarray(r.delta(k)).reshape(-1, 3)[: t.shape[0]]
            g.set_targets(0, t)
            assert g.step()[0][0] == 0
        state = g.get_state(0)
        g.close()
        k0 = r.n_steps

        def delta(k, d=r.delta, k0=k0):
            return d(k0 + k)
        one.append(Request(rid=r.rid, scene=r.scene, delta=delta, n_steps=1, arrival=r.arrival, state=state))
    srv = Server(GpuEngine(prm, graphs=True), slots_per_pool=2, mem_reserve=1 << 30)
    rep = srv.run(one)
    assert rep.completed == len(one) and rep.pools == 4
    _compare(rep, one, prm, 1e-4)
