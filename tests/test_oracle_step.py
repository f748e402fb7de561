"""Pins for the oracle's whole step (closed forms, invariants, brute force)."""
import itertools

import numpy as np
import pytest

import scenes
from oracle import OracleEnv
from oracle import distance as ds
from oracle.broadphase import candidates, canonical
from oracle.ccd import accd_batch, accd_toi, exact_toi


def _run(sc, params=None, steps=None):
    env = OracleEnv(sc.scene, params or sc.params)
    x, v, y, yd = env.rest_state()
    if sc.v0 is not None:
        v = sc.v0.copy()
    if sc.ydot0 is not None:
        yd = sc.ydot0.copy()
    out = [(x, v, y, yd, None)]
    for s in range(steps if steps is not None else sc.n_steps):
        sy = env.targets_from_delta(sc.delta(s))
        x, v, y, yd, st = env.step(x, v, y, yd, sy)
        out.append((x, v, y, yd, st))
    return env, out


def test_free_fall_closed_form():
    sc = scenes.free_fall_scene()
    prm = sc.params.parity()
    env, out = _run(sc, prm)
    x0, v0, y0, yd0, _ = out[0]
    h, g = prm.dt, np.asarray(prm.gravity)
    for n, (x, v, y, yd, st) in enumerate(out[1:], start=1):
        assert st.status == 0
        xe = x0 + n * h * v0 + 0.5 * n * (n + 1) * h * h * g
        assert np.abs(x - xe).max() < 1e-12
        pe = y0[0, :3] + n * h * yd0[0, :3] + 0.5 * n * (n + 1) * h * h * g
        assert np.abs(y[0, :3] - pe).max() < 1e-12
        assert np.abs(y[0, 3:] - y0[0, 3:]).max() < 1e-12
        assert st.newton_iters <= 2


def test_momentum_conserved_through_contact():
    sc = scenes.small_contact_scene(body="cube", driven=False)
    sc.scene.pinned[:] = False
    prm = sc.params.parity()
    prm.gravity = (0.0, 0.0, 0.0)
    env = OracleEnv(sc.scene, prm)
    x, v, y, yd = env.rest_state()
    yd[0, 2] = -0.08                       # cube moves down onto the gel
    m = env.gel.mass
    mb = env.bodies[0].mass
    P0 = (m[:, None] * v).sum(0) + mb * yd[0, :3]
    touched = False
    for s in range(8):
        x, v, y, yd, st = env.step(x, v, y, yd, y.copy())
        assert st.status == 0
        P = (m[:, None] * v).sum(0) + mb * yd[0, :3]
        assert np.abs(P - P0).max() < 1e-5 * np.abs(P0).max()
        touched |= st.min_dist < prm.dhat
    assert touched, "the cube never came within dhat of the gel"


def test_rigid_spin_stays_rotation():
    sc = scenes.spin_scene(omega=(0.0, 0.0, 20.0))
    prm = sc.params.parity()
    env, out = _run(sc, prm)
    h = prm.dt
    for n, (x, v, y, yd, st) in enumerate(out[1:], start=1):
        A = np.stack([y[0, 3:6], y[0, 6:9], y[0, 9:12]], axis=1)
        assert abs(np.linalg.det(A) - 1.0) < 1e-7
        assert np.abs(A.T @ A - np.eye(3)).max() < 1e-7
        ang = np.arctan2(A[1, 0], A[0, 0])
        assert 0.9 * n * 20.0 * h <= ang <= n * 20.0 * h * (1 + 1e-9)


def test_config0_invariants_and_monotone_energy():
    sc = scenes.config0()
    env, out = _run(sc)
    for x, v, y, yd, st in out[1:]:
        assert st.status == 0
        assert st.min_dist > 0.0
        assert st.min_J > 0.0
        for E0, E1 in st.energies:
            assert E1 <= E0
    # by the end the cube has pressed the gel: contact pairs within dhat exist
    assert out[-1][4].min_dist < sc.params.dhat


def test_step_is_translation_invariant():
    """Moving the whole scene (gel, body, and with them the pinned vertices
    and the driven body's targets) by a constant vector moves every step's
    result by that vector: no absolute position enters the step (a body
    mapped through x = A X instead of p + A (X - X_c), or a contact test on
    absolute coordinates, would fail).  Three contact steps of a driven
    sphere at the parity tolerances."""
    import copy
    sc = scenes.small_contact_scene(body="sphere", driven=True, depth=2e-4, n_steps=3)
    c = np.array([0.0125, -0.0375, 0.00625])           # exact in binary: no rounding of the shift
    moved = copy.deepcopy(sc.scene)
    moved.gel_x = moved.gel_x + c
    for b in moved.bodies:
        b.rest_x = b.rest_x + c
    prm = sc.params.parity()
    ea, eb = OracleEnv(sc.scene, prm), OracleEnv(moved, prm)
    sa, sb = ea.rest_state(), eb.rest_state()
    diag = float(np.linalg.norm(sc.scene.gel_x.max(0) - sc.scene.gel_x.min(0)))
    touched = False
    for s in range(3):
        sa = ea.step(*sa, ea.targets_from_delta(sc.delta(s)))
        sb = eb.step(*sb, eb.targets_from_delta(sc.delta(s)))
        assert sa[4].status == 0 and sb[4].status == 0
        assert np.abs((sb[0] - c) - sa[0]).max() <= 1e-9 * diag
        assert np.abs((sb[2][:, :3] - c) - sa[2][:, :3]).max() <= 1e-9 * diag
        assert np.abs(sb[2][:, 3:] - sa[2][:, 3:]).max() <= 1e-9
        assert np.abs(sb[1] - sa[1]).max() <= 1e-9 * diag / prm.dt
        touched |= sa[4].min_dist < prm.dhat
        sa, sb = sa[:4], sb[:4]
    assert touched


def test_converged_step_is_stationary():
    sc = scenes.small_contact_scene(body="sphere", driven=True, depth=2e-4, n_steps=3)
    prm = sc.params.parity()
    env = OracleEnv(sc.scene, prm)
    x, v, y, yd = env.rest_state()
    for s in range(3):
        x, v, y, yd, st = env.step(x, v, y, yd, env.targets_from_delta(sc.delta(s)))
        assert st.status == 0
    assert st.min_dist < prm.dhat
    pairs = env.pair_arrays(*env.static_pairs(x, y))
    g, _ = env.grad_hess(x, y, st.ctx, pairs)
    # compare with the gravity force scale of a gel vertex
    scale = prm.dt ** 2 * 9.81 * env.gel.mass.max()
    assert np.abs(g[env.free]).max() < 1e-3 * scale


def test_objective_gradient_matches_energy():
    sc = scenes.small_contact_scene(body="sphere", driven=True, depth=2e-4, n_steps=3)
    prm = sc.params.parity()
    env = OracleEnv(sc.scene, prm)
    x, v, y, yd = env.rest_state()
    x, v, y, yd, st = env.step(x, v, y, yd, env.targets_from_delta(sc.delta(0)))
    x, v, y, yd, st = env.step(x, v, y, yd, env.targets_from_delta(sc.delta(1)))
    ctx = env.make_ctx(x, v, y, yd, env.targets_from_delta(sc.delta(2)))
    rng = np.random.default_rng(3)
    ctx["lam_y"] = rng.normal(size=ctx["lam_y"].shape) * 1e-6
    pairs = env.pair_arrays(*env.static_pairs(x, y))
    assert len(pairs[0]) > 0
    g, H = env.grad_hess(x, y, ctx, pairs, project=False)
    q = env.join(x, y)
    for _ in range(4):
        u = rng.normal(size=q.shape) * env.free
        u *= 1e-9 / np.abs(u).max()
        f = lambda t: env.energy(*env.split(q + t * u), ctx, pairs)
        fd = (f(1.0) - f(-1.0)) / 2.0
        assert fd == pytest.approx(g @ u, rel=1e-5, abs=1e-9 * np.abs(g).max() * 1e-9)
        # Hessian by FD of the gradient along a shorter u (the barrier is
        # strongly nonlinear at micrometre gaps)
        w = u * 1e-2
        gp, _ = env.grad_hess(*env.split(q + w), ctx, pairs, project=False)
        gm, _ = env.grad_hess(*env.split(q - w), ctx, pairs, project=False)
        Hw = H @ w
        assert np.abs((gp - gm) / 2.0 - Hw).max() < 1e-6 * np.abs(Hw).max()


# ---------------------------------------------------------------- broad phase
def test_candidates_match_naive_loops_and_cover_dhat():
    sc = scenes.small_contact_scene(body="sphere", level=1, gap=3e-5, n_steps=2)
    env = OracleEnv(sc.scene, sc.params)
    x, v, y, yd = env.rest_state()
    rng = np.random.default_rng(5)
    y = y.copy()
    y[0, :3] += rng.normal(scale=2e-5, size=3) + np.array([0, 0, -1e-5])
    Xc = env.contact_positions(x, y)
    sd, dhat = env.sd, sc.params.dhat
    pt, ee = candidates(sd, Xc, dhat, env.excluded)

    def box(ids):
        P = Xc[list(ids)]
        return P.min(0), P.max(0)

    def ov(a, b):
        return all(a[0][k] <= b[1][k] + dhat and b[0][k] <= a[1][k] + dhat for k in range(3))
    npt = set()
    for pi, p in enumerate(sd.points):
        for ti, t in enumerate(sd.tris):
            if sd.point_obj[pi] != sd.tri_obj[ti] and ov(box([p]), box(t)):
                npt.add((int(p), ti))
    nee = set()
    for i, j in itertools.combinations(range(len(sd.edges)), 2):
        oi, oj = sd.edge_obj[i], sd.edge_obj[j]
        if oi == oj:
            continue
        a, b = (i, j) if oi < oj else (j, i)
        if ov(box(sd.edges[a]), box(sd.edges[b])):
            nee.add((a, b))
    npt = {pr for pr in npt if not (sd.fixed[pr[0]] and all(sd.fixed[sd.tris[pr[1]]]))}
    assert set(map(tuple, pt.tolist())) == npt
    assert set(map(tuple, ee.tolist())) == nee
    # every pair of different objects closer than dhat is a candidate
    allpt = np.array([(p, t) for (p, t) in itertools.product(range(len(sd.points)), range(len(sd.tris)))
                      if sd.point_obj[p] != sd.tri_obj[t]])
    X12 = np.concatenate([Xc[sd.points[allpt[:, 0]]][:, None], Xc[sd.tris[allpt[:, 1]]]], axis=1)
    d = ds.pair_distance(X12, np.zeros(len(allpt), bool))
    close = {(int(sd.points[p]), int(t)) for (p, t), dd in zip(allpt, d) if dd < dhat}
    assert close and close <= npt
    a, b = canonical(sd, pt, ee)
    assert a.shape == (len(pt), 4) and b.shape == (len(ee), 4)


def test_self_contact_candidates_match_naive_loops_and_cover_dhat():
    """Gel self-contact: within a flagged pad a point pairs with every
    triangle not incident to it and an edge with every edge it shares no
    vertex with (each unordered pair once); across objects as before."""
    sc = scenes.self_contact_scene()
    env = OracleEnv(sc.scene, sc.params)
    x, v, y, yd = env.rest_state()
    rng = np.random.default_rng(6)
    x = x + rng.normal(scale=1e-5, size=x.shape)
    Xc = env.contact_positions(x, y)
    sd, dhat = env.sd, sc.params.dhat
    pt, ee = candidates(sd, Xc, dhat, env.excluded)

    def box(ids):
        P = Xc[list(ids)]
        return P.min(0), P.max(0)

    def ov(a, b):
        return all(a[0][k] <= b[1][k] + dhat and b[0][k] <= a[1][k] + dhat for k in range(3))

    def may_pair(oa, ob):
        return oa != ob or oa == 0          # object 0 is the pad (self-contact on); bodies never self-pair
    npt = set()
    for pi, p in enumerate(sd.points):
        for ti, t in enumerate(sd.tris):
            if may_pair(sd.point_obj[pi], sd.tri_obj[ti]) and p not in t and ov(box([p]), box(t)):
                npt.add((int(p), ti))
    nee = set()
    for i, j in itertools.combinations(range(len(sd.edges)), 2):
        oi, oj = sd.edge_obj[i], sd.edge_obj[j]
        if not may_pair(oi, oj) or set(sd.edges[i]) & set(sd.edges[j]):
            continue
        a, b = (i, j) if oi <= oj else (j, i)
        if ov(box(sd.edges[a]), box(sd.edges[b])):
            nee.add((a, b))
    npt = {pr for pr in npt if not (sd.fixed[pr[0]] and all(sd.fixed[sd.tris[pr[1]]]))}
    nee = {pr for pr in nee if not (all(sd.fixed[sd.edges[pr[0]]]) and all(sd.fixed[sd.edges[pr[1]]]))}
    assert set(map(tuple, pt.tolist())) == npt
    assert set(map(tuple, ee.tolist())) == nee
    own_pt = [(p, t) for (p, t) in npt if sd.point_obj[p] == 0 and sd.tri_obj[t] == 0]
    assert own_pt                                     # the blocks start 50 um apart: pairs within the pad
    # every non-incident point-triangle pair of the pad closer than dhat is a candidate
    allpt = np.array([(p, t) for (p, t) in itertools.product(range(len(sd.points)), range(len(sd.tris)))
                      if sd.point_obj[p] == 0 and sd.tri_obj[t] == 0 and sd.points[p] not in sd.tris[t]])
    X12 = np.concatenate([Xc[sd.points[allpt[:, 0]]][:, None], Xc[sd.tris[allpt[:, 1]]]], axis=1)
    d = ds.pair_distance(X12, np.zeros(len(allpt), bool))
    close = {(int(sd.points[p]), int(t)) for (p, t), dd in zip(allpt, d) if dd < dhat}
    assert close and close <= npt


def _heights_above_base(sc, x):
    """Height of every bottom vertex of the upper block above the deformed
    top face of the base, at the same (x, y) (barycentric on the base's
    top-face triangles)."""
    g = sc.scene.gel_x
    n_low = int(np.sum(g[:, 2] <= 0.0))
    top = np.nonzero(np.isclose(g[:n_low, 2], 0.0))[0]
    bottom_up = n_low + np.nonzero(np.isclose(g[n_low:, 2], g[n_low:, 2].min()))[0]
    from scipy.spatial import Delaunay
    tri = Delaunay(g[top, :2])                          # the rest top face, as triangles in (x, y)
    out = []
    for u in bottom_up:
        s = int(tri.find_simplex(x[u, :2]))
        assert s >= 0
        T = top[tri.simplices[s]]
        A = np.c_[x[T, :2], np.ones(3)].T
        lam = np.linalg.solve(A, np.r_[x[u, :2], 1.0])
        out.append(x[u, 2] - lam @ x[T, 2])
    return np.array(out)


def test_self_contact_holds_the_blocks_of_one_pad_apart():
    """The same scene with and without the pad's self-contact flag: with it
    the pressed upper block rests on the base (positive heights, active
    pairs within the pad), without it the block sinks into the base."""
    heights = {}
    for flag in (True, False):
        sc = scenes.self_contact_scene(self_contact=flag)
        env, out = _run(sc)
        assert all(st.status == 0 for *_, st in out[1:])
        x, _, y, _, _ = out[-1]
        heights[flag] = _heights_above_base(sc, x)
    assert heights[True].min() > 0.0
    assert heights[True].max() < 1e-4                  # pressed down onto the base
    assert heights[False].min() < -1e-4                # no self-contact: interpenetration


# ---------------------------------------------------------------- CCD
@pytest.mark.parametrize("seed", range(20))
def test_accd_conservative_vs_exact_roots(seed):
    rng = np.random.default_rng(900 + seed)
    is_ee = bool(seed % 2)
    x0 = rng.normal(size=(4, 3))
    p = rng.normal(size=(4, 3)) * 2.0
    d0 = ds.pair_distance(x0[None], np.array([is_ee]))[0]
    t = accd_toi(x0, p, is_ee)
    tb = accd_batch(x0[None], p[None], np.array([is_ee]))[0]
    assert t == tb
    te = exact_toi(x0, p, is_ee)
    assert 0.0 < t <= 1.0
    assert t <= te + 1e-12
    # the pair stays apart on [0, t]
    for s in np.linspace(0.0, t, 50):
        assert ds.pair_distance((x0 + s * p)[None], np.array([is_ee]))[0] > 0.0
    if te < 1.0:
        # ACCD stops short of contact but keeps a fraction of the gap
        dt = ds.pair_distance((x0 + t * p)[None], np.array([is_ee]))[0]
        assert dt >= 0.1 * d0 * (1 - 1e-9) or t == 1.0


def test_accd_head_on_point_triangle():
    # point falling straight onto a triangle interior from height 1 by 2:
    # exact contact at t = 0.5, ACCD returns t < 0.5 with gap >= 0.1
    x0 = np.array([[0.2, 0.2, 1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    p = np.zeros((4, 3))
    p[0, 2] = -2.0
    assert exact_toi(x0, p, False) == pytest.approx(0.5, abs=1e-9)
    t = accd_toi(x0, p, False)
    assert t < 0.5
    assert 1.0 - 2.0 * t >= 0.1 - 1e-12
    # no approach: full step
    assert accd_toi(x0, np.ones((4, 3)), False) == 1.0


def test_restart_helper_keeps_converged_states_and_moves_others():
    """The helper the mixed-precision GPU test uses to accept a different
    minimiser: restarted at the oracle's own end state, Newton stays there;
    restarted at a perturbed state, it moves back; the validity check
    rejects an inverted tet."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from gpu_util import all_points, bbox_diag, oracle_restart, valid_state
    sc = scenes.config0()
    prm = sc.params.parity()
    env = OracleEnv(sc.scene, prm)
    x, v, y, yd = env.rest_state()
    sy = env.targets_from_delta(sc.delta(0))
    x1, v1, y1, yd1, st = env.step(x, v, y, yd, sy)
    assert st.status == 0
    diag = bbox_diag(env, x, y)
    xr, yr, st2 = oracle_restart(env, x, v, y, yd, sy, x1, y1)
    assert st2.status == 0
    assert np.abs(all_points(env, xr, yr) - all_points(env, x1, y1)).max() <= 1e-6 * diag
    free = ~sc.scene.pinned
    xp = x1.copy()
    xp[free] += 2e-6 * np.random.default_rng(1).standard_normal((int(free.sum()), 3))
    xr2, yr2, st3 = oracle_restart(env, x, v, y, yd, sy, xp, y1)
    assert st3.status == 0
    assert np.abs(all_points(env, xr2, yr2) - all_points(env, x1, y1)).max() <= 1e-6 * diag
    assert np.abs(xp - x1).max() > 1e-6
    assert valid_state(env, x1, y1)
    xb = x1.copy()
    t = sc.scene.gel_tets[0]
    xb[t[0]] = xb[t[1]] + (xb[t[1]] - xb[t[0]])            # fold one tet over
    assert not valid_state(env, xb, y1)


def test_newton_filter_switches_after_the_set_iterations():
    sc = scenes.config0()
    prm = scenes.SolverParams(**sc.params.__dict__)
    prm.newton_abs_after = 10
    env = OracleEnv(sc.scene, prm)
    assert [env.newton_filter(i) for i in (0, 9, 10, 15)] == ["clamp", "clamp", "abs", "abs"]
    # the default clamps throughout
    assert OracleEnv(sc.scene, sc.params).newton_filter(500) == "clamp"


def test_converged_state_does_not_depend_on_the_filter():
    # the filter only changes the path of projected Newton: at the parity
    # tolerances a step filtered with |lambda| from its first iteration ends
    # where the clamped step ends (same minimiser from the same start)
    sc = scenes.small_contact_scene(body="sphere", driven=True, depth=2e-4, n_steps=3)
    prm_c = sc.params.parity()
    prm_a = scenes.SolverParams(**prm_c.__dict__)
    prm_a.newton_abs_after = 0
    ec, out_c = _run(sc, prm_c, 3)
    ea, out_a = _run(sc, prm_a, 3)
    assert ea.newton_filter(0) == "abs"
    diag = np.linalg.norm(out_c[0][0].max(0) - out_c[0][0].min(0))
    for (xc, _, yc, _, stc), (xa, _, ya, _, sta) in zip(out_c[1:], out_a[1:]):
        assert stc.status == 0 and sta.status == 0
        assert np.abs(xc - xa).max() <= 1e-6 * diag
        assert np.abs(yc - ya).max() <= 1e-6 * diag
