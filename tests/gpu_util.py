"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""
import numpy as np

from oracle import OracleEnv
from oracle import energy as oen


def bbox_diag(env: OracleEnv, x, y) -> float:
    P = env.contact_positions(x, y)
    P = np.concatenate([x, P])
    return float(np.linalg.norm(P.max(0) - P.min(0)))


def all_points(env: OracleEnv, x, y):
    """Gel vertices and every body vertex phi(y) (the compared positions)."""
    parts = [x]
    for b, br in enumerate(env.bodies):
        parts.append(oen.body_points(y[b], br.xbar))
    return np.concatenate(parts)


def oracle_states(scenario, params, n_steps):
    """Oracle trajectory: list of (x, v, y, ydot, targets used for the next step)."""
    env = OracleEnv(scenario.scene, params)
    x, v, y, yd = env.rest_state()
    if scenario.v0 is not None:
        v = scenario.v0.copy()
    if scenario.ydot0 is not None:
        yd = scenario.ydot0.copy()
    out = []
    for s in range(n_steps):
        sy = env.targets_from_delta(scenario.delta(s))
        out.append((x, v, y, yd, sy))
        x, v, y, yd, st = env.step(x, v, y, yd, sy)
        assert st.status == 0, f"oracle did not converge at step {s}"
    out.append((x, v, y, yd, None))
    return env, out


def gpu_targets(genv, e, oracle_env: OracleEnv, sy):
    """Targets in the GPU's convention (p = its own com) for the same
    rest-placement translation the oracle used."""
    t = sy.copy()
    for b in range(oracle_env.nb):
        # translation the oracle applied to its own com
        t[b, :3] = genv.body_com(e, b) + (sy[b, :3] - oracle_env.bodies[b].com)
    return t


def to_gpu_y(genv, e, oracle_env: OracleEnv, y):
    """Same physical body placement in the GPU's frame (p offset by the
    difference between the two sides' computed centres of mass)."""
    yg = y.copy()
    for b in range(oracle_env.nb):
        A = np.stack([y[b, 3:6], y[b, 6:9], y[b, 9:12]], axis=1)
        yg[b, :3] = y[b, :3] + A @ (genv.body_com(e, b) - oracle_env.bodies[b].com)
    return yg


def from_gpu_y(genv, e, oracle_env: OracleEnv, yg):
    y = yg.copy()
    for b in range(oracle_env.nb):
        A = np.stack([yg[b, 3:6], yg[b, 6:9], yg[b, 9:12]], axis=1)
        y[b, :3] = yg[b, :3] - A @ (genv.body_com(e, b) - oracle_env.bodies[b].com)
    return y


def oracle_restart(env: OracleEnv, x_n, v_n, y_n, yd_n, s_y, x, y):
    """The oracle's step from (x_n, v_n, y_n, yd_n) with Newton (and its AL
    loop) started at a candidate end state (x, y) instead of at x_n.  A
    converged end state of the step is (close to) a fixed point of this."""
    xo, vo, yo, ydo, st = env.step(x_n, v_n, y_n, yd_n, s_y, x_start=x, y_start=y)
    return xo, yo, st


def other_minimiser(env: OracleEnv, x_n, v_n, y_n, yd_n, s_y, xg, yg, xo, yo, bar=1e-4):
    """Reading C-21: is the GPU's end state (xg, yg), farther than the bar
    from the oracle's (xo, yo), another converged point of the same step
    rather than a stall?  Three tests, all on the oracle:
    - the oracle's Newton + AL solve restarted at it, at the parity
      tolerance (1e-7 m/s: a stall on a flat direction keeps moving there),
      stays within the bar and converges;
    - it is free of contact and inversion;
    - its objective (the incremental potential with the step's targets, AL
      multipliers zero, each point's own contact pairs) is not above the
      oracle end point's by more than 1e-3 of the oracle step's decrease.
    Returns (accepted, details)."""
    prm = type(env.prm)(**env.prm.__dict__)
    prm.newton_tol = 1e-7
    tight = OracleEnv(env.scene, prm)
    xr, yr, st = oracle_restart(tight, x_n, v_n, y_n, yd_n, s_y, xg, yg)
    diag = bbox_diag(env, x_n, y_n)
    moved = float(np.abs(all_points(env, xr, yr) - all_points(env, xg, yg)).max() / diag)
    ctx = env.make_ctx(x_n, v_n, y_n, yd_n, s_y)

    def energy(x, y):
        return float(env.energy(x, y, ctx, env.pair_arrays(*env.static_pairs(x, y))))
    e_n, e_g, e_o = energy(x_n, y_n), energy(xg, yg), energy(xo, yo)
    de = (e_g - e_o) / max(e_n - e_o, 1e-300)
    ok = st.status == 0 and moved <= bar and valid_state(env, xg, yg) and de <= 1e-3
    return ok, {"moved": moved, "status": int(st.status), "dE_rel": de, "E_gpu": e_g, "E_oracle": e_o}


def valid_state(env: OracleEnv, x, y) -> bool:
    """No touching pair and no inverted tet."""
    from oracle import distance as ods
    pt, ee = env.static_pairs(x, y)
    pa = env.pair_arrays(pt, ee)
    if len(pa[0]) and ods.pair_distance(env.contact_positions(x, y)[pa[0]], pa[1]).min() <= 0.0:
        return False
    T = env.scene.gel_tets
    F = oen.deformation_gradient(x[T], env.gel.Dm_inv)
    return bool(np.linalg.det(F).min() > 0.0)


def oracle_press_step(args):
    """One oracle step of env e of the 256-env press batch from a given
    state (run in a child process by the full-size tests)."""
    import scenes
    e, k, state, prm = args
    scene, _, deltas = scenes.config1_batch(e + 1)
    oenv = OracleEnv(scene, prm)
    x, v, y, yd = state
    sy = oenv.targets_from_delta(deltas[e](k))
    xo, vo, yo, ydo, st = oenv.step(x, v, y, yd, sy)
    return {"x": xo, "y": yo, "status": st.status, "newton": st.newton_iters}
