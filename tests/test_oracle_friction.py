"""Pins of the oracle's lagged friction term (App. A.3, D_k = mu lambda f0(|u|)).

f0 / f1 against their defining integral and cases, closest points against
dense sampling of the primitives, derivatives against central finite
differences, the tangent-frame Hessian's sign, and the physics: a cube
sliding on a stiff gel decelerates at mu g, keeps its speed without
friction, and stays put on a slope below the friction angle."""
import numpy as np
import pytest

import scenes
from oracle import OracleEnv
from oracle import distance as ods
from oracle import friction as fr

EH = 1e-6          # eps_v h of eps_v = 1e-3 m/s, h = 1e-3 s


def test_f0_is_the_integral_of_f1_and_f1_matches_its_cases():
    y = np.linspace(0.0, 3 * EH, 3001)
    # f0(y) = int_{eh}^{y} f1 + eh, by the trapezoid rule on a fine grid
    f1v = fr.f1(y, EH)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (f1v[1:] + f1v[:-1]) * np.diff(y))])
    i_eh = np.argmin(np.abs(y - EH))
    integral = cum - cum[i_eh] + EH
    assert np.allclose(fr.f0(y, EH), integral, atol=1e-6 * EH)
    assert fr.f0(0.0, EH) == pytest.approx(EH / 3.0)
    assert fr.f0(EH, EH) == pytest.approx(EH) and fr.f1(EH, EH) == pytest.approx(1.0)
    assert fr.f1(0.0, EH) == 0.0 and float(fr.f1(2 * EH, EH)) == 1.0
    # f1 / y and the derivative of g = f1 / y
    yy = np.array([0.1, 0.5, 0.9, 1.5, 4.0]) * EH
    assert np.allclose(fr.f1_over_y(yy, EH) * yy, fr.f1(yy, EH), rtol=1e-14)
    dy = 1e-6 * EH
    num = (fr.f1_over_y(yy + dy, EH) - fr.f1_over_y(yy - dy, EH)) / (2 * dy)
    assert np.allclose(fr.dg_over_y(yy, EH) * yy, num, rtol=1e-6)
    assert fr.f1_over_y(0.0, EH) == pytest.approx(2.0 / EH)


def _sample_dist(X, is_ee, n=200):
    if not is_ee:
        p, t0, t1, t2 = X
        u = np.linspace(0, 1, n)
        a, b = np.meshgrid(u, u)
        m = a + b <= 1.0
        pts = t0 + a[m][:, None] * (t1 - t0) + b[m][:, None] * (t2 - t0)
        return np.sqrt(((pts - p) ** 2).sum(1)).min()
    a0, a1, b0, b1 = X
    s = np.linspace(0, 1, n)
    pa = a0 + s[:, None] * (a1 - a0)
    pb = b0 + s[:, None] * (b1 - b0)
    return np.sqrt(((pa[:, None] - pb[None]) ** 2).sum(-1)).min()


@pytest.mark.parametrize("is_ee", [False, True])
def test_closest_weights_give_the_pair_distance(is_ee):
    rng = np.random.default_rng(21 + int(is_ee))
    for _ in range(60):
        X = rng.normal(size=(4, 3))
        if rng.random() < 0.3 and is_ee:                  # near-parallel edges
            X[3] = X[2] + (X[1] - X[0]) * rng.uniform(0.5, 2) + 1e-6 * rng.normal(size=3)
        w = fr.closest_weights(X, is_ee)
        d = np.linalg.norm(w @ X)
        assert abs(w.sum()) < 1e-12                        # a difference of two points
        assert d == pytest.approx(float(ods.pair_distance(X[None], np.array([is_ee]))[0]), rel=1e-9, abs=1e-12)
        assert d <= _sample_dist(X, is_ee) + 1e-12


def test_tangent_basis_is_orthonormal_and_normal_to_n():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        T = fr.tangent_basis(n)
        assert np.allclose(T.T @ T, np.eye(2), atol=1e-14)
        assert np.allclose(T.T @ n, 0.0, atol=1e-14)


@pytest.mark.parametrize("scale", [0.3, 3.0])           # |u| below / above eps_v h
def test_pair_friction_derivatives_match_finite_differences(scale):
    rng = np.random.default_rng(9)
    Xn = rng.normal(size=(3, 4, 3)) * 1e-3
    is_ee = np.array([False, True, False])
    dhat = 10.0                                           # every pair active
    W, T, lam, rn = fr.lagged(Xn, is_ee, np.full(3, 2.0), np.full(3, 1e-30), dhat)
    assert np.all(lam > 0)
    # displacements of the order of eps_v h (in the tangent plane or not)
    X = Xn + rng.normal(size=Xn.shape) * scale * EH
    mu = 0.4
    E, G, H = fr.pair_friction(X, W, T, lam, rn, mu, EH)
    step = 1e-4 * EH
    for k in range(3):
        Gn = np.zeros(12)
        Hn = np.zeros((12, 12))
        for j in range(12):
            dX = np.zeros(12)
            dX[j] = step
            Ep, Gp, _ = fr.pair_friction((X[k].ravel() + dX).reshape(1, 4, 3), W[k:k + 1], T[k:k + 1],
                                         lam[k:k + 1], rn[k:k + 1], mu, EH)
            Em, Gm, _ = fr.pair_friction((X[k].ravel() - dX).reshape(1, 4, 3), W[k:k + 1], T[k:k + 1],
                                         lam[k:k + 1], rn[k:k + 1], mu, EH)
            Gn[j] = (Ep[0] - Em[0]) / (2 * step)
            Hn[:, j] = (Gp[0] - Gm[0]) / (2 * step)
        assert np.allclose(G[k], Gn, rtol=1e-6, atol=1e-9 * np.abs(G[k]).max())
        assert np.allclose(H[k], Hn, rtol=1e-5, atol=1e-7 * np.abs(H[k]).max())
        assert np.linalg.eigvalsh(H[k]).min() >= -1e-9 * np.abs(H[k]).max()
        assert np.allclose(H[k], H[k].T)


def _cube_on_stiff_gel(mu, gravity=(0.0, 0.0, -9.81)):
    sc = scenes.small_contact_scene(body="cube", driven=False, gap=5e-5)
    sc.scene.E = 1e7                                      # a near-rigid floor
    prm = sc.params
    prm.friction_mu = mu
    prm.newton_tol = 1e-6
    prm.gravity = gravity
    env = OracleEnv(sc.scene, prm)
    x, v, y, yd = env.rest_state()
    return env, prm, x, v, y, yd


def _settle(env, x, v, y, yd, n):
    for _ in range(n):
        x, v, y, yd, st = env.step(x, v, y, yd)
        assert st.status == 0
    return x, v, y, yd


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_sliding_cube_decelerates_at_mu_g(mu):
    env, prm, x, v, y, yd = _cube_on_stiff_gel(mu)
    x, v, y, yd = _settle(env, x, v, y, yd, 15)
    yd = yd.copy()
    yd[0, 0] = 0.2                                        # 0.2 m/s along x, far above eps_v
    vs = [yd[0, 0]]
    for _ in range(8):
        x, v, y, yd, st = env.step(x, v, y, yd)
        assert st.status == 0
        vs.append(yd[0, 0])
    a = (vs[-1] - vs[0]) / (8 * prm.dt)
    # the lagged normal force tracks the weight up to the cube's small
    # vertical oscillation on the stiff floor
    assert a == pytest.approx(-mu * 9.81, abs=0.1 * 9.81 * max(mu, 0.05))


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_cube_on_a_slope_below_the_friction_angle_sticks(mu):
    # gravity tilted by atan(0.3): below the friction angle atan(0.5)
    th = np.arctan(0.3)
    g = 9.81 * np.array([np.sin(th), 0.0, -np.cos(th)])
    env, prm, x, v, y, yd = _cube_on_stiff_gel(mu, gravity=tuple(g))
    x, v, y, yd = _settle(env, x, v, y, yd, 15)
    if mu > 0.0:
        # static regime: creeps at most about eps_v
        assert abs(yd[0, 0]) < 2.0 * prm.friction_eps_v
    else:
        # frictionless: slides down the slope, v = n h g sin(theta) at most
        assert yd[0, 0] > 0.5 * 15 * prm.dt * g[0]
