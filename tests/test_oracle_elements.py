"""Pins for the oracle's per-element terms (closed forms, FD, invariants)."""
import numpy as np
import pytest

import scenes
from oracle import energy as en
from oracle import distance as ds
from oracle.rest import body_rest, gel_rest, lame, surface_data

RNG = np.random.default_rng(7)


def _rand_rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ---------------------------------------------------------------- rest data
def test_cube_mass_matrix_closed_form():
    # cube of side s, density rho: m = rho s^3, int x_i^2 dm = rho s^5 / 12
    s, rho = 8e-3, 1200.0
    x, t = scenes.box_surface((0.1, -0.2, 0.3), (0.1 + s, -0.2 + s, 0.3 + s))
    br = body_rest(scenes.Body(rest_x=x, tris=t, rho=rho, kappa_s=1e8, driven=False))
    assert br.mass == pytest.approx(6.144e-4, rel=1e-12)
    assert np.allclose(br.S, np.eye(3) * 3.2768e-9, rtol=1e-10, atol=1e-22)
    assert np.allclose(br.com, [0.1 + s / 2, -0.2 + s / 2, 0.3 + s / 2], atol=1e-15)
    # M^y = J^T M J assembled from the 8 corner-mass lumping is NOT exact;
    # the exact solid integral gives block-diagonal [m I, S_kl I]
    assert np.allclose(br.My[:3, :3], br.mass * np.eye(3))
    assert np.allclose(br.My[:3, 3:], 0.0, atol=1e-20)


def test_icosphere_volume_and_inertia_converge_to_sphere():
    r, rho = 1e-2, 800.0
    for level, tol in ((3, 2e-2), (4, 5e-3)):
        x, t = scenes.icosphere(level, r, center=(0.3, 0.1, -0.2))
        br = body_rest(scenes.Body(rest_x=x, tris=t, rho=rho, kappa_s=1e8, driven=False))
        # inscribed polyhedron: volume below the sphere's, approaching it
        assert br.vol < 4.0 / 3.0 * np.pi * r ** 3
        assert br.vol == pytest.approx(4.0 / 3.0 * np.pi * r ** 3, rel=tol)
        # solid sphere: int x_i^2 dm = m r^2 / 5
        assert np.allclose(np.diag(br.S), br.mass * r * r / 5.0, rtol=2 * tol)
        assert np.allclose(br.com, [0.3, 0.1, -0.2], atol=1e-12)


def test_gel_rest_volume_mass_and_lame():
    x, tets, _, _ = scenes.gel_grid(5, 4, 3, size=(0.01, 0.008, 0.003))
    sc = scenes.Scene(gel_x=x, gel_tets=tets, gel_obj=np.zeros(len(x), np.int32),
                      pinned=np.zeros(len(x), bool), attach=-np.ones(len(x), np.int32),
                      E=3e5, nu=0.45, rho=1000.0)
    gr = gel_rest(sc)
    assert gr.vol.sum() == pytest.approx(0.01 * 0.008 * 0.003, rel=1e-12)
    assert gr.mass.sum() == pytest.approx(1000.0 * 0.01 * 0.008 * 0.003, rel=1e-12)
    # linear-elastic small strain: uniaxial stress with free lateral faces
    # recovers E and nu from the neo-Hookean stress (pins lame() and piola())
    mu, lam = lame(3e5, 0.45)
    eps = 1e-7
    # lateral strain that zeroes the lateral stress, by bisection on P_yy
    lo, hi = -1e-6, 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        F = np.diag([1 + eps, 1 + mid, 1 + mid])[None]
        if en.piola(F, mu, lam)[0, 1, 1] > 0:
            hi = mid
        else:
            lo = mid
    F = np.diag([1 + eps, 1 + mid, 1 + mid])[None]
    P = en.piola(F, mu, lam)[0]
    assert -mid / eps == pytest.approx(0.45, rel=1e-5)
    assert P[0, 0] / eps == pytest.approx(3e5, rel=1e-5)


def test_surface_counts_config0():
    sc = scenes.config0().scene
    sd = surface_data(sc, [body_rest(b) for b in sc.bodies])
    gel_pts = (sd.points < sc.n_verts).sum()
    assert gel_pts == 194
    assert (sd.tri_obj == 0).sum() == 384
    assert (sd.edge_obj == 0).sum() == 576
    assert (sd.tri_obj == 1).sum() == 12 and (sd.edge_obj == 1).sum() == 18
    # vertex areas partition the total surface area
    tot = 2 * (0.02 * 0.02) + 4 * (0.02 * 0.004)
    assert sd.point_area[sd.point_obj == 0].sum() == pytest.approx(tot, rel=1e-12)
    assert sd.edge_area[sd.edge_obj == 0].sum() == pytest.approx(tot, rel=1e-12)


# ---------------------------------------------------------------- elastic
def _tet(rng, scale=1e-3):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * scale
    X = X + rng.normal(scale=0.1 * scale, size=X.shape)
    Dm = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    return X, np.linalg.inv(Dm)[None], np.array([np.linalg.det(Dm) / 6.0])


def test_elastic_zero_at_rest_and_rigid_motion():
    mu, lam = lame(3e5, 0.45)
    X, Dmi, V = _tet(RNG)
    R = _rand_rot(RNG)
    for x in (X, X @ R.T + np.array([0.3, -0.1, 2.0])):
        assert abs(en.tet_energy(x[None], Dmi, V, mu, lam)[0]) < 1e-18
        assert np.abs(en.tet_grad(x[None], Dmi, V, mu, lam)).max() < 1e-12 * mu * 1e-6


def test_elastic_frame_indifferent_at_deformed_states():
    """A rotation R and a translation of a deformed tet leave the energy
    unchanged and rotate its gradient (g_i -> R g_i) and its projected
    Hessian (H -> Q H Q^T, Q = diag(R, R, R, R)): the energy depends on F
    only through F^T F, as a neo-Hookean energy must (a term in F itself,
    or a transposed F, fails this away from the rest state)."""
    mu, lam = lame(3e5, 0.45)
    for _ in range(5):
        X, Dmi, V = _tet(RNG)
        x = X + RNG.normal(scale=1.5e-4, size=X.shape)   # ~15% strains, det F > 0
        R = _rand_rot(RNG)
        xr = x @ R.T + RNG.normal(size=3)
        E0 = en.tet_energy(x[None], Dmi, V, mu, lam)[0]
        E1 = en.tet_energy(xr[None], Dmi, V, mu, lam)[0]
        assert E0 > 0 and E1 == pytest.approx(E0, rel=1e-9)
        g0 = en.tet_grad(x[None], Dmi, V, mu, lam)[0].reshape(4, 3)
        g1 = en.tet_grad(xr[None], Dmi, V, mu, lam)[0].reshape(4, 3)
        assert np.allclose(g1, g0 @ R.T, rtol=1e-8, atol=1e-10 * np.abs(g0).max())
        Q = np.kron(np.eye(4), R)
        for project in (False, True):
            H0 = en.tet_hess(x[None], Dmi, V, mu, lam, project=project)[0]
            H1 = en.tet_hess(xr[None], Dmi, V, mu, lam, project=project)[0]
            assert np.allclose(H1, Q @ H0 @ Q.T, rtol=1e-7, atol=1e-9 * np.abs(H0).max())


def test_orthogonality_invariant_under_rotations_of_either_side():
    """|A A^T - I|_F^2 is unchanged by A -> R A and by A -> A R for
    rotations R (the columns of A, the body's affine axes, rotate
    together), at non-orthogonal A."""
    for _ in range(5):
        A = _rand_rot(RNG) + RNG.normal(scale=0.1, size=(3, 3))
        R = _rand_rot(RNG)
        e0 = en.orth_energy(A.T.ravel())
        assert e0 > 0
        assert en.orth_energy((R @ A).T.ravel()) == pytest.approx(e0, rel=1e-10)
        assert en.orth_energy((A @ R).T.ravel()) == pytest.approx(e0, rel=1e-10)


def test_elastic_gradient_and_hessian_fd():
    mu, lam = lame(3e5, 0.45)
    X, Dmi, V = _tet(RNG)
    x = X + RNG.normal(scale=1e-4, size=X.shape)
    q = x.ravel()
    f = lambda q: en.tet_energy(q.reshape(1, 4, 3), Dmi, V, mu, lam)[0]
    g = en.tet_grad(x[None], Dmi, V, mu, lam)[0]
    h = 1e-9
    gfd = np.array([(f(q + h * e) - f(q - h * e)) / (2 * h) for e in np.eye(12)])
    assert np.allclose(g, gfd, rtol=1e-6, atol=1e-8 * np.abs(g).max())
    H = en.tet_hess(x[None], Dmi, V, mu, lam, project=False)[0]
    gf = lambda q: en.tet_grad(q.reshape(1, 4, 3), Dmi, V, mu, lam)[0]
    Hfd = np.stack([(gf(q + h * e) - gf(q - h * e)) / (2 * h) for e in np.eye(12)], axis=1)
    assert np.allclose(H, Hfd, rtol=1e-5, atol=1e-6 * np.abs(H).max())


def test_elastic_projection_properties():
    mu, lam = lame(3e5, 0.45)
    X, Dmi, V = _tet(RNG)
    # compressed state: raw Hessian indefinite, projection PSD and idempotent
    x = X.copy()
    x[3] = x[0] + 0.45 * (X[3] - X[0])
    Hr = en.tet_hess(x[None], Dmi, V, mu, lam, project=False)[0]
    Hp = en.tet_hess(x[None], Dmi, V, mu, lam, project=True)[0]
    assert np.linalg.eigvalsh(Hr).min() < -1e-6 * np.abs(Hr).max()
    assert np.linalg.eigvalsh(Hp).min() > -1e-9 * np.abs(Hp).max()
    A = en.dPdF(en.deformation_gradient(x[None], Dmi), mu, lam)
    Ap = en.psd_clamp(A)
    assert np.allclose(en.psd_clamp(Ap), Ap, atol=1e-9 * np.abs(Ap).max())
    # stretched state where dP/dF is already PD: projection is the identity
    x2 = X * 1.05
    A2 = en.dPdF(en.deformation_gradient(x2[None], Dmi), mu, lam)
    assert np.linalg.eigvalsh(A2[0]).min() > 0
    assert np.allclose(en.psd_clamp(A2), A2, rtol=1e-12, atol=1e-12 * np.abs(A2).max())


def test_elastic_inverted_is_infinite():
    mu, lam = lame(3e5, 0.45)
    X, Dmi, V = _tet(RNG)
    x = X.copy()
    x[3] = x[0] - (X[3] - X[0])
    assert np.isinf(en.tet_energy(x[None], Dmi, V, mu, lam)[0])


# ---------------------------------------------------------------- affine body
def test_orthogonality_zero_on_rotations_and_fd():
    R = _rand_rot(RNG)
    yA = R.T.ravel()   # columns of R
    assert np.allclose(np.stack([yA[0:3], yA[3:6], yA[6:9]], axis=1), R)
    assert abs(en.orth_energy(yA)) < 1e-28
    assert np.abs(en.orth_grad(yA)).max() < 1e-14
    A = R + RNG.normal(scale=0.05, size=(3, 3))
    yA = A.T.ravel()
    # direct definition
    assert en.orth_energy(yA) == pytest.approx(np.sum((A.T @ A - np.eye(3)) ** 2), rel=1e-12)
    h = 1e-7
    gfd = np.array([(en.orth_energy(yA + h * e) - en.orth_energy(yA - h * e)) / (2 * h) for e in np.eye(9)])
    assert np.allclose(en.orth_grad(yA), gfd, rtol=1e-6, atol=1e-9)
    Hfd = np.stack([(en.orth_grad(yA + h * e) - en.orth_grad(yA - h * e)) / (2 * h) for e in np.eye(9)], axis=1)
    assert np.allclose(en.orth_hess(yA), Hfd, rtol=1e-6, atol=1e-8)


# ---------------------------------------------------------------- distances
def _sample_tri(t0, t1, t2, n=120):
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    m = u + v <= 1
    u, v = u[m], v[m]
    return t0 + u[:, None] * (t1 - t0) + v[:, None] * (t2 - t0)


def _sample_seg(a, b, n=2000):
    s = np.linspace(0, 1, n)
    return a + s[:, None] * (b - a)


@pytest.mark.parametrize("seed", range(12))
def test_pt_distance_vs_dense_sampling(seed):
    rng = np.random.default_rng(100 + seed)
    X = rng.normal(size=(1, 4, 3))
    X[0, 0] *= 1.5
    d = ds.pair_distance(X, np.array([False]))[0]
    S = _sample_tri(X[0, 1], X[0, 2], X[0, 3])
    dmin = np.linalg.norm(S - X[0, 0], axis=1).min()
    assert d <= dmin + 1e-12
    assert d == pytest.approx(dmin, abs=3e-2 * np.abs(X).max() / 100 + 1e-3)


@pytest.mark.parametrize("seed", range(12))
def test_ee_distance_vs_dense_sampling(seed):
    rng = np.random.default_rng(200 + seed)
    X = rng.normal(size=(1, 4, 3))
    d = ds.pair_distance(X, np.array([True]))[0]
    A = _sample_seg(X[0, 0], X[0, 1], 1500)
    B = _sample_seg(X[0, 2], X[0, 3], 1500)
    dd = np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)).min()
    assert d <= dd + 1e-12
    assert d == pytest.approx(dd, abs=5e-3)


def test_parallel_edges_distance():
    # two parallel segments offset by (0, h, 0), overlapping in x: distance h
    X = np.array([[[0, 0, 0], [1, 0, 0], [0.3, 0.25, 0], [1.7, 0.25, 0]]], float)
    assert ds.pair_distance(X, np.array([True]))[0] == pytest.approx(0.25, rel=1e-14)


def test_barrier_scalar_properties():
    dhat = 1e-4
    d = np.linspace(1e-7, 1.2e-4, 50)
    b = ds.barrier(d, dhat)
    assert np.all(b[d >= dhat] == 0.0)
    assert np.all(b[d < dhat] > 0.0)
    assert np.all(np.diff(b[d < dhat]) < 0.0)          # decreasing
    h = 1e-10
    m = (d > 2e-7) & (d < dhat - 2e-7)
    fd1 = (ds.barrier(d + h, dhat) - ds.barrier(d - h, dhat)) / (2 * h)
    fd2 = (ds.barrier_d1(d + h, dhat) - ds.barrier_d1(d - h, dhat)) / (2 * h)
    assert np.allclose(ds.barrier_d1(d, dhat)[m], fd1[m], rtol=1e-5)
    assert np.allclose(ds.barrier_d2(d, dhat)[m], fd2[m], rtol=1e-5)
    # C^2 at dhat: value and first derivative vanish there
    assert abs(ds.barrier_d1(dhat * (1 - 1e-9), dhat)) < 1e-12


def test_point_above_triangle_barrier_is_weighted_b():
    dhat, w = 1e-4, 3.7
    for d in (1e-6, 2e-5, 9e-5):
        X = np.array([[[0.2e-3, 0.3e-3, d], [0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0]]])
        E, G, _ = ds.pair_barrier(X, np.array([False]), np.array([w]), np.zeros(1), dhat, order=1)
        assert E[0] == pytest.approx(w * float(ds.barrier(d, dhat)), rel=1e-12)
        # force on the point is along +z only (normal to the triangle)
        assert abs(G[0, 0]) < 1e-12 * abs(G[0, 2]) and abs(G[0, 1]) < 1e-12 * abs(G[0, 2])
        # and the total force on the pair vanishes (translation invariance)
        assert np.allclose(G[0].reshape(4, 3).sum(0), 0.0, atol=1e-12 * np.abs(G).max())


def _fd_pair(X, is_ee, eps, dhat, w=1.0):
    q = X.ravel()
    f = lambda q: ds.pair_barrier(q.reshape(1, 4, 3), np.array([is_ee]), np.array([w]), np.array([eps]),
                                  dhat, order=0)[0][0]
    gf = lambda q: ds.pair_barrier(q.reshape(1, 4, 3), np.array([is_ee]), np.array([w]), np.array([eps]),
                                   dhat, order=1)[1][0]
    _, G, H = ds.pair_barrier(X[None], np.array([is_ee]), np.array([w]), np.array([eps]), dhat,
                              order=2, project=False)
    h = 1e-11
    gfd = np.array([(f(q + h * e) - f(q - h * e)) / (2 * h) for e in np.eye(12)])
    Hfd = np.stack([(gf(q + h * e) - gf(q - h * e)) / (2 * h) for e in np.eye(12)], axis=1)
    return G[0], gfd, H[0], Hfd


@pytest.mark.parametrize("case", ["pt_interior", "pt_edge", "pt_vertex", "ee_interior", "ee_endpoint",
                                  "ee_mollified"])
def test_pair_barrier_fd(case):
    dhat = 1e-4
    rng = np.random.default_rng(hash(case) % 1000)
    s = 1e-3
    if case == "pt_interior":
        X = np.array([[0.2, 0.3, 0.04], [0, 0, 0], [1, 0, 0], [0, 1, 0]]) * s
        is_ee, eps = False, 0.0
    elif case == "pt_edge":
        X = np.array([[0.5, -0.03, 0.02], [0, 0, 0], [1, 0, 0], [0, 1, 0]]) * s
        is_ee, eps = False, 0.0
    elif case == "pt_vertex":
        X = np.array([[-0.03, -0.02, 0.03], [0, 0, 0], [1, 0, 0], [0, 1, 0]]) * s
        is_ee, eps = False, 0.0
    elif case == "ee_interior":
        X = np.array([[0, 0, 0], [1, 0.1, 0], [0.5, -0.5, 0.05], [0.4, 0.5, 0.06]]) * s
        is_ee, eps = True, 1e-3 * s ** 4 * 0.01
    elif case == "ee_endpoint":
        X = np.array([[0, 0, 0], [1, 0.1, 0], [0.5, 0.07, 0.03], [0.6, 1.0, 0.5]]) * s
        is_ee, eps = True, 1e-3 * s ** 4 * 0.01
    else:
        X = np.array([[0, 0, 0], [1, 0.0, 0], [0.2, 0.01, 0.05], [1.3, 0.02, 0.05]]) * s
        is_ee, eps = True, 1e-3 * s ** 4
    X = X + rng.normal(scale=1e-3 * s * 0.01, size=X.shape)
    G, gfd, H, Hfd = _fd_pair(X, is_ee, eps, dhat)
    assert np.abs(G).max() > 0
    assert np.allclose(G, gfd, rtol=1e-5, atol=1e-5 * np.abs(G).max())
    assert np.allclose(H, Hfd, rtol=1e-4, atol=1e-4 * np.abs(H).max())


def test_mollifier_smooth_at_threshold():
    dhat = 1e-4
    s = 1e-3
    base = np.array([[0, 0, 0], [1, 0.0, 0], [0.2, 0.0, 0.05], [1.3, 0.0, 0.05]]) * s
    # rotate edge b about z so that |a x b|^2 sweeps across eps
    eps = 1e-3 * np.sum((base[1] - base[0]) ** 2) * np.sum((base[3] - base[2]) ** 2)
    Es = []
    for ang in np.linspace(0.0, 0.1, 400):
        X = base.copy()
        c, sn = np.cos(ang), np.sin(ang)
        mid = 0.5 * (X[2] + X[3])
        for i in (2, 3):
            r = X[i] - mid
            X[i] = mid + np.array([c * r[0] - sn * r[1], sn * r[0] + c * r[1], r[2]])
        Es.append(ds.pair_barrier(X[None], np.array([True]), np.ones(1), np.array([eps]), dhat, order=0)[0][0])
    Es = np.array(Es)
    assert Es[0] == 0.0                       # parallel: mollified to zero
    assert np.all(np.abs(np.diff(Es)) < 0.05 * Es.max())   # no jumps


def _sqrtm_sym(M):
    """Principal square root of a symmetric PSD matrix by Denman-Beavers
    iteration (no eigendecomposition)."""
    Y, Z = M.copy(), np.eye(M.shape[0])
    for _ in range(60):
        Y, Z = 0.5 * (Y + np.linalg.inv(Z)), 0.5 * (Z + np.linalg.inv(Y))
    return Y


def test_absolute_value_filter_is_the_matrix_modulus():
    # |H| = (H^2)^(1/2): the absolute-value filter computed by another route
    rng = np.random.default_rng(5)
    for n in (9, 12):
        A = rng.normal(size=(n, n))
        H = A + A.T
        ref = _sqrtm_sym(H @ H)
        assert np.allclose(en.psd_abs(H[None])[0], ref, atol=1e-9 * np.abs(ref).max())
        # PSD input unchanged, NSD input negated, clamp <= abs in the PSD order
        P = A @ A.T
        assert np.allclose(en.psd_abs(P[None])[0], P, atol=1e-10 * np.abs(P).max())
        assert np.allclose(en.psd_abs(-P[None])[0], P, atol=1e-10 * np.abs(P).max())
        d = en.psd_abs(H[None])[0] - en.psd_clamp(H[None])[0]
        assert np.linalg.eigvalsh(d).min() > -1e-9 * np.abs(H).max()
        # and |H| - clamp(H) is the clamp of -H
        assert np.allclose(d, en.psd_clamp(-H[None])[0], atol=1e-9 * np.abs(H).max())


def test_elastic_abs_filter_on_a_compressed_tet():
    mu, lam = lame(3e5, 0.45)
    X, Dmi, V = _tet(RNG)
    x = X.copy()
    x[3] = x[0] + 0.45 * (X[3] - X[0])
    A = en.dPdF(en.deformation_gradient(x[None], Dmi), mu, lam)[0]
    assert np.linalg.eigvalsh(A).min() < 0
    B = en.dF_dx(Dmi)[0]
    want = V[0] * B.T @ _sqrtm_sym(A @ A) @ B
    got = en.tet_hess(x[None], Dmi, V, mu, lam, project="abs")[0]
    assert np.allclose(got, want, atol=1e-8 * np.abs(want).max())
    assert np.linalg.eigvalsh(got).min() > -1e-9 * np.abs(got).max()
