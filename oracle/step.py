"""One implicit ABD-IPC time step, projected Newton (oracle side).

Objective (Eq. unified_ipc with the AL term of Eq. unified_ipc_AL):
    E(x, y) = 1/2 |x - xt|_M^2 - h^2 sum_i m_i g.x_i
            + sum_b [1/2 (y_b - yt_b)^T M^y_b (y_b - yt_b) - h^2 m_b g.p_b
                     + h^2 kappa_s V_b |A_b^T A_b - I|_F^2]
            + h^2 sum_e V_e Psi(F_e)
            + h^2 kappa sum_k A_k c_k b(d_k)
            + h^2 sum_k mu lambda_k^n f0(|u_k|)          (lagged friction, when mu > 0)
            + sum_{c driven} [kappa_A/2 |q_c - s_c|_{M_c}^2 - lambda_c^T M_c (q_c - s_c)]
with xt = x^n + h v^n, yt = y^n + h ydot^n (App. A.2) and the backward-Euler
velocity update v^{n+1} = (x^{n+1} - x^n) / h.

Readings (the paper is silent or garbled on these):
  * h^2 multiplies every potential, the barrier included.
  * pinned gel vertices (targets equal to their current position) are
    eliminated; driven DoFs (scripted bodies, gel vertices attached to a
    body) use the augmented Lagrangian the paper names, in its standard
    mass-weighted form (the printed squared scalar is not an AL), with the
    multiplier update lambda <- lambda - kappa_A (q - s) once the inner
    Newton loop has converged and the constraint residual is still above
    tolerance.
  * line search starts at min(1, alpha_CCD) and halves until the energy
    does not increase and no tet is inverted (cap ls_max halvings).
  * Newton stops when |p|_inf / h < tol, p measured as full-space
    vertex displacements (gel p and J_j p_y on body vertices).
  * the Hessians are made PSD by clamping negative eigenvalues to zero
    (optionally, from Newton iteration newton_abs_after on, by replacing
    them with their absolute values: newton_filter).
  * the linear solve is a sparse direct solve here (the GPU uses PCG).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import energy as en
from . import friction as fr
from .broadphase import candidates, excluded_object_pairs
from .ccd import accd_batch
from .distance import pair_barrier, pair_distance
from .rest import body_rest, gel_rest, surface_data

OK, ENOTCONV = 0, 3


@dataclass
class StepStats:
    status: int = OK
    newton_iters: int = 0
    ls_halvings: int = 0
    al_updates: int = 0
    n_pt: int = 0
    n_ee: int = 0
    min_dist: float = np.inf
    min_J: float = np.inf
    energies: list = field(default_factory=list)   # (E_before, E_after) per line search
    ctx: dict = field(default_factory=dict)         # final targets and multipliers


class OracleEnv:
    """Oracle for one environment (scene + solver parameters)."""

    def __init__(self, scene, params):
        self.scene = scene
        self.prm = params
        self.gel = gel_rest(scene)
        self.bodies = [body_rest(b) for b in scene.bodies]
        self.sd = surface_data(scene, self.bodies)
        self.N = scene.n_verts
        self.nb = len(scene.bodies)
        self.ndof = 3 * self.N + 12 * self.nb
        self.excluded = excluded_object_pairs(scene)
        # degree-of-freedom map of contact vertices: (ncv, 3, 4) ids / weights
        ncv = self.N + int(self.sd.body_vert_off[-1])
        dof = np.zeros((ncv, 3, 4), np.int64)
        w = np.zeros((ncv, 3, 4))
        for c in range(3):
            dof[:self.N, c, 0] = 3 * np.arange(self.N) + c
            w[:self.N, c, 0] = 1.0
        for b, br in enumerate(self.bodies):
            o = self.N + self.sd.body_vert_off[b]
            n = br.xbar.shape[0]
            base = 3 * self.N + 12 * b
            for c in range(3):
                dof[o:o + n, c, 0] = base + c
                w[o:o + n, c, 0] = 1.0
                for k in range(3):
                    dof[o:o + n, c, 1 + k] = base + 3 + 3 * k + c
                    w[o:o + n, c, 1 + k] = br.xbar[:, k]
        self.cv_dof, self.cv_w = dof, w
        # free DoFs: everything but pinned gel vertices
        free = np.ones(self.ndof, bool)
        pin = np.nonzero(scene.pinned)[0]
        for c in range(3):
            free[3 * pin + c] = False
        self.free = free
        # driven sets
        self.driven_bodies = [b for b, bd in enumerate(scene.bodies) if bd.driven]
        self.attached = np.nonzero(scene.attach >= 0)[0]
        self.attach_body = scene.attach[self.attached]
        self.attach_xbar = (scene.gel_x[self.attached]
                            - np.array([self.bodies[b].com for b in self.attach_body]).reshape(-1, 3))
        g = np.asarray(params.gravity, dtype=np.float64)
        self.g = g

    # ------------------------------------------------------------------
    # state helpers
    # ------------------------------------------------------------------
    def rest_y(self) -> np.ndarray:
        y = np.zeros((self.nb, 12))
        for b, br in enumerate(self.bodies):
            y[b, :3] = br.com
            y[b, 3:] = np.eye(3).T.ravel()   # columns of I
        return y

    def rest_state(self):
        return (self.scene.gel_x.copy(), np.zeros((self.N, 3)), self.rest_y(), np.zeros((self.nb, 12)))

    def targets_from_delta(self, delta: np.ndarray) -> np.ndarray:
        """Body targets [com + delta, I] from rest-placement translations."""
        s = self.rest_y()
        s[:, :3] += delta[:, :3]
        return s

    def contact_positions(self, x, y):
        parts = [x]
        for b, br in enumerate(self.bodies):
            parts.append(en.body_points(y[b], br.xbar))
        return np.concatenate(parts) if len(parts) > 1 else x

    def split(self, q):
        return q[:3 * self.N].reshape(self.N, 3), q[3 * self.N:].reshape(self.nb, 12)

    def join(self, x, y):
        return np.concatenate([x.ravel(), y.ravel()])

    # ------------------------------------------------------------------
    # pair data
    # ------------------------------------------------------------------
    def pair_arrays(self, pt, ee):
        sd = self.sd
        pts = np.concatenate([np.concatenate([pt[:, :1], sd.tris[pt[:, 1]]], axis=1),
                              np.concatenate([sd.edges[ee[:, 0]], sd.edges[ee[:, 1]]], axis=1)]) \
            if (len(pt) + len(ee)) else np.zeros((0, 4), np.int64)
        is_ee = np.concatenate([np.zeros(len(pt), bool), np.ones(len(ee), bool)])
        pidx = np.searchsorted(sd.points, pt[:, 0]) if len(pt) else np.zeros(0, np.int64)
        area = np.concatenate([0.5 * sd.point_area[pidx],
                               0.25 * (sd.edge_area[ee[:, 0]] + sd.edge_area[ee[:, 1]])])
        eps = np.concatenate([np.zeros(len(pt)),
                              self.prm.ee_mollifier * sd.edge_rest_len2[ee[:, 0]] * sd.edge_rest_len2[ee[:, 1]]])
        return pts, is_ee, area, eps

    # ------------------------------------------------------------------
    # energy / gradient / Hessian
    # ------------------------------------------------------------------
    def energy(self, x, y, ctx, pairs) -> float:
        """Total objective at (x, y); +inf if inverted or any pair touches."""
        prm, h = self.prm, self.prm.dt
        m = self.gel.mass
        E = 0.5 * np.sum(m[:, None] * (x - ctx["xt"]) ** 2) - h * h * np.sum(m * (x @ self.g))
        T = self.scene.gel_tets
        Ee = en.tet_energy(x[T], self.gel.Dm_inv, self.gel.vol, self.gel.mu, self.gel.lam)
        if not np.all(np.isfinite(Ee)):
            return np.inf
        E += h * h * np.sum(Ee)
        for b, br in enumerate(self.bodies):
            dy = y[b] - ctx["yt"][b]
            E += 0.5 * dy @ br.My @ dy - h * h * br.mass * (y[b, :3] @ self.g)
            E += h * h * self.scene.bodies[b].kappa_s * br.vol * en.orth_energy(y[b, 3:])
        E += self._al_energy(x, y, ctx)
        pts, is_ee, area, eps = pairs
        if len(pts):
            X12 = self.contact_positions(x, y)[pts]
            d = pair_distance(X12, is_ee)
            if np.any(d <= 0.0):
                return np.inf
            Eb, _, _ = pair_barrier(X12, is_ee, h * h * prm.kappa * area, eps, prm.dhat, order=0)
            E += np.sum(Eb)
        ft = self._friction_terms(x, y, ctx, 0)
        if ft is not None:
            E += h * h * float(np.sum(ft[0]))
        return float(E)

    def _al_energy(self, x, y, ctx):
        ka = self.prm.al_kappa
        E = 0.0
        for b in self.driven_bodies:
            r = y[b] - ctx["s_y"][b]
            My = self.bodies[b].My
            E += 0.5 * ka * r @ My @ r - ctx["lam_y"][b] @ My @ r
        if len(self.attached):
            r = x[self.attached] - ctx["s_x"]
            m = self.gel.mass[self.attached]
            E += 0.5 * ka * np.sum(m[:, None] * r * r) - np.sum(m[:, None] * ctx["lam_x"] * r)
        return E

    def grad_hess(self, x, y, ctx, pairs, project=True):
        """Full gradient (ndof,) and Hessian (sparse ndof x ndof); project:
        the eigenvalue filter of the element, body and pair Hessians (False:
        raw, True / "clamp", "abs")."""
        prm, h = self.prm, self.prm.dt
        N = self.N
        m = self.gel.mass
        g = np.zeros(self.ndof)
        rows, cols, vals = [], [], []
        # gel inertia + gravity
        g[:3 * N] += (m[:, None] * (x - ctx["xt"])).ravel() - h * h * (m[:, None] * self.g[None]).ravel()
        di = np.arange(3 * N)
        rows.append(di); cols.append(di); vals.append(np.repeat(m, 3))
        # elastic
        T = self.scene.gel_tets
        ge = en.tet_grad(x[T], self.gel.Dm_inv, self.gel.vol, self.gel.mu, self.gel.lam)
        He = en.tet_hess(x[T], self.gel.Dm_inv, self.gel.vol, self.gel.mu, self.gel.lam, project=project)
        ed = (3 * T[:, :, None] + np.arange(3)[None, None]).reshape(-1, 12)
        np.add.at(g, ed.ravel(), (h * h * ge).ravel())
        rows.append(np.repeat(ed, 12, axis=1).ravel())
        cols.append(np.tile(ed, (1, 12)).ravel())
        vals.append((h * h * He).ravel())
        # bodies
        ka = prm.al_kappa
        for b, br in enumerate(self.bodies):
            o = 3 * N + 12 * b
            dy = y[b] - ctx["yt"][b]
            gb = br.My @ dy
            gb[:3] -= h * h * br.mass * self.g
            ks = self.scene.bodies[b].kappa_s
            gb[3:] += h * h * ks * br.vol * en.orth_grad(y[b, 3:])
            Hb = br.My.copy()
            Ho = h * h * ks * br.vol * en.orth_hess(y[b, 3:])
            Hb[3:, 3:] += en.psd_filter(Ho, project)
            if b in self.driven_bodies:
                r = y[b] - ctx["s_y"][b]
                gb += ka * br.My @ r - br.My @ ctx["lam_y"][b]
                Hb += ka * br.My
            g[o:o + 12] += gb
            ii = o + np.arange(12)
            rows.append(np.repeat(ii, 12)); cols.append(np.tile(ii, 12)); vals.append(Hb.ravel())
        # attached gel vertices
        if len(self.attached):
            r = x[self.attached] - ctx["s_x"]
            ma = m[self.attached]
            ga = ka * ma[:, None] * r - ma[:, None] * ctx["lam_x"]
            ids = (3 * self.attached[:, None] + np.arange(3)[None])
            np.add.at(g, ids.ravel(), ga.ravel())
            rows.append(ids.ravel()); cols.append(ids.ravel()); vals.append(np.repeat(ka * ma, 3))
        # contact
        pts, is_ee, area, eps = pairs
        if len(pts):
            X12 = self.contact_positions(x, y)[pts]
            _, Gk, Hk = pair_barrier(X12, is_ee, h * h * prm.kappa * area, eps, prm.dhat,
                                     order=2, project=project)
            dof = self.cv_dof[pts].reshape(-1, 12, 4)
            w = self.cv_w[pts].reshape(-1, 12, 4)
            np.add.at(g, dof.ravel(), (w * Gk[:, :, None]).ravel())
            act = np.any(Hk != 0.0, axis=(1, 2))
            if np.any(act):
                dA, wA, HA = dof[act], w[act], Hk[act]
                v = wA[:, :, :, None, None] * wA[:, None, None, :, :] * HA[:, :, None, :, None]
                r_ = np.broadcast_to(dA[:, :, :, None, None], v.shape)
                c_ = np.broadcast_to(dA[:, None, None, :, :], v.shape)
                nz = v != 0.0
                rows.append(r_[nz]); cols.append(c_[nz]); vals.append(v[nz])
        # lagged friction (its tangent-frame Hessian is PSD as it stands)
        ft = self._friction_terms(x, y, ctx, 2)
        if ft is not None:
            _, Gf, Hf = ft
            pts_f = ctx["fric"]["pts"]
            dof = self.cv_dof[pts_f].reshape(-1, 12, 4)
            w = self.cv_w[pts_f].reshape(-1, 12, 4)
            np.add.at(g, dof.ravel(), (w * (h * h * Gf)[:, :, None]).ravel())
            v = w[:, :, :, None, None] * w[:, None, None, :, :] * (h * h * Hf)[:, :, None, :, None]
            r_ = np.broadcast_to(dof[:, :, :, None, None], v.shape)
            c_ = np.broadcast_to(dof[:, None, None, :, :], v.shape)
            nz = v != 0.0
            rows.append(r_[nz]); cols.append(c_[nz]); vals.append(v[nz])
        H = sps.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.ndof, self.ndof)).tocsr()
        return g, H

    # ------------------------------------------------------------------
    # norms used by the stopping rules
    # ------------------------------------------------------------------
    def fullspace_inf(self, px, py) -> float:
        v = np.abs(px).max() if px.size else 0.0
        for b, br in enumerate(self.bodies):
            A = en.body_A(py[b])
            d = py[b, :3] + br.xbar @ A.T
            v = max(v, np.abs(d).max())
        return float(v)

    def constraint_residual(self, x, y, ctx) -> float:
        v = 0.0
        for b in self.driven_bodies:
            r = y[b] - ctx["s_y"][b]
            d = r[:3] + self.bodies[b].xbar @ en.body_A(r).T
            v = max(v, np.abs(d).max())
        if len(self.attached):
            v = max(v, np.abs(x[self.attached] - ctx["s_x"]).max())
        return float(v)

    # ------------------------------------------------------------------
    # the step
    # ------------------------------------------------------------------
    def make_ctx(self, x_n, v_n, y_n, ydot_n, s_y):
        h = self.prm.dt
        ctx = {"xt": x_n + h * v_n, "yt": y_n + h * ydot_n,
               "s_y": np.array(s_y, dtype=np.float64).reshape(self.nb, 12) if self.nb else np.zeros((0, 12)),
               "lam_y": np.zeros((self.nb, 12)), "lam_x": np.zeros((len(self.attached), 3))}
        if len(self.attached):
            sy = ctx["s_y"][self.attach_body]
            A = np.stack([sy[:, 3:6], sy[:, 6:9], sy[:, 9:12]], axis=2)
            ctx["s_x"] = sy[:, :3] + np.einsum("nij,nj->ni", A, self.attach_xbar)
        else:
            ctx["s_x"] = np.zeros((0, 3))
        ctx["fric"] = self._friction_lagged(x_n, y_n)
        return ctx

    def _friction_lagged(self, x_n, y_n):
        """Lagged friction data at x^n (friction module docstring), or None."""
        mu = float(getattr(self.prm, "friction_mu", 0.0))
        if mu <= 0.0:
            return None
        pt, ee = self.static_pairs(x_n, y_n)
        pts, is_ee, area, eps = self.pair_arrays(pt, ee)
        if not len(pts):
            return None
        Xn = self.contact_positions(x_n, y_n)[pts]
        W, T, lam, rn = fr.lagged(Xn, is_ee, self.prm.kappa * area, eps, self.prm.dhat)
        keep = lam > 0.0
        if not np.any(keep):
            return None
        return {"pts": pts[keep], "W": W[keep], "T": T[keep], "lam": lam[keep], "rn": rn[keep],
                "mu": mu, "eh": float(self.prm.friction_eps_v) * self.prm.dt}

    def _friction_terms(self, x, y, ctx, order):
        fc = ctx.get("fric")
        if fc is None:
            return None
        X = self.contact_positions(x, y)[fc["pts"]]
        return fr.pair_friction(X, fc["W"], fc["T"], fc["lam"], fc["rn"], fc["mu"], fc["eh"], order)

    def static_pairs(self, x, y):
        Xc = self.contact_positions(x, y)
        pt, ee = candidates(self.sd, Xc, self.prm.dhat, self.excluded)
        return pt, ee

    def newton_filter(self, it: int) -> str:
        """Eigenvalue filter of Newton iteration `it` (0-based) of a step.
        The paper does not say how its Hessians are made PSD.  Default
        reading: clamp negative eigenvalues to zero.  Option: from iteration
        newton_abs_after on, replace them by their absolute values instead
        (an iterate near a saddle of the energy moves away from it faster;
        measured on the press workload it did not make the slow steps
        converge sooner once the linear solves are inexact, so it is off by
        default)."""
        return "abs" if it >= getattr(self.prm, "newton_abs_after", 1000000) else "clamp"

    def step(self, x_n, v_n, y_n, ydot_n, s_y=None, x_start=None, y_start=None):
        """Advance one time step.  s_y: (nb, 12) body targets (driven rows).
        Newton starts from (x_n, y_n) as in the paper's step; the tests may
        pass another feasible starting iterate (x_start, y_start) to check
        that a candidate end state is a converged point of this step."""
        prm, h = self.prm, self.prm.dt
        if s_y is None:
            s_y = y_n.copy()
        ctx = self.make_ctx(x_n, v_n, y_n, ydot_n, s_y)
        x = (x_n if x_start is None else x_start).copy()
        y = (y_n if y_start is None else y_start).copy()
        st = StepStats()
        has_driven = bool(self.driven_bodies) or len(self.attached) > 0
        converged = False
        for it in range(prm.newton_max):
            st.newton_iters = it + 1
            pt, ee = self.static_pairs(x, y)
            pairs = self.pair_arrays(pt, ee)
            g, H = self.grad_hess(x, y, ctx, pairs, project=self.newton_filter(it))
            f = self.free
            p = np.zeros(self.ndof)
            rhs = -g[f]
            if np.any(rhs != 0.0):
                p[f] = spla.spsolve(H[f][:, f].tocsc(), rhs)
            px, py = self.split(p)
            if self.fullspace_inf(px, py) / h <= prm.newton_tol:
                if not has_driven or self.constraint_residual(x, y, ctx) / h <= prm.newton_tol:
                    converged = True
                    break
                if st.al_updates >= prm.al_max:
                    break
                for b in self.driven_bodies:
                    ctx["lam_y"][b] = ctx["lam_y"][b] - prm.al_kappa * (y[b] - ctx["s_y"][b])
                if len(self.attached):
                    ctx["lam_x"] = ctx["lam_x"] - prm.al_kappa * (x[self.attached] - ctx["s_x"])
                st.al_updates += 1
                continue
            # swept candidates, CCD, line search
            Xc0 = self.contact_positions(x, y)
            Xc1 = self.contact_positions(x + px, y + py)
            spt, see = candidates(self.sd, Xc0, prm.dhat, self.excluded, Xc_end=Xc1)
            sp_pairs = self.pair_arrays(spt, see)
            alpha = 1.0
            if len(sp_pairs[0]):
                toi = accd_batch(Xc0[sp_pairs[0]], (Xc1 - Xc0)[sp_pairs[0]], sp_pairs[1],
                                 s=prm.accd_s, t_max=1.0, max_iter=prm.accd_max)
                alpha = min(1.0, float(toi.min()))
            E0 = self.energy(x, y, ctx, sp_pairs)
            accepted = False
            for ls in range(prm.ls_max):
                xn, yn = x + alpha * px, y + alpha * py
                E1 = self.energy(xn, yn, ctx, sp_pairs)
                if E1 <= E0:
                    accepted = True
                    break
                alpha *= 0.5
                st.ls_halvings += 1
            if not accepted:
                break
            st.energies.append((E0, E1))
            x, y = xn, yn
        if not converged:
            st.status = ENOTCONV
        pt, ee = self.static_pairs(x, y)
        st.n_pt, st.n_ee = len(pt), len(ee)
        pa = self.pair_arrays(pt, ee)
        if len(pa[0]):
            st.min_dist = float(pair_distance(self.contact_positions(x, y)[pa[0]], pa[1]).min())
        T = self.scene.gel_tets
        F = en.deformation_gradient(x[T], self.gel.Dm_inv)
        st.min_J = float(np.linalg.det(F).min())
        v = (x - x_n) / h
        ydot = (y - y_n) / h
        v[self.scene.pinned] = 0.0
        st.ctx = ctx
        return x, v, y, ydot, st
