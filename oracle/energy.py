"""Per-element energies, gradients and PSD-projected Hessians (oracle side).

Elastic (Sec. 3.1 / App. A.1): the paper names the neo-Hookean model with
parameters (E, nu) but prints no density.  Reading: the IPC-standard form
    Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2,  J = det F,
    mu = E / (2 (1 + nu)),  lam = E nu / ((1 + nu)(1 - 2 nu)),
with Psi = +inf for J <= 0 (inversion-free, Sec. 1 claims).  F = D_s D_m^{-1}.
First Piola-Kirchhoff stress and its derivative (textbook):
    P = mu F - mu F^{-T} + lam ln J F^{-T}
    dP_ij/dF_kl = mu d_ik d_jl + (mu - lam ln J) G_il G_kj + lam G_ij G_kl,
    G = F^{-T}.
The projected element Hessian is V_e B^T Pi(dP/dF) B where B = dF/dx (9x12)
and Pi filters the negative eigenvalues of the symmetric 9x9 dP/dF
(numpy.linalg.eigh): set to zero ("clamp"), or replaced by their absolute
values ("abs"); both give a PSD matrix.  The paper does not say how its
Hessians are made PSD: the step clamps by default (oracle/step.py,
newton_filter).

Affine body (Sec. 3.3, Eq. unified_ipc): inertia 1/2 (y - ytilde)^T M^y
(y - ytilde), gravity -m g.p, and the stiffness term on A read as the
orthogonality potential kappa_s V_b ||A^T A - I||_F^2 (the paper's ARAP term
with large kappa_s).  Its gradient and Hessian are derived symbolically
(sympy) from that polynomial; the 9x9 affine block is clamped to PSD.
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sp


# ----------------------------------------------------------------------------
# neo-Hookean
# ----------------------------------------------------------------------------
def deformation_gradient(x4: np.ndarray, Dm_inv: np.ndarray) -> np.ndarray:
    """x4: (T, 4, 3) vertex positions -> F (T, 3, 3)."""
    Ds = np.stack([x4[:, 1] - x4[:, 0], x4[:, 2] - x4[:, 0], x4[:, 3] - x4[:, 0]], axis=-1)
    return Ds @ Dm_inv


def psi(F: np.ndarray, mu: float, lam) -> np.ndarray:
    J = np.linalg.det(F)
    with np.errstate(invalid="ignore", divide="ignore"):
        lnJ = np.where(J > 0.0, np.log(np.where(J > 0.0, J, 1.0)), 0.0)
        val = 0.5 * mu * (np.einsum("tij,tij->t", F, F) - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2
    return np.where(J > 0.0, val, np.inf)


def piola(F: np.ndarray, mu: float, lam) -> np.ndarray:
    J = np.linalg.det(F)
    G = np.transpose(np.linalg.inv(F), (0, 2, 1))
    lnJ = np.log(J)
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), J.shape)
    return mu * F - mu * G + (lam * lnJ)[:, None, None] * G


def dPdF(F: np.ndarray, mu: float, lam) -> np.ndarray:
    """(T, 9, 9) with row index 3i+j (P_ij) and column index 3k+l (F_kl)."""
    J = np.linalg.det(F)
    G = np.transpose(np.linalg.inv(F), (0, 2, 1))
    lnJ = np.log(J)
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), J.shape)
    eye = np.eye(3)
    t1 = mu * np.einsum("ik,jl->ijkl", eye, eye)[None]
    t2 = (mu - lam * lnJ)[:, None, None, None, None] * np.einsum("til,tkj->tijkl", G, G)
    t3 = lam[:, None, None, None, None] * np.einsum("tij,tkl->tijkl", G, G)
    return (t1 + t2 + t3).reshape(-1, 9, 9)


def dF_dx(Dm_inv: np.ndarray) -> np.ndarray:
    """B (T, 9, 12): dF_ij / dx_{v,c} for the four vertices v and axes c."""
    T = Dm_inv.shape[0]
    B = np.zeros((T, 3, 3, 4, 3))
    colsum = Dm_inv.sum(axis=1)          # (T, 3): sum_a Dm_inv[a, j]
    for i in range(3):
        B[:, i, :, 0, i] = -colsum
        for v in range(1, 4):
            B[:, i, :, v, i] = Dm_inv[:, v - 1, :]
    return B.reshape(T, 9, 12)


def psd_clamp(H: np.ndarray) -> np.ndarray:
    """Symmetric PSD projection V max(L, 0) V^T (batched)."""
    Hs = 0.5 * (H + np.swapaxes(H, -1, -2))
    w, V = np.linalg.eigh(Hs)
    return np.einsum("...ik,...k,...jk->...ij", V, np.maximum(w, 0.0), V)


def psd_abs(H: np.ndarray) -> np.ndarray:
    """Symmetric PSD projection V |L| V^T (batched)."""
    Hs = 0.5 * (H + np.swapaxes(H, -1, -2))
    w, V = np.linalg.eigh(Hs)
    return np.einsum("...ik,...k,...jk->...ij", V, np.abs(w), V)


def psd_filter(H: np.ndarray, project) -> np.ndarray:
    """project: False / None = raw; True or "clamp" = psd_clamp; "abs" = psd_abs."""
    if not project:
        return H
    if project == "abs":
        return psd_abs(H)
    return psd_clamp(H)


def tet_energy(x4, Dm_inv, vol, mu, lam):
    """Per-tet V_e Psi(F) (T,), +inf where inverted."""
    return vol * psi(deformation_gradient(x4, Dm_inv), mu, lam)


def tet_grad(x4, Dm_inv, vol, mu, lam):
    """(T, 12) gradient of V_e Psi w.r.t. the four vertex positions."""
    F = deformation_gradient(x4, Dm_inv)
    P = piola(F, mu, lam)
    B = dF_dx(Dm_inv)
    return vol[:, None] * np.einsum("tk,tkm->tm", P.reshape(-1, 9), B)


def tet_hess(x4, Dm_inv, vol, mu, lam, project=True):
    """(T, 12, 12) element Hessian, dP/dF filtered to PSD per `project`
    (False: raw; True / "clamp"; "abs")."""
    F = deformation_gradient(x4, Dm_inv)
    A = psd_filter(dPdF(F, mu, lam), project)
    B = dF_dx(Dm_inv)
    return vol[:, None, None] * np.einsum("tkm,tkl,tln->tmn", B, A, B)


# ----------------------------------------------------------------------------
# affine body
# ----------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def _orth_funcs():
    a = sp.symbols("a0:9", real=True)
    # y[3 + 3k + c] = A[c, k]  (column k of A)
    A = sp.Matrix(3, 3, lambda c, k: a[3 * k + c])
    C = A.T * A - sp.eye(3)
    f = sum(C[i, j] ** 2 for i in range(3) for j in range(3))
    g = [sp.diff(f, s) for s in a]
    H = [[sp.diff(gi, s) for s in a] for gi in g]
    fe = sp.lambdify([a], f, "numpy", cse=True)
    ge = sp.lambdify([a], g, "numpy", cse=True)
    he = sp.lambdify([a], H, "numpy", cse=True)
    return fe, ge, he


def orth_energy(yA: np.ndarray) -> float:
    """||A^T A - I||_F^2 for the 9 affine DoFs y[3:12]."""
    return float(_orth_funcs()[0](list(yA)))


def orth_grad(yA: np.ndarray) -> np.ndarray:
    return np.asarray(_orth_funcs()[1](list(yA)), dtype=np.float64)


def orth_hess(yA: np.ndarray) -> np.ndarray:
    return np.asarray(_orth_funcs()[2](list(yA)), dtype=np.float64)


def body_A(y: np.ndarray) -> np.ndarray:
    """Affine matrix A from y = [p, a0, a1, a2] (columns)."""
    return np.stack([y[3:6], y[6:9], y[9:12]], axis=1)


def body_points(y: np.ndarray, xbar: np.ndarray) -> np.ndarray:
    """phi(y): x_j = p + A xbar_j (Sec. 3.3)."""
    return y[:3] + xbar @ body_A(y).T


def body_jacobian(xbar_j: np.ndarray) -> np.ndarray:
    """J_j (3 x 12) = [I, xbar_j0 I, xbar_j1 I, xbar_j2 I]."""
    I = np.eye(3)
    return np.concatenate([I, xbar_j[0] * I, xbar_j[1] * I, xbar_j[2] * I], axis=1)
