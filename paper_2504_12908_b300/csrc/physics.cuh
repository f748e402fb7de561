// Per-element physics of the ABD-IPC step, as device functions.
//
//  * neo-Hookean tetrahedron (App. A.1): Psi = mu/2 (|F|^2 - 3) - mu ln J
//    + lam/2 (ln J)^2, its gradient, and the PSD-projected Hessian built
//    from the analytic eigensystem of d2Psi/dF2 in the singular-value frame
//    of F (scaling, twist and flip modes), so no 9x9/12x12 eigensolve runs.
//  * IPC barrier of a point-triangle or edge-edge pair (App. A.3, Eq.
//    ipc_energy) with the edge-edge mollifier; squared-distance derivatives
//    come from the closest-point envelope: D(q) = min_theta |r(q, theta)|^2
//    with r affine in theta, so grad D = 2 W^T r and
//    hess D = f_qq - f_qtheta f_thetatheta^{-1} f_thetaq.
//  * additive CCD time of impact of a pair.
#pragma once

#include "common.cuh"
#ifdef __CUDACC__
#include "ctx.h"
#endif

namespace ipc {

// =====================================================================
// neo-Hookean
// =====================================================================
template <class T>
IPC_HD void tet_deformation(const V3<T>* x, const T* Dmi, T* F) {
  V3<T> e[3] = {x[1] - x[0], x[2] - x[0], x[3] - x[0]};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      F[3 * i + j] = comp3(e[0], i) * Dmi[j] + comp3(e[1], i) * Dmi[3 + j] + comp3(e[2], i) * Dmi[6 + j];
}

template <class T> IPC_HD T comp3(V3<T> v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

template <class T>
IPC_HD T det3(const T* F) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// vol * Psi(F); +inf when J <= 0.
template <class T>
IPC_HD T nh_energy(const T* F, T vol, T mu, T lam) {
  T J = det3(F);
  if (!(J > T(0))) return T(INFINITY);
  T I1 = 0;
  for (int k = 0; k < 9; ++k) I1 += F[k] * F[k];
  T lnJ = log(J);
  return vol * (T(0.5) * mu * (I1 - T(3)) - mu * lnJ + T(0.5) * lam * lnJ * lnJ);
}

// Gradient w.r.t. the four vertices: g[3a + i].
template <class T>
IPC_HD void nh_gradient(const T* F, const T* Dmi, T vol, T mu, T lam, T* g) {
  T J = det3(F);
  T cof[9];
  cof[0] = F[4] * F[8] - F[5] * F[7];
  cof[1] = F[5] * F[6] - F[3] * F[8];
  cof[2] = F[3] * F[7] - F[4] * F[6];
  cof[3] = F[2] * F[7] - F[1] * F[8];
  cof[4] = F[0] * F[8] - F[2] * F[6];
  cof[5] = F[1] * F[6] - F[0] * F[7];
  cof[6] = F[1] * F[5] - F[2] * F[4];
  cof[7] = F[2] * F[3] - F[0] * F[5];
  cof[8] = F[0] * F[4] - F[1] * F[3];
  T lnJ = log(J);
  T c = (lam * lnJ - mu) / J;  // P = mu F + (lam lnJ - mu) F^{-T},  F^{-T} = cof / J
  T P[9];
  for (int k = 0; k < 9; ++k) P[k] = mu * F[k] + c * cof[k];
  for (int i = 0; i < 3; ++i) {
    T s = 0;
    for (int a = 1; a < 4; ++a) {
      T v = vol * (P[3 * i] * Dmi[3 * (a - 1)] + P[3 * i + 1] * Dmi[3 * (a - 1) + 1] +
                   P[3 * i + 2] * Dmi[3 * (a - 1) + 2]);
      g[3 * a + i] = v;
      s += v;
    }
    g[i] = -s;
  }
}

// SVD of a 3x3 F (det F > 0) by Jacobi on F^T F; U, V row-major with
// columns u_k, v_k, det U = det V = +1, F = U diag(s) V^T.
template <class T>
IPC_HD void svd3(const T* F, T* U, T* s, T* V) {
  T C[9], W[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  jacobi_eigen<3, T>(C, V, 20);
  // det V = +1
  T dV = det3(V);
  if (dV < T(0)) for (int i = 0; i < 3; ++i) V[3 * i + 2] = -V[3 * i + 2];
  // b_k = F v_k
  T b[3][3];
  T nb[3];
  for (int k = 0; k < 3; ++k) {
    for (int i = 0; i < 3; ++i) b[k][i] = F[3 * i] * V[k] + F[3 * i + 1] * V[3 + k] + F[3 * i + 2] * V[6 + k];
    nb[k] = b[k][0] * b[k][0] + b[k][1] * b[k][1] + b[k][2] * b[k][2];
  }
  // order by |b_k| descending: k0, k1, k2
  int k0 = 0, k1 = 1, k2 = 2;
  if (nb[k1] > nb[k0]) { int t = k0; k0 = k1; k1 = t; }
  if (nb[k2] > nb[k0]) { int t = k0; k0 = k2; k2 = t; }
  if (nb[k2] > nb[k1]) { int t = k1; k1 = k2; k2 = t; }
  T u[3][3];
  T n0 = sqrt(nb[k0]);
  for (int i = 0; i < 3; ++i) u[k0][i] = b[k0][i] / n0;
  T pr = u[k0][0] * b[k1][0] + u[k0][1] * b[k1][1] + u[k0][2] * b[k1][2];
  T w1[3] = {b[k1][0] - pr * u[k0][0], b[k1][1] - pr * u[k0][1], b[k1][2] - pr * u[k0][2]};
  T nw = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
  if (nw > T(0)) {
    for (int i = 0; i < 3; ++i) u[k1][i] = w1[i] / nw;
  } else {  // any unit vector orthogonal to u_k0
    T a[3] = {T(1), T(0), T(0)};
    if (fabs(u[k0][0]) > T(0.9)) { a[0] = 0; a[1] = 1; }
    T d = a[0] * u[k0][0] + a[1] * u[k0][1] + a[2] * u[k0][2];
    T w[3] = {a[0] - d * u[k0][0], a[1] - d * u[k0][1], a[2] - d * u[k0][2]};
    T nn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int i = 0; i < 3; ++i) u[k1][i] = w[i] / nn;
  }
  // u_k2 completes a right-handed frame consistent with the index order
  bool even = (k0 == 0 && k1 == 1) || (k0 == 1 && k1 == 2) || (k0 == 2 && k1 == 0);
  T* ua = even ? u[k0] : u[k1];
  T* ub = even ? u[k1] : u[k0];
  u[k2][0] = ua[1] * ub[2] - ua[2] * ub[1];
  u[k2][1] = ua[2] * ub[0] - ua[0] * ub[2];
  u[k2][2] = ua[0] * ub[1] - ua[1] * ub[0];
  for (int k = 0; k < 3; ++k) {
    s[k] = u[k][0] * b[k][0] + u[k][1] * b[k][1] + u[k][2] * b[k][2];
    for (int i = 0; i < 3; ++i) U[3 * i + k] = u[k][i];
  }
}

// Eigenvalue filter of a projected Hessian: FILT_NONE keeps the raw
// Hessian, FILT_CLAMP sets negative eigenvalues to zero, FILT_ABS replaces
// them by their absolute values (both give a PSD matrix).
enum { FILT_NONE = 0, FILT_CLAMP = 1, FILT_ABS = 2 };

#ifdef __CUDACC__
// Filter of env e's current Newton iteration: clamping for the first
// Dev::abs_after iterations of a step, absolute values after that (by
// default abs_after exceeds any Newton cap: clamping throughout).
__device__ __forceinline__ int newton_filter(const Dev& d, int e) {
  return d.env_i[e * NUM_INTS + I_NEWTON] > d.abs_after ? FILT_ABS : FILT_CLAMP;
}
#endif

// Projected 9x9 d2Psi/dF2 (index 3i+j <-> F_ij), upper triangle packed into
// Pi[45] row by row; filt: FILT_NONE / FILT_CLAMP / FILT_ABS.
template <class T>
IPC_HD void nh_projected_dPdF(const T* F, T mu, T lam, T* Pi, int filt = FILT_CLAMP) {
  T U[9], V[9], s[3];
  svd3(F, U, s, V);
  T lnJ = log(s[0] * s[1] * s[2]);
  T c = mu - lam * lnJ;
  for (int k = 0; k < 45; ++k) Pi[k] = 0;
  auto add_mode = [&](T lmb, const T* Q) {
    if (filt == FILT_ABS) lmb = fabs(lmb);
    if (filt != FILT_NONE && !(lmb > T(0))) return;
    int idx = 0;
    for (int a = 0; a < 9; ++a)
      for (int b = a; b < 9; ++b) Pi[idx++] += lmb * Q[a] * Q[b];
  };
  // scaling modes: eigen-decomposition of d2psi/dsigma2
  T A[9], Z[9];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      A[3 * k + l] = (k == l) ? (mu + (c + lam) / (s[k] * s[k])) : lam / (s[k] * s[l]);
  jacobi_eigen<3, T>(A, Z, 20);
  T Q[9];
  for (int m = 0; m < 3; ++m) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T q = 0;
        for (int k = 0; k < 3; ++k) q += Z[3 * k + m] * U[3 * i + k] * V[3 * j + k];
        Q[3 * i + j] = q;
      }
    add_mode(A[4 * m], Q);
  }
  // twist (u_i v_j^T - u_j v_i^T)/sqrt2 and flip (+) modes
  const T r2 = T(0.70710678118654752440);
  for (int p = 0; p < 2; ++p)
    for (int q = p + 1; q < 3; ++q) {
      T ss = s[p] * s[q];
      T lt = mu - c / ss;
      T lf = mu + c / ss;
      for (int sign = 0; sign < 2; ++sign) {
        T sg = sign == 0 ? T(-1) : T(1);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            Q[3 * i + j] = r2 * (U[3 * i + p] * V[3 * j + q] + sg * U[3 * i + q] * V[3 * j + p]);
        add_mode(sign == 0 ? lt : lf, Q);
      }
    }
}

IPC_HD int sym9(int a, int b) {  // packed index of (a, b), a, b in [0, 9)
  if (a > b) { int t = a; a = b; b = t; }
  return a * 9 - a * (a - 1) / 2 + (b - a);
}

// Projected element Hessian, all 16 3x3 blocks: H[(a*4+b)*9 + i*3 + j]
// = vol * sum_{n,n'} D_a[n] Pi[(i,n),(j,n')] D_b[n'].
template <class T, class Out>
IPC_HD void nh_hessian_blocks(const T* F, const T* Dmi, T vol, T mu, T lam, Out&& out, int filt = FILT_CLAMP) {
  T Pi[45];
  nh_projected_dPdF(F, mu, lam, Pi, filt);
  T D[4][3];
  for (int n = 0; n < 3; ++n) {
    D[1][n] = Dmi[n];
    D[2][n] = Dmi[3 + n];
    D[3][n] = Dmi[6 + n];
    D[0][n] = -(D[1][n] + D[2][n] + D[3][n]);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // t_b[n] = sum_n' Pi[(i,n),(j,n')] D_b[n']
      T t[4][3];
      for (int b = 0; b < 4; ++b)
        for (int n = 0; n < 3; ++n) {
          T acc = 0;
          for (int m = 0; m < 3; ++m) acc += Pi[sym9(3 * i + n, 3 * j + m)] * D[b][m];
          t[b][n] = acc;
        }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          out(a, b, i, j, vol * (D[a][0] * t[b][0] + D[a][1] * t[b][1] + D[a][2] * t[b][2]));
    }
}

// =====================================================================
// distances and barrier
// =====================================================================
enum DistKind { K_PP = 0, K_PE = 1, K_PT = 2, K_EE = 3 };

// Closest-feature description of a pair: r = sum_i w_i x_i with w affine in
// up to two parameters theta (dw_i/dtheta_m = c[i][m]) and R_m = dr/dtheta_m.
struct Closest {
  int kind;
  int k;          // number of parameters
  double w[4];
  double c[4][2];
  D3 r;
  D3 R[2];
  double D;       // squared distance
};

IPC_D void point_segment(D3 p, D3 e0, D3 e1, double& d2, int& kind /*0 PP e0,1 PP e1,2 PE*/, double& t) {
  D3 e = e1 - e0;
  t = dot(p - e0, e) / dot(e, e);
  double tc = fmin(fmax(t, 0.0), 1.0);
  D3 c = e0 + tc * e;
  d2 = norm2(p - c);
  kind = (t <= 0.0) ? 0 : ((t >= 1.0) ? 1 : 2);
}

// Fill `cl` for the point-segment closest feature of point index ip against
// the segment (i0, i1) given its classification.
IPC_D void closest_ps(const D3* X, int ip, int i0, int i1, int pk, double t, Closest& cl) {
  for (int i = 0; i < 4; ++i) { cl.w[i] = 0; cl.c[i][0] = cl.c[i][1] = 0; }
  if (pk == 2) {
    cl.kind = K_PE;
    cl.k = 1;
    cl.w[ip] = 1.0;
    cl.w[i0] = -(1.0 - t);
    cl.w[i1] = -t;
    cl.c[i0][0] = 1.0;
    cl.c[i1][0] = -1.0;
    cl.R[0] = X[i0] - X[i1];
    cl.r = X[ip] - ((1.0 - t) * X[i0] + t * X[i1]);
  } else {
    int q = pk == 0 ? i0 : i1;
    cl.kind = K_PP;
    cl.k = 0;
    cl.w[ip] = 1.0;
    cl.w[q] = -1.0;
    cl.r = X[ip] - X[q];
  }
  cl.D = norm2(cl.r);
}

// Point (X[0]) - triangle (X[1..3]).
IPC_D void classify_pt(const D3* X, Closest& cl) {
  D3 e0 = X[2] - X[1], e1 = X[3] - X[1], w = X[0] - X[1];
  double a = dot(e0, e0), b = dot(e0, e1), c = dot(e1, e1), d = dot(e0, w), e = dot(e1, w);
  double det = a * c - b * b;
  double b1 = (c * d - b * e) / det;
  double b2 = (a * e - b * d) / det;
  if (b1 >= 0.0 && b2 >= 0.0 && b1 + b2 <= 1.0) {
    cl.kind = K_PT;
    cl.k = 2;
    cl.w[0] = 1.0;
    cl.w[1] = -(1.0 - b1 - b2);
    cl.w[2] = -b1;
    cl.w[3] = -b2;
    cl.c[0][0] = cl.c[0][1] = 0.0;
    cl.c[1][0] = 1.0; cl.c[1][1] = 1.0;
    cl.c[2][0] = -1.0; cl.c[2][1] = 0.0;
    cl.c[3][0] = 0.0; cl.c[3][1] = -1.0;
    cl.R[0] = X[1] - X[2];
    cl.R[1] = X[1] - X[3];
    cl.r = w - b1 * e0 - b2 * e1;
    cl.D = norm2(cl.r);
    return;
  }
  const int seg[3][2] = {{1, 2}, {2, 3}, {3, 1}};
  double best = INFINITY;
  int bs = 0, bk = 0;
  double bt = 0;
  for (int s = 0; s < 3; ++s) {
    double d2, t;
    int k;
    point_segment(X[0], X[seg[s][0]], X[seg[s][1]], d2, k, t);
    if (d2 < best) { best = d2; bs = s; bk = k; bt = t; }
  }
  closest_ps(X, 0, seg[bs][0], seg[bs][1], bk, bt, cl);
}

// Edge (X[0], X[1]) - edge (X[2], X[3]).
IPC_D void classify_ee(const D3* X, Closest& cl) {
  D3 a = X[1] - X[0], b = X[3] - X[2], w = X[0] - X[2];
  double aa = dot(a, a), bb = dot(b, b), ab = dot(a, b), aw = dot(a, w), bw = dot(b, w);
  double det = aa * bb - ab * ab;
  if (det > 1e-20 * aa * bb) {
    double s = (ab * bw - bb * aw) / det;
    double t = (aa * bw - ab * aw) / det;
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
      cl.kind = K_EE;
      cl.k = 2;
      cl.w[0] = 1.0 - s; cl.w[1] = s; cl.w[2] = -(1.0 - t); cl.w[3] = -t;
      cl.c[0][0] = -1.0; cl.c[0][1] = 0.0;
      cl.c[1][0] = 1.0;  cl.c[1][1] = 0.0;
      cl.c[2][0] = 0.0;  cl.c[2][1] = 1.0;
      cl.c[3][0] = 0.0;  cl.c[3][1] = -1.0;
      cl.R[0] = a;
      cl.R[1] = -1.0 * b;
      cl.r = w + s * a - t * b;
      cl.D = norm2(cl.r);
      return;
    }
  }
  const int cmb[4][3] = {{0, 2, 3}, {1, 2, 3}, {2, 0, 1}, {3, 0, 1}};
  double best = INFINITY;
  int bc = 0, bk = 0;
  double bt = 0;
  for (int m = 0; m < 4; ++m) {
    double d2, t;
    int k;
    point_segment(X[cmb[m][0]], X[cmb[m][1]], X[cmb[m][2]], d2, k, t);
    if (d2 < best) { best = d2; bc = m; bk = k; bt = t; }
  }
  closest_ps(X, cmb[bc][0], cmb[bc][1], cmb[bc][2], bk, bt, cl);
}

IPC_D void classify(const D3* X, bool is_ee, Closest& cl) {
  for (int i = 0; i < 4; ++i) { cl.w[i] = 0; cl.c[i][0] = cl.c[i][1] = 0; }
  if (is_ee) classify_ee(X, cl); else classify_pt(X, cl);
}

IPC_D double pair_sqdist(const D3* X, bool is_ee) {
  Closest cl;
  classify(X, is_ee, cl);
  return cl.D;
}

// grad D (12, FP64) from the closest-feature data.
IPC_D void sqdist_grad(const Closest& cl, double* gD) {
  for (int i = 0; i < 4; ++i) {
    gD[3 * i + 0] = 2.0 * cl.w[i] * cl.r.x;
    gD[3 * i + 1] = 2.0 * cl.w[i] * cl.r.y;
    gD[3 * i + 2] = 2.0 * cl.w[i] * cl.r.z;
  }
}

// hess D (12x12 row-major) in T from the closest-feature data:
// 2 (w w^T) (x) I3 - F Mi F^T.  The k x k system Mi (nearly singular for
// near-parallel edges) and the factor F Mi are formed in FP64 and only the
// final outer products in T, so T = float loses no more than its rounding
// of well-scaled factors.
template <class T>
IPC_D void sqdist_hess(const Closest& cl, T* HD) {
  // f_qq = 2 (w w^T) (x) I3
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      T v = T(2) * (T)cl.w[i] * (T)cl.w[j];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) HD[(3 * i + a) * 12 + 3 * j + b] = (a == b) ? v : T(0);
    }
  if (cl.k == 0) return;
  // f_qtheta (12 x k) and f_thetatheta^{-1} (k x k), FP64
  double Fq[12][2];
  for (int i = 0; i < 4; ++i)
    for (int m = 0; m < cl.k; ++m) {
      D3 v = cl.c[i][m] * cl.r + cl.w[i] * cl.R[m];
      Fq[3 * i + 0][m] = 2.0 * v.x;
      Fq[3 * i + 1][m] = 2.0 * v.y;
      Fq[3 * i + 2][m] = 2.0 * v.z;
    }
  double Mi[2][2];
  if (cl.k == 1) {
    Mi[0][0] = 1.0 / (2.0 * norm2(cl.R[0]));
  } else {
    double m00 = 2.0 * norm2(cl.R[0]), m01 = 2.0 * dot(cl.R[0], cl.R[1]), m11 = 2.0 * norm2(cl.R[1]);
    double det = m00 * m11 - m01 * m01;
    Mi[0][0] = m11 / det;
    Mi[0][1] = Mi[1][0] = -m01 / det;
    Mi[1][1] = m00 / det;
  }
  // HD -= (F Mi) F^T
  T Ft[12][2], Gt[12][2];
  for (int p = 0; p < 12; ++p) {
    if (cl.k == 1) {
      Gt[p][0] = (T)(Fq[p][0] * Mi[0][0]);
      Gt[p][1] = T(0);
      Ft[p][1] = T(0);
    } else {
      Gt[p][0] = (T)(Fq[p][0] * Mi[0][0] + Fq[p][1] * Mi[1][0]);
      Gt[p][1] = (T)(Fq[p][0] * Mi[0][1] + Fq[p][1] * Mi[1][1]);
      Ft[p][1] = (T)Fq[p][1];
    }
    Ft[p][0] = (T)Fq[p][0];
  }
  for (int p = 0; p < 12; ++p)
    for (int q = 0; q < 12; ++q) {
      T s = Gt[p][0] * Ft[q][0];
      if (cl.k == 2) s += Gt[p][1] * Ft[q][1];
      HD[p * 12 + q] -= s;
    }
}

// grad D (12) and hess D (12x12 row-major), both FP64.
IPC_D void sqdist_derivs(const Closest& cl, double* gD, double* HD) {
  sqdist_grad(cl, gD);
  sqdist_hess<double>(cl, HD);
}

// b(d) and derivatives w.r.t. d (App. A.3, Eq. ipc_energy), valid for 0 < d < dhat.
IPC_HD void barrier_d(double d, double dhat, double& b, double& b1, double& b2) {
  double l = log(d / dhat);
  double e = d - dhat;
  b = -e * e * l;
  b1 = -2.0 * e * l - e * e / d;
  b2 = -2.0 * l - 4.0 * e / d + e * e / (d * d);
}

// Skew matrix [u]x applied bookkeeping: S[a][b] such that (u x v)_a = S[a][b] v_b
template <class T>
IPC_HD void skew(V3<T> u, T S[3][3]) {
  S[0][0] = 0;    S[0][1] = -u.z; S[0][2] = u.y;
  S[1][0] = u.z;  S[1][1] = 0;    S[1][2] = -u.x;
  S[2][0] = -u.y; S[2][1] = u.x;  S[2][2] = 0;
}

// Hessian (12x12, T) of the mollifier argument x = |(a1 - a0) x (b1 - b0)|^2.
template <class T>
IPC_D void ee_cross2_hess(const D3* X, T* Hx) {
  const D3 ead = X[1] - X[0], ebd = X[3] - X[2];
  const V3<T> ea{(T)ead.x, (T)ead.y, (T)ead.z}, eb{(T)ebd.x, (T)ebd.y, (T)ebd.z};
  const V3<T> n = cross(ea, eb);
  const T sg[4] = {T(-1), T(1), T(-1), T(1)};
  T Sa[3][3], Sb[3][3], Sn[3][3];
  skew(ea, Sa); skew(eb, Sb); skew(n, Sn);
  T Haa[3][3], Hbb[3][3], Hab[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T sbb = 0, saa = 0, sba = 0;
      for (int k = 0; k < 3; ++k) {
        sbb += Sb[i][k] * Sb[k][j];
        saa += Sa[i][k] * Sa[k][j];
        sba += Sb[i][k] * Sa[k][j];
      }
      Haa[i][j] = T(-2) * sbb;
      Hbb[i][j] = T(-2) * saa;
      Hab[i][j] = T(2) * (-Sn[i][j] + sba);
    }
  for (int P = 0; P < 4; ++P)
    for (int Q = 0; Q < 4; ++Q) {
      T s = sg[P] * sg[Q];
      bool pa = P < 2, qa = Q < 2;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          T v;
          if (pa && qa) v = Haa[i][j];
          else if (!pa && !qa) v = Hbb[i][j];
          else if (pa) v = Hab[i][j];
          else v = Hab[j][i];
          Hx[(3 * P + i) * 12 + 3 * Q + j] = s * v;
        }
    }
}

// Mollifier argument x = |(a1 - a0) x (b1 - b0)|^2 with its gradient (gx,
// when non-null) and Hessian (Hx, when non-null), FP64.
IPC_D double ee_cross2(const D3* X, double* gx, double* Hx) {
  D3 ea = X[1] - X[0], eb = X[3] - X[2];
  D3 n = cross(ea, eb);
  double x = norm2(n);
  if (gx) {
    D3 ga = 2.0 * cross(eb, n);  // d x / d ea
    D3 gb = 2.0 * cross(n, ea);  // d x / d eb
    for (int c = 0; c < 3; ++c) {
      gx[c] = -comp(ga, c); gx[3 + c] = comp(ga, c);
      gx[6 + c] = -comp(gb, c); gx[9 + c] = comp(gb, c);
    }
  }
  if (Hx) ee_cross2_hess<double>(X, Hx);
  return x;
}

// Exact PSD projection of a symmetric 12x12 H whose range lies in the span of
// the closest-feature basis {w (x) e_c (c = 0..2), c_m (x) r (m < k)}: this
// holds for the unmollified barrier, H = bD2 gD gD^T + bD1 hess D, because
// gD = 2 w (x) r and hess D = 2 (w w^T (x) I3) - F Mi F^T with
// F_m = 2 (c_m (x) r + w (x) R_m).  With Q an orthonormal basis of that span
// (dimension <= 5), H = Q (Q^T H Q) Q^T and the clamp acts on the small matrix.
// Gram-Schmidt acceptance threshold on |u|^2 after / before (relative)
template <class T> struct GsTol;
template <> struct GsTol<double> { static constexpr double v = 1e-24; };
template <> struct GsTol<float> { static constexpr float v = 1e-8f; };

template <class T>
static __host__ __device__ __noinline__ void gs_push(T (*Q)[12], int& nq, T* u) {
  T n0 = 0;
  for (int p = 0; p < 12; ++p) n0 += u[p] * u[p];
  if (!(n0 > T(0))) return;
  for (int round = 0; round < 2; ++round)  // two rounds of Gram-Schmidt
    for (int j = 0; j < nq; ++j) {
      T dd = 0;
      for (int p = 0; p < 12; ++p) dd += Q[j][p] * u[p];
      for (int p = 0; p < 12; ++p) u[p] -= dd * Q[j][p];
    }
  T n1 = 0;
  for (int p = 0; p < 12; ++p) n1 += u[p] * u[p];
  if (!(n1 > GsTol<T>::v * n0)) return;
  T inv = T(1) / sqrt(n1);
  for (int p = 0; p < 12; ++p) Q[nq][p] = u[p] * inv;
  ++nq;
}

template <class T>
static __host__ __device__ __noinline__ void psd_project_closest(const Closest& cl, T* H, bool absval) {
  T Q[5][12];
  int nq = 0;
  T u[12];
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 4; ++i)
      for (int a = 0; a < 3; ++a) u[3 * i + a] = (a == c) ? (T)cl.w[i] : T(0);
    gs_push<T>(Q, nq, u);
  }
  const T rx = (T)cl.r.x, ry = (T)cl.r.y, rz = (T)cl.r.z;
  for (int m = 0; m < cl.k; ++m) {
    for (int i = 0; i < 4; ++i) {
      const T cm = (T)cl.c[i][m];
      u[3 * i] = cm * rx;
      u[3 * i + 1] = cm * ry;
      u[3 * i + 2] = cm * rz;
    }
    gs_push<T>(Q, nq, u);
  }
  // M = Q^T H Q (padded to 5x5)
  T HQ[12][5];
  for (int p = 0; p < 12; ++p)
    for (int j = 0; j < 5; ++j) {
      T acc = 0;
      if (j < nq)
        for (int q = 0; q < 12; ++q) acc += H[p * 12 + q] * Q[j][q];
      HQ[p][j] = acc;
    }
  T M[25], V[25];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      T acc = 0;
      if (i < nq && j < nq)
        for (int p = 0; p < 12; ++p) acc += Q[i][p] * HQ[p][j];
      M[5 * i + j] = acc;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = i + 1; j < 5; ++j) {
      T sm = T(0.5) * (M[5 * i + j] + M[5 * j + i]);
      M[5 * i + j] = M[5 * j + i] = sm;
    }
  jacobi_eigen<5, T>(M, V, 20);
  bool neg = false;
  for (int k = 0; k < 5; ++k) neg |= M[6 * k] < T(0);
  if (!neg) return;
  // H = sum_k f(l_k) (Q^T v_k)(Q^T v_k)^T, f(l) = max(l, 0) or |l|
  T Y[5][12];
  for (int k = 0; k < 5; ++k)
    for (int p = 0; p < 12; ++p) {
      T acc = 0;
      for (int i = 0; i < nq; ++i) acc += Q[i][p] * V[5 * i + k];
      Y[k][p] = acc;
    }
  for (int p = 0; p < 12; ++p)
    for (int q = p; q < 12; ++q) {
      T acc = 0;
      for (int k = 0; k < 5; ++k) {
        T l = M[6 * k];
        if (absval) l = fabs(l);
        if (l > T(0)) acc += l * Y[k][p] * Y[k][q];
      }
      H[p * 12 + q] = acc;
      H[q * 12 + p] = acc;
    }
}

// full 12x12 eigen-filter with its own scratch
template <class T>
static __host__ __device__ __noinline__ void psd_project12(T* H, bool absval) {
  T scratch[288];
  psd_project<12, T>(H, scratch, absval);
}

// Weighted barrier of one pair: E = w c(x) b(d).  Returns false when the
// pair is inactive (d >= dhat): E = 0 and g/H untouched.  g (12, FP64) and
// H (144, PSD-projected, arithmetic type T) are written when non-null.  The
// distance, the barrier and mollifier derivatives and the gradient are FP64
// whatever T; with T = float the Hessian is formed and projected in FP32
// from the FP64 per-pair factors (the mixed mode stores it in FP32).
template <class T>
IPC_D bool pair_barrier(const D3* X, bool is_ee, double w, double eps_x, double dhat,
                        double* E, double* g, T* H, int filt = FILT_CLAMP) {
  Closest cl;
  classify(X, is_ee, cl);
  double D = cl.D;
  double d = sqrt(D);
  if (!(d < dhat)) { *E = 0.0; return false; }
  double b, b1, b2;
  barrier_d(d, dhat, b, b1, b2);
  double bD1 = b1 / (2.0 * d);                   // db/dD
  double bD2 = (b2 - b1 / d) / (4.0 * D);        // d2b/dD2
  double c = 1.0, c1 = 0.0, c2 = 0.0;
  double xm = 0.0;
  bool moll = false;
  if (is_ee) {
    xm = ee_cross2(X, nullptr, nullptr);
    if (xm < eps_x) {
      moll = true;
      c = (-xm / eps_x + 2.0) * xm / eps_x;
      c1 = -2.0 * xm / (eps_x * eps_x) + 2.0 / eps_x;
      c2 = -2.0 / (eps_x * eps_x);
    }
  }
  *E = w * c * b;
  if (!g && !H) return true;
  double gD[12], gx[12];
  sqdist_grad(cl, gD);
  if (moll) ee_cross2(X, gx, nullptr);
  if (g) {
    for (int p = 0; p < 12; ++p) {
      double gb = bD1 * gD[p];
      g[p] = w * (c * gb + (moll ? b * c1 * gx[p] : 0.0));
    }
  }
  if (H) {
    // H = w c (bD2 gD gD^T + bD1 hess D)
    //   + w [bD1 (gD gx^T + gx gD^T) c1 + b (c2 gx gx^T + c1 hess x)]  (mollified)
    // with the per-pair factors folded into FP64 vectors first
    T HD[144];
    sqdist_hess<T>(cl, HD);
    T u[12], v[12];
    const double wc = w * c;
    for (int p = 0; p < 12; ++p) {
      u[p] = (T)gD[p];
      v[p] = (T)(wc * bD2 * gD[p]);
    }
    const T khd = (T)(wc * bD1);
    for (int p = 0; p < 12; ++p)
      for (int q = 0; q < 12; ++q) H[p * 12 + q] = v[p] * u[q] + khd * HD[p * 12 + q];
    if (moll) {
      T* Hx = HD;  // reuse
      ee_cross2_hess<T>(X, Hx);
      T ga[12], gc[12], gh[12], gxt[12];
      for (int p = 0; p < 12; ++p) {
        ga[p] = (T)(w * bD1 * gD[p]);
        gc[p] = (T)(c1 * gx[p]);
        gh[p] = (T)(w * b * c2 * gx[p]);
        gxt[p] = (T)gx[p];
      }
      const T khx = (T)(w * b * c1);
      for (int p = 0; p < 12; ++p)
        for (int q = 0; q < 12; ++q)
          H[p * 12 + q] += ga[p] * gc[q] + gc[p] * ga[q] + gh[p] * gxt[q] + khx * Hx[p * 12 + q];
    }
    // symmetrise then project: low-rank exact projection unless mollified
    for (int p = 0; p < 12; ++p)
      for (int q = p + 1; q < 12; ++q) {
        T s = T(0.5) * (H[p * 12 + q] + H[q * 12 + p]);
        H[p * 12 + q] = s;
        H[q * 12 + p] = s;
      }
    if (filt == FILT_NONE) return true;
    if (moll) psd_project12<T>(H, filt == FILT_ABS);
    else psd_project_closest<T>(cl, H, filt == FILT_ABS);
  }
  return true;
}

// =====================================================================
// additive CCD
// =====================================================================
// t_cap (optional) points at a shared running minimum of the TOIs of other
// pairs; the advancement stops early once t reaches it.  t only grows, so a
// pair stopped there cannot lower that minimum, and the minimum over all
// pairs is the same as with every pair advanced to its own end.
// *unfinished (optional) is set when the run stopped at max_iter only.
IPC_D double accd_toi(const D3* X0, const D3* P, bool is_ee, double s, double t_max, int max_iter,
                      int* iters = nullptr, const double* t_cap = nullptr, bool* unfinished = nullptr) {
  D3 pm = 0.25 * (P[0] + P[1] + P[2] + P[3]);
  double nq[4];
  for (int i = 0; i < 4; ++i) nq[i] = sqrt(norm2(P[i] - pm));
  double lp = is_ee ? fmax(nq[0], nq[1]) + fmax(nq[2], nq[3])
                    : nq[0] + fmax(nq[1], fmax(nq[2], nq[3]));
  if (iters) *iters = 0;
  if (unfinished) *unfinished = false;
  if (lp == 0.0) return t_max;
  double d0 = sqrt(pair_sqdist(X0, is_ee));
  double gap = s * d0;
  double t = 0.0;
  double tl = (1.0 - s) * d0 / lp;
  D3 X[4];
  for (int it = 0; it < max_iter; ++it) {
    if (iters) *iters = it + 1;
    double tt = t + tl;
    for (int i = 0; i < 4; ++i) X[i] = X0[i] + tt * P[i];
    double d = sqrt(pair_sqdist(X, is_ee));
    if (t > 0.0 && d < gap) return t;
    t = tt;
    if (t >= t_max) return t_max;
    tl = 0.9 * d / lp;
    if (t_cap && (it & 7) == 7 && t >= *(const volatile double*)t_cap) return t;
  }
  if (unfinished) *unfinished = true;
  return t;
}

}  // namespace ipc
