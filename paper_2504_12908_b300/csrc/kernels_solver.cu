// Solver kernels: prediction, per-tet elastic (K3) and per-body ABD (K4)
// terms, gather assembly into SELL-32 (K5), block-Jacobi PCG (K6), Newton
// bookkeeping and line-search energies (K8, K9).
//
// Row space: every "row" is 3 DoFs - a gel vertex, or one of the 4 sub-rows
// [p, a0, a1, a2] of an affine body.  Rows of one env form a contiguous range
// padded to a multiple of 128 so that a 128-thread CTA never straddles envs.
#include "common.cuh"
#include "fpconv.cuh"
#include "kernels.h"
#include "pcgvec.cuh"
#include "physics.cuh"

namespace ipc {

#define ENVI(d, e, k) (d).env_i[(e) * NUM_INTS + (k)]
#define ENVS(d, e, k) (d).env_s[(e) * NUM_SCALARS + (k)]

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ bool is_gel(uint8_t k) { return k <= ROW_ATTACHED; }
__device__ __forceinline__ bool is_body(uint8_t k) { return k == ROW_BODY || k == ROW_BODY_DRIVEN; }
__device__ __forceinline__ bool is_driven(uint8_t k) { return k == ROW_ATTACHED || k == ROW_BODY_DRIVEN; }

// ---------------------------------------------------------------------------
// prediction: xn = x, xt = x + h v (body rows: y, ydot), multipliers zero
// ---------------------------------------------------------------------------
__global__ void k_predict(Dev d, int flag) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, flag)) return;
  D3 x = ld3(d.x, r), v = ld3(d.v, r);
  st3(d.xn, r, x);
  st3(d.xt, r, x + d.h * v);
  st3(d.lam, r, D3{0, 0, 0});
}

// targets of attached gel rows: s = p_t + A_t xbar (from the body's target rows)
__global__ void k_attach_targets(Dev d, int flag) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, flag) || d.row_kind[r] != ROW_ATTACHED) return;
  int br = d.body_row[d.row_body[r]];
  D3 xb = ld3(d.row_xbar, r);
  D3 s = ld3(d.s_tgt, br) + xb.x * ld3(d.s_tgt, br + 1) + xb.y * ld3(d.s_tgt, br + 2) + xb.z * ld3(d.s_tgt, br + 3);
  st3(d.s_tgt, r, s);
}

// ---------------------------------------------------------------------------
// K3: per-tet neo-Hookean gradient and projected Hessian blocks
// ---------------------------------------------------------------------------
// HT: precision of the Hessian (computed and stored).  The gradient is FP64
// in both modes: it fixes the converged state.  Positions are differenced in
// FP64 before F is rounded to HT.  (An FP32 gradient was measured: the
// kernel's time did not change and the mixed-vs-FP64 step error grew.)
template <class HT>
__global__ void __launch_bounds__(64) k_tet(Dev d) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = t < d.n_tets;
  int e = ok ? find_env(d.env_tet_off, d.n_envs, t) : 0;
  ok = ok && ENVI(d, e, I_NEWT);
  // mixed mode: each warp stages its 32 tets' 144 Hessian values in shared
  // memory (rows padded to 145 words: conflict-free) and writes the 32 x 144
  // block out contiguously; FP64 mode stores directly
  constexpr bool kStage = sizeof(HT) == 4;
  __shared__ float sH[kStage ? 2 * 32 * 145 : 1];
  const int lane = threadIdx.x & 31;
  float* mine = sH + (kStage ? ((threadIdx.x >> 5) * 32 + lane) * 145 : 0);
  if (ok) {
    const int* q = d.tets + 4 * (long long)t;
    for (int a = 0; a < 4; ++a) ok = ok && IPC_CHECK(d.check_word, (unsigned)q[a] < (unsigned)d.n_rows, CHK_TET_VERT, t);
  }
  if (ok) {
    const int* q = d.tets + 4 * (long long)t;
    D3 X[4];
    for (int a = 0; a < 4; ++a) X[a] = ld3(d.x, q[a]);
    double Dmi[9];
    for (int k = 0; k < 9; ++k) Dmi[k] = d.Dm_inv[9 * (long long)t + k];
    double F[9];
    tet_deformation<double>(X, Dmi, F);
    double vol = d.tet_vol[t], mu = d.env_mu[e], lam = d.env_lam[e];
    double g[12];
    nh_gradient<double>(F, Dmi, vol, mu, lam, g);
    double* G = d.tetG + 12 * (long long)t;
    for (int k = 0; k < 12; ++k) G[k] = g[k];
    HT Fh[9], Dh[9];
    for (int k = 0; k < 9; ++k) { Fh[k] = (HT)F[k]; Dh[k] = (HT)Dmi[k]; }
    const int filt = newton_filter(d, e);
    if (kStage) {
      nh_hessian_blocks<HT>(Fh, Dh, (HT)vol, (HT)mu, (HT)lam,
                            [&](int a, int b, int i, int j, HT v) { mine[(a * 4 + b) * 9 + i * 3 + j] = (float)v; },
                            filt);
    } else {
      HT* H = reinterpret_cast<HT*>(d.tetH) + 144 * (long long)t;
      nh_hessian_blocks<HT>(Fh, Dh, (HT)vol, (HT)mu, (HT)lam,
                            [&](int a, int b, int i, int j, HT v) { H[(a * 4 + b) * 9 + i * 3 + j] = v; }, filt);
    }
  }
  if (kStage) {
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    if (okm == 0u) return;  // no tet of this warp is in a starting env
    __syncwarp();
    const int t0 = t - lane;
    const float* wsh = sH + (threadIdx.x >> 5) * 32 * 145;
    float* H = reinterpret_cast<float*>(d.tetH) + 144 * (long long)t0;
    for (int i = lane; i < 32 * 144; i += 32) {
      const int tt = i / 144;
      if ((okm >> tt) & 1u) H[i] = wsh[tt * 145 + (i - tt * 144)];
    }
  }
}

// ---------------------------------------------------------------------------
// K4: per-body inertia, gravity, orthogonality (Sec. 3.3) and AL terms
//   orthogonality V = kappa_s V_b sum_kl (a_k.a_l - d_kl)^2:
//     dV/da_m = 4 kappa_s V_b sum_l C_ml a_l
//     d2V/da_m da_n = 4 kappa_s V_b [d_mn A A^T + a_n a_m^T + C_mn I]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void body_My_mul(double m, const double* S, const double* v, double* out) {
  for (int c = 0; c < 3; ++c) out[c] = m * v[c];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int l = 0; l < 3; ++l) s += S[3 * k + l] * v[3 + 3 * l + c];
      out[3 + 3 * k + c] = s;
    }
}

// One warp per body (4 bodies per 128-thread CTA): the lanes build the
// gradient entry by entry, lane 0 takes the SVD of the body's 3x3 affine
// part, the lanes form the orthogonality term's nine Hessian eigenpairs in
// closed form and the filtered 9x9 block from them, and write the 12x12
// body Hessian.  No iterative eigen-decomposition runs: on B300 a serial
// FP64 Jacobi sweep set a ~1 ms floor under every Newton iteration.
__global__ void __launch_bounds__(128) k_body(Dev d) {
  __shared__ double sy[4][12], sdy[4][12], sHo[4][81], swork[4][120];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * 4 + w;
  if (b >= d.n_bodies) return;                    // warp-uniform; no block barriers below
  const int e = d.body_env[b];
  if (!ENVI(d, e, I_NEWT)) return;
  const int br = d.body_row[b];
  double* y = sy[w];
  double* dy = sdy[w];
  double* Ho = sHo[w];
  if (lane < 12) {
    y[lane] = d.x[3 * br + lane];
    dy[lane] = y[lane] - d.xt[3 * br + lane];
  }
  __syncwarp();
  const double m = d.body_mass[b];
  const double* S = d.body_S + 9 * b;
  const double h2 = d.h * d.h;
  const double ko = h2 * d.body_kappa[b] * d.body_vol[b];
  const double* a = y + 3;  // a_k = a[3k..3k+3)
  double C[9];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      C[3 * k + l] = a[3 * k] * a[3 * l] + a[3 * k + 1] * a[3 * l + 1] + a[3 * k + 2] * a[3 * l + 2] - (k == l ? 1.0 : 0.0);
  // gradient: lane k < 12 owns entry k (inertia, gravity, orthogonality, AL)
  double gk = 0.0;
  if (lane < 12) {
    if (lane < 3) {
      gk = m * dy[lane] - h2 * m * d.grav[lane];
    } else {
      const int k = (lane - 3) / 3, c = (lane - 3) % 3;
      for (int l = 0; l < 3; ++l) gk += S[3 * k + l] * dy[3 + 3 * l + c];
      double s2 = 0;
      for (int l = 0; l < 3; ++l) s2 += C[3 * k + l] * a[3 * l + c];
      gk += 4.0 * ko * s2;
    }
  }
  const bool driven = d.body_driven[b] != 0;
  if (driven && lane < 12) {
    // M^y (y - s) and M^y lambda, entry `lane`
    auto my = [&](const double* v) {
      if (lane < 3) return m * v[lane];
      const int k = (lane - 3) / 3, c = (lane - 3) % 3;
      double t = 0;
      for (int l = 0; l < 3; ++l) t += S[3 * k + l] * v[3 + 3 * l + c];
      return t;
    };
    double rr[12], lm[12];
    for (int k = 0; k < 12; ++k) {
      rr[k] = y[k] - d.s_tgt[3 * br + k];
      lm[k] = d.lam[3 * br + k];
    }
    gk += d.al_kappa * my(rr) - my(lm);
  }
  if (lane < 12) d.body_g[12 * b + lane] = gk;
  __syncwarp();
  // a positive definite Hessian is its own projection (the common case near
  // rigid states); the eigen-decomposition only runs otherwise
  // Projected orthogonality Hessian from its analytic eigensystem.  The
  // term is ko Psi(A), Psi = |A A^T - I|_F^2 = sum_i (s_i^2 - 1)^2 over the
  // singular values of A (rows a_k), an isotropic function of A, so with
  // A = U diag(s) V^T the Hessian d2Psi/dA2 has the nine eigenpairs
  //   U e_i e_i^T V^T                       12 s_i^2 - 4          (scaling)
  //   U (e_i e_j^T -/+ e_j e_i^T) V^T / r2   4 (s_i^2 -/+ s_i s_j + s_j^2 - 1)
  // (second derivative of Psi along each direction; the directions are
  // orthonormal and the mixed second derivatives vanish).  The filter acts
  // on these eigenvalues directly: no iterative eigen-decomposition.
  double* U = swork[w];        // [9] row-major, columns u_k
  double* V = swork[w] + 9;    // [9]
  double* sv = swork[w] + 18;  // [3]
  double* G = swork[w] + 24;   // [9 modes][9]
  double* L = swork[w] + 105;  // [9] filtered eigenvalues
  if (lane == 0) svd3<double>(a, U, sv, V);
  __syncwarp();
  if (lane < 9) {
    const bool absval = newton_filter(d, e) == FILT_ABS;
    int i, j;
    double sg, lam;
    if (lane < 3) {
      i = j = lane;
      sg = 0.0;
      lam = 12.0 * sv[i] * sv[i] - 4.0;
    } else {
      const int pr = (lane - 3) >> 1;            // (0,1) (0,2) (1,2)
      i = pr == 2 ? 1 : 0;
      j = pr == 0 ? 1 : 2;
      sg = (lane & 1) ? -1.0 : 1.0;              // lane 3, 5, 7: twist (-); 4, 6, 8: flip (+)
      lam = 4.0 * (sv[i] * sv[i] + sg * sv[i] * sv[j] + sv[j] * sv[j] - 1.0);
    }
    const double nrm = lane < 3 ? 1.0 : 0.70710678118654752440;
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) {
        // (U E V^T)_kc, E = e_i e_j^T + sg e_j e_i^T (E = e_i e_i^T for scaling)
        double g = U[3 * k + i] * V[3 * c + j];
        if (lane >= 3) g += sg * U[3 * k + j] * V[3 * c + i];
        G[9 * lane + 3 * k + c] = nrm * g;
      }
    L[lane] = absval ? fabs(lam) : fmax(lam, 0.0);
  }
  __syncwarp();
  for (int idx = lane; idx < 81; idx += 32) {
    const int row = idx / 9, col = idx - 9 * row;
    double v = 0.0;
    for (int m = 0; m < 9; ++m) v += L[m] * G[9 * m + row] * G[9 * m + col];
    Ho[idx] = ko * v;
  }
  __syncwarp();
  double* H = d.body_H + 144 * (long long)b;
  for (int idx = lane; idx < 144; idx += 32) {
    const int row = idx / 12, col = idx - 12 * row;
    double v = 0.0;
    if (row < 3 && col < 3) {
      v = row == col ? m * (1.0 + (driven ? d.al_kappa : 0.0)) : 0.0;
    } else if (row >= 3 && col >= 3) {
      const int k = (row - 3) / 3, c = (row - 3) % 3, l = (col - 3) / 3, c2 = (col - 3) % 3;
      if (c == c2) v = S[3 * k + l] * (1.0 + (driven ? d.al_kappa : 0.0));
      v += Ho[(row - 3) * 9 + (col - 3)];
    }
    H[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// K5: gather assembly, one warp per 32-row chunk.  Value layout: block
// (chunk, slot, lane) component c at (chunk_ptr + slot*32)*9 + c*32 + lane.
// ---------------------------------------------------------------------------
template <class HT>
__global__ void k_assemble(Dev d) {
  int ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (ch >= d.n_chunks) return;
  int r = ch * 32 + lane;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_NEWT)) return;
  uint8_t kr = d.row_kind[r];
  int slots = d.chunk_slots[ch];
  long long base = d.chunk_ptr[ch];
  double h2 = d.h * d.h;
  for (int sl = 0; sl < slots; ++sl) {
    long long blk = base + (long long)sl * 32 + lane;
    int col = d.sell_col[blk];
    HT v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (is_gel(kr)) {
      // slot 0 is the diagonal block; a later slot with col == r is padding
      bool diag = (sl == 0);
      bool live = diag || col != r;
      if (live && (kr == ROW_PINNED || d.row_kind[col] == ROW_PINNED)) {
        if (diag) v[0] = v[4] = v[8] = 1.0;
      } else if (live) {
        const HT* tH = reinterpret_cast<const HT*>(d.tetH);
        for (int k = d.asm_ptr[blk]; k < d.asm_ptr[blk + 1]; ++k) {
          if (!IPC_CHECK(d.check_word, (unsigned)d.asm_src[k] < 16u * (unsigned)d.n_tets, CHK_ASM_SRC, k)) continue;
          const HT* src = tH + 9 * (long long)d.asm_src[k];
          for (int c = 0; c < 9; ++c) v[c] += src[c];
        }
        for (int c = 0; c < 9; ++c) v[c] *= (HT)h2;
        if (diag) {
          double m = d.row_mass[r];
          HT dm = (HT)(m + (kr == ROW_ATTACHED ? d.al_kappa * m : 0.0));
          v[0] += dm; v[4] += dm; v[8] += dm;
        }
      }
    } else if (is_body(kr) && sl < 4) {
      int b = d.row_body[r];
      int kk = r - d.body_row[b];
      const double* H = d.body_H + 144 * (long long)b;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[3 * i + j] = (HT)H[(3 * kk + i) * 12 + 3 * sl + j];
    }
    HT* out = reinterpret_cast<HT*>(d.sell_val) + (base + (long long)sl * 32) * 9 + lane;
    for (int c = 0; c < 9; ++c) out[c * 32] = v[c];
  }
}

// gradient per row: h^2 elastic + inertia + gravity + AL + contact (in qc);
// also starts PCG: r = -g (the right-hand side), qc cleared
__global__ void k_grad(Dev d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_NEWT)) return;
  uint8_t kr = d.row_kind[r];
  D3 g{0, 0, 0};
  if (kr == ROW_FREE || kr == ROW_ATTACHED) {
    double h2 = d.h * d.h;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = d.vt_ptr[r]; k < d.vt_ptr[r + 1]; ++k) {
      int src = d.vt_src[k];
      const double* G = d.tetG + 12 * (long long)(src >> 2) + 3 * (src & 3);
      s0 += G[0]; s1 += G[1]; s2 += G[2];
    }
    double m = d.row_mass[r];
    D3 x = ld3(d.x, r), xt = ld3(d.xt, r);
    g = h2 * D3{s0, s1, s2} + m * (x - xt) - (h2 * m) * D3{d.grav[0], d.grav[1], d.grav[2]};
    if (kr == ROW_ATTACHED) g = g + (d.al_kappa * m) * (x - ld3(d.s_tgt, r)) - m * ld3(d.lam, r);
    g = g + ld3(d.qc, r);
  } else if (is_body(kr)) {
    int b = d.row_body[r];
    int kk = r - d.body_row[b];
    g = D3{d.body_g[12 * b + 3 * kk], d.body_g[12 * b + 3 * kk + 1], d.body_g[12 * b + 3 * kk + 2]} + ld3(d.qc, r);
  }
  st3(d.g, r, g);
  st3(d.qc, r, D3{0, 0, 0});
}

// block-Jacobi preconditioner: 3x3 per gel row, 12x12 per body
template <class HT>
__global__ void k_precond_rows(Dev d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_NEWT)) return;
  uint8_t kr = d.row_kind[r];
  double P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (kr == ROW_FREE || kr == ROW_ATTACHED) {
    int ch = r >> 5, lane = r & 31;
    const HT* A = reinterpret_cast<const HT*>(d.sell_val) + d.chunk_ptr[ch] * 9 + lane;  // slot 0 = diagonal
    double M[9];
    for (int c = 0; c < 9; ++c) M[c] = (double)A[c * 32] + d.pc_acc[9 * r + c];
    double det = inv3(M, P);
    if (!(fabs(det) > 0)) { P[0] = P[4] = P[8] = 1.0; P[1] = P[2] = P[3] = P[5] = P[6] = P[7] = 0.0; }
  }
  // symmetric: [xx, xy, xz, yy, yz, zz], off-diagonals averaged
  HT* pc = reinterpret_cast<HT*>(d.pc) + 6 * (long long)r;
  pc[0] = (HT)P[0];
  pc[1] = (HT)(0.5 * (P[1] + P[3]));
  pc[2] = (HT)(0.5 * (P[2] + P[6]));
  pc[3] = (HT)P[4];
  pc[4] = (HT)(0.5 * (P[5] + P[7]));
  pc[5] = (HT)P[8];
  for (int c = 0; c < 9; ++c) d.pc_acc[9 * r + c] = 0.0;
}

// Body blocks of the preconditioner: the inverse of each body's 12x12
// diagonal block (its Hessian plus the contact terms on it), one warp per
// body, 4 bodies per 128-thread CTA.  Gauss-Jordan with partial pivoting on
// [M | I] in shared memory: for each column the lanes find the pivot (the
// first row with the largest magnitude, as a serial scan would), swap and
// scale the pivot row and eliminate the other rows, each lane owning entries
// of the 12 x 24 array; every entry sees the same operations in the same
// order as in the one-thread elimination.  A singular block gets the
// identity.
__global__ void __launch_bounds__(128) k_precond_body(Dev d) {
  __shared__ double sM[4][12][25];   // rows padded to 25 words
  __shared__ int s_bad[4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * 4 + w;
  if (b >= d.n_bodies) return;                    // warp-uniform; no block barriers below
  const int e = d.body_env[b];
  if (!ENVI(d, e, I_NEWT)) return;
  double (*M)[25] = sM[w];
  for (int i = lane; i < 144; i += 32) {
    const int r = i / 12, c = i - 12 * r;
    M[r][c] = d.body_H[144 * b + i] + d.body_pc_acc[144 * b + i];
    M[r][12 + c] = (r == c) ? 1.0 : 0.0;
    d.body_pc_acc[144 * b + i] = 0.0;
  }
  if (lane == 0) s_bad[w] = 0;
  __syncwarp();
  for (int c = 0; c < 12; ++c) {
    // pivot: largest |M[r][c]| for r >= c, the first one on ties
    double best = lane >= c && lane < 12 ? fabs(M[lane][c]) : -1.0;
    int piv = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int op = __shfl_down_sync(0xffffffffu, piv, o);
      if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    piv = __shfl_sync(0xffffffffu, piv, 0);
    if (!(best > 0.0)) {                           // singular (or NaN): identity below
      if (lane == 0) s_bad[w] = 1;
      break;
    }
    if (piv != c && lane < 24) {
      const double t = M[c][lane];
      M[c][lane] = M[piv][lane];
      M[piv][lane] = t;
    }
    __syncwarp();
    const double inv = 1.0 / M[c][c];
    __syncwarp();
    if (lane < 24) M[c][lane] *= inv;
    __syncwarp();
    // factors of the other rows, read before any row changes
    double f[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) f[r] = M[r][c];
    __syncwarp();
    if (lane < 24) {
      const double pc = M[c][lane];
#pragma unroll
      for (int r = 0; r < 12; ++r)
        if (r != c && f[r] != 0.0) M[r][lane] -= f[r] * pc;
    }
    __syncwarp();
  }
  __syncwarp();
  const bool bad = s_bad[w] != 0;
  for (int i = lane; i < 144; i += 32) {
    const int r = i / 12, c = i - 12 * r;
    d.body_pc[144 * b + i] = bad ? ((r == c) ? 1.0 : 0.0) : M[r][12 + c];
  }
}

// ---------------------------------------------------------------------------
// Newton bookkeeping
// ---------------------------------------------------------------------------
// |p|_inf over gel rows -> S_PNORM; AL residual of attached rows -> S_CRES
__global__ void k_newton_rows(Dev d) {
  __shared__ double sh[32];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_DEC)) return;
  uint8_t kr = d.row_kind[r];
  double pn = 0, cr = 0;
  if (is_gel(kr)) {
    D3 p = ld3(d.p, r);
    pn = fmax(fabs(p.x), fmax(fabs(p.y), fabs(p.z)));
    if (kr == ROW_ATTACHED) {
      D3 c = ld3(d.x, r) - ld3(d.s_tgt, r);
      cr = fmax(fabs(c.x), fmax(fabs(c.y), fabs(c.z)));
    }
  }
  pn = block_max(pn, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(&ENVS(d, e, S_PNORM), pn);
  cr = block_max(cr, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(&ENVS(d, e, S_CRES), cr);
}

// per env: converged / AL multiplier update / line search
__global__ void k_newton_decide(Dev d) {
  const int* has_driven = d.env_has_driven;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs || !ENVI(d, e, I_DEC) || !ENVI(d, e, I_ACTIVE)) return;
  ENVI(d, e, I_LS) = 0;
  ENVI(d, e, I_PAIRTOT) += min(ENVI(d, e, I_NPAIRS), d.env_pair_cap[e]);  // this iteration's static list
  // the solve's contact mat-vec work: its active pairs are fixed over the solve
  ENVS(d, e, S_APCG) += (double)ENVI(d, e, I_PCGIT) * min(ENVI(d, e, I_NACT), d.env_pair_cap[e]);
  double res = ENVS(d, e, S_PNORM) / d.h;
  if (res <= d.newton_tol) {
    if (!has_driven[e] || ENVS(d, e, S_CRES) / d.h <= d.newton_tol) {
      ENVI(d, e, I_MODE) = 1;
      ENVI(d, e, I_ACTIVE) = 0;
    } else if (ENVI(d, e, I_AL) >= d.al_max) {
      ENVI(d, e, I_MODE) = 1;
      ENVI(d, e, I_ACTIVE) = 0;
      ENVI(d, e, I_STATUS) = IPC_ENOTCONV;
    } else {
      ENVI(d, e, I_MODE) = 2;
      ENVI(d, e, I_AL) += 1;
    }
  } else {
    ENVI(d, e, I_MODE) = 0;
    ENVI(d, e, I_LS) = 1;
    ENVI(d, e, I_LSIT) = 0;
    ENVS(d, e, S_ACCD) = 1.0;
  }
}

__global__ void k_al_update(Dev d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_DEC) || !ENVI(d, e, I_ACTIVE) || ENVI(d, e, I_MODE) != 2) return;
  if (!is_driven(d.row_kind[r])) return;
  st3(d.lam, r, ld3(d.lam, r) - d.al_kappa * (ld3(d.x, r) - ld3(d.s_tgt, r)));
}

// ---------------------------------------------------------------------------
// line search (K8)
// ---------------------------------------------------------------------------
__global__ void k_ls_init(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs || !ENVI(d, e, I_LS)) return;
  ENVS(d, e, S_ALPHA) = fmin(1.0, ENVS(d, e, S_ACCD));
  ENVI(d, e, I_SWEPTTOT) += min(ENVI(d, e, I_NPAIRS), d.env_pair_cap[e]);
  if (ENVS(d, e, S_ACCD) < 1.0) ENVI(d, e, I_CCDCUT) += 1;
}

__global__ void k_energy_tet(Dev d, int use_alpha) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tets) return;
  int e = find_env(d.env_tet_off, d.n_envs, t);
  if (!ENVI(d, e, I_LS)) return;
  double a = use_alpha ? ENVS(d, e, S_ALPHA) : 0.0;
  const int* q = d.tets + 4 * (long long)t;
  D3 X[4];
  for (int k = 0; k < 4; ++k) X[k] = ld3(d.x, q[k]) + a * ld3(d.p, q[k]);
  double Dmi[9];
  for (int k = 0; k < 9; ++k) Dmi[k] = d.Dm_inv[9 * (long long)t + k];
  double F[9];
  tet_deformation<double>(X, Dmi, F);
  d.tetE[t] = d.h * d.h * nh_energy<double>(F, d.tet_vol[t], d.env_mu[e], d.env_lam[e]);
}

__global__ void k_energy_row(Dev d, int use_alpha) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_LS)) return;
  uint8_t kr = d.row_kind[r];
  double E = 0;
  if (kr == ROW_FREE || kr == ROW_ATTACHED || kr == ROW_PINNED) {
    double a = use_alpha ? ENVS(d, e, S_ALPHA) : 0.0;
    double m = d.row_mass[r];
    D3 x = ld3(d.x, r) + a * ld3(d.p, r);
    D3 dx = x - ld3(d.xt, r);
    E = 0.5 * m * dot(dx, dx) - d.h * d.h * m * (d.grav[0] * x.x + d.grav[1] * x.y + d.grav[2] * x.z);
    if (kr == ROW_ATTACHED) {
      D3 c = x - ld3(d.s_tgt, r);
      E += 0.5 * d.al_kappa * m * dot(c, c) - m * dot(ld3(d.lam, r), c);
    }
  }
  d.row_E[r] = E;
}

__global__ void k_energy_body(Dev d, int use_alpha) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.n_bodies) return;
  int e = d.body_env[b];
  if (!ENVI(d, e, I_LS)) return;
  double a = use_alpha ? ENVS(d, e, S_ALPHA) : 0.0;
  int br = d.body_row[b];
  double y[12], dy[12], t[12];
  for (int k = 0; k < 12; ++k) {
    y[k] = d.x[3 * br + k] + a * d.p[3 * br + k];
    dy[k] = y[k] - d.xt[3 * br + k];
  }
  double m = d.body_mass[b];
  const double* S = d.body_S + 9 * b;
  body_My_mul(m, S, dy, t);
  double E = 0;
  for (int k = 0; k < 12; ++k) E += 0.5 * dy[k] * t[k];
  double h2 = d.h * d.h;
  E -= h2 * m * (d.grav[0] * y[0] + d.grav[1] * y[1] + d.grav[2] * y[2]);
  double orth = 0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double c = y[3 + 3 * k] * y[3 + 3 * l] + y[4 + 3 * k] * y[4 + 3 * l] + y[5 + 3 * k] * y[5 + 3 * l] - (k == l ? 1.0 : 0.0);
      orth += c * c;
    }
  E += h2 * d.body_kappa[b] * d.body_vol[b] * orth;
  if (d.body_driven[b]) {
    double rr[12];
    for (int k = 0; k < 12; ++k) rr[k] = y[k] - d.s_tgt[3 * br + k];
    body_My_mul(m, S, rr, t);
    for (int k = 0; k < 12; ++k) E += 0.5 * d.al_kappa * rr[k] * t[k] - d.lam[3 * br + k] * t[k];
  }
  d.body_E[b] = E;
}

// total per env in a fixed order: tets, rows, bodies, pairs (one CTA per env)
__global__ void k_env_energy(Dev d, int which) {
  __shared__ double sh[32];
  int e = blockIdx.x;
  if (!ENVI(d, e, I_LS)) return;
  double s = 0;
  for (int t = d.env_tet_off[e] + threadIdx.x; t < d.env_tet_off[e + 1]; t += blockDim.x) s += d.tetE[t];
  for (int r = d.env_row_off[e] + threadIdx.x; r < d.env_row_off[e + 1]; r += blockDim.x) s += d.row_E[r];
  for (int b = d.env_body_off[e] + threadIdx.x; b < d.env_body_off[e + 1]; b += blockDim.x) s += d.body_E[b];
  int np = min(ENVI(d, e, I_NPAIRS), d.env_pair_cap[e]);
  for (int k = threadIdx.x; k < np; k += blockDim.x) s += d.pair_E[d.env_pair_off[e] + k];
  if (d.fr_mu > 0.0) {
    int nf = min(ENVI(d, e, I_NFRIC), d.env_pair_cap[e]);
    for (int k = threadIdx.x; k < nf; k += blockDim.x) s += d.fr_E[d.env_pair_off[e] + k];
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (!(s == s)) s = INFINITY;
    ENVS(d, e, which == 0 ? S_E0 : S_E1) = s;
  }
}

__global__ void k_ls_decide(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs || !ENVI(d, e, I_LS)) return;
  ENVI(d, e, I_LSTOT) += 1;
  double E0 = ENVS(d, e, S_E0), E1 = ENVS(d, e, S_E1);
  if (E1 <= E0) {
    ENVI(d, e, I_ACCEPT) = 1;
    ENVI(d, e, I_LS) = 0;
    ENVS(d, e, S_ASUM) += ENVS(d, e, S_ALPHA);
    return;
  }
  ENVS(d, e, S_ALPHA) *= 0.5;
  if (++ENVI(d, e, I_LSIT) >= d.ls_max) {
    ENVI(d, e, I_LS) = 0;
    ENVI(d, e, I_ACTIVE) = 0;
    ENVI(d, e, I_STATUS) = IPC_ENOTCONV;
  }
}

__global__ void k_ls_apply(Dev d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_ACCEPT)) return;
  st3(d.x, r, ld3(d.x, r) + ENVS(d, e, S_ALPHA) * ld3(d.p, r));
}

__global__ void k_clear_accept(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_envs) ENVI(d, e, I_ACCEPT) = 0;
}

// velocities (App. A.2, backward Euler): v = (x - x^n) / h; overflowed envs restored
__global__ void k_finalize_rows(Dev d, int flag) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, flag)) return;
  uint8_t kr = d.row_kind[r];
  if (kr == ROW_PAD) return;
  if (ENVI(d, e, I_STATUS) == IPC_EOVERFLOW) {
    st3(d.x, r, ld3(d.xn, r));
    return;
  }
  if (kr == ROW_PINNED) { st3(d.v, r, D3{0, 0, 0}); return; }
  st3(d.v, r, (1.0 / d.h) * (ld3(d.x, r) - ld3(d.xn, r)));
}

__global__ void k_finalize_envs(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs || !ENVI(d, e, I_SEL)) return;
  if (ENVI(d, e, I_ACTIVE)) {  // Newton cap reached
    ENVI(d, e, I_ACTIVE) = 0;
    if (ENVI(d, e, I_STATUS) == IPC_OK) ENVI(d, e, I_STATUS) = IPC_ENOTCONV;
  }
}

// what: 0 = new step (counters, status), 1 = Newton-iteration start (which
// envs start one, their scalars), 2 / 5 / 6 = pair count of the envs
// starting a Newton iteration / in a line search / selected, 3 = min
// distance, 4 = select every env
__global__ void k_env_reset(Dev d, int what) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (what == 0 && e < 8) d.step_ctl[e] = 0u;  // new step: loop counters
  if (e >= d.n_envs) return;
  if (what == 0) {
    if (!ENVI(d, e, I_SEL)) return;
    ENVI(d, e, I_ACTIVE) = 1;
    ENVI(d, e, I_PCG) = 0;
    ENVI(d, e, I_DEC) = 0;
    ENVI(d, e, I_STATUS) = IPC_OK;
    ENVI(d, e, I_NEWTON) = 0;
    ENVI(d, e, I_AL) = 0;
    ENVI(d, e, I_PCGTOT) = 0;
    ENVI(d, e, I_LSTOT) = 0;
    ENVI(d, e, I_ACCEPT) = 0;
    ENVI(d, e, I_OVERFLOW) = 0;
    ENVI(d, e, I_CCDCUT) = 0;
    ENVI(d, e, I_ACCDIT) = 0;
    ENVI(d, e, I_ACCDMAX) = 0;
    ENVI(d, e, I_NFRIC) = 0;
    ENVI(d, e, I_PAIRTOT) = 0;
    ENVI(d, e, I_SWEPTTOT) = 0;
    ENVS(d, e, S_ASUM) = 0.0;
    ENVS(d, e, S_APCG) = 0.0;
  } else if (what == 1) {
    // an env starts a Newton iteration unless its solve carries over; the
    // decision of its previous iteration is done
    const int newt = ENVI(d, e, I_ACTIVE) && !ENVI(d, e, I_PCG);
    ENVI(d, e, I_NEWT) = newt;
    ENVI(d, e, I_DEC) = 0;
    if (!newt) return;
    ENVS(d, e, S_PNORM) = 0.0;
    ENVS(d, e, S_CRES) = 0.0;
    ENVI(d, e, I_NEWTON) += 1;
    ENVI(d, e, I_GEN) += 1;
    ENVI(d, e, I_NACT) = 0;
  } else if (what == 2) {  // the static list is rebuilt
    if (ENVI(d, e, I_NEWT)) ENVI(d, e, I_NPAIRS) = 0;
  } else if (what == 5) {  // the swept list is rebuilt
    if (ENVI(d, e, I_LS)) ENVI(d, e, I_NPAIRS) = 0;
  } else if (what == 6) {  // a selected env's list is rebuilt (set_state, diagnostics)
    if (ENVI(d, e, I_SEL)) ENVI(d, e, I_NPAIRS) = 0;
  } else if (what == 3) {
    ENVS(d, e, S_MIND) = INFINITY;
    ENVI(d, e, I_FLAG) = 0;
  } else if (what == 4) {
    ENVI(d, e, I_SEL) = 1;
  }
}

// ---------------------------------------------------------------------------
// Rollout: every selected env runs roll_ctl[1] steps inside one device loop,
// each on its own schedule.  One loop iteration is one Newton iteration of
// the envs inside a step; an env whose step ends (converged, failed or at
// the Newton cap) is finalised in that iteration and begins its next step
// in the next one, while the others keep iterating.  Per env the sequence
// of operations is the same as that of ipc_step called once per step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void begin_step_counters(const Dev& d, int e) {
  ENVI(d, e, I_ACTIVE) = 1;
  ENVI(d, e, I_PCG) = 0;
  ENVI(d, e, I_DEC) = 0;
  ENVI(d, e, I_STATUS) = IPC_OK;
  ENVI(d, e, I_NEWTON) = 0;
  ENVI(d, e, I_AL) = 0;
  ENVI(d, e, I_PCGTOT) = 0;
  ENVI(d, e, I_LSTOT) = 0;
  ENVI(d, e, I_ACCEPT) = 0;
  ENVI(d, e, I_OVERFLOW) = 0;
  ENVI(d, e, I_CCDCUT) = 0;
  ENVI(d, e, I_ACCDIT) = 0;
  ENVI(d, e, I_ACCDMAX) = 0;
  ENVI(d, e, I_NFRIC) = 0;
  ENVI(d, e, I_PAIRTOT) = 0;
  ENVI(d, e, I_SWEPTTOT) = 0;
  ENVS(d, e, S_ASUM) = 0.0;
  ENVS(d, e, S_APCG) = 0.0;
}

// the table address, steps and loop cap of the next rollout (1 thread)
__global__ void k_roll_setup(Dev d, const double* table, int n_steps, unsigned long long cap) {
  d.roll_ctl[0] = (unsigned long long)(uintptr_t)table;
  d.roll_ctl[1] = (unsigned long long)n_steps;
  d.roll_ctl[2] = cap;
}

// before the loop: selected envs begin step 0; loop counters zeroed
__global__ void k_roll_init(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 8) d.step_ctl[e] = 0u;
  if (e >= d.n_envs) return;
  const int sel = ENVI(d, e, I_SEL) != 0 && d.roll_ctl[1] > 0 && ENVI(d, e, I_RLIMIT) > 0;
  ENVI(d, e, I_RSTEP) = 0;
  ENVI(d, e, I_BEGIN) = sel;
  ENVI(d, e, I_LIVE) = sel;
  ENVI(d, e, I_RUN) = 0;
  ENVI(d, e, I_ENDNOW) = 0;
  ENVI(d, e, I_ACTIVE) = 0;
  if (sel) ENVI(d, e, I_STATUS) = IPC_OK;
  for (int k = I_RNEWTON; k <= I_RPAIRSMAX; ++k) ENVI(d, e, k) = 0;
  ENVS(d, e, S_RASUM) = 0.0;
  ENVS(d, e, S_RAPCG) = 0.0;
}

// envs that begin a step: their targets for step I_RSTEP from the table
// [steps][n_envs][max_bodies][12], the per-step counters reset (one warp per
// env; lane j copies target entries j, j + 32, ...)
__global__ void k_roll_begin(Dev d) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (e >= d.n_envs || !ENVI(d, e, I_BEGIN)) return;
  const double* table = reinterpret_cast<const double*>((uintptr_t)d.roll_ctl[0]);
  const long long k = ENVI(d, e, I_RSTEP);
  const int b0 = d.env_body_off[e], nb = d.env_body_off[e + 1] - b0;
  const double* src = table + (k * d.n_envs + e) * (long long)d.max_bodies * 12;
  for (int j = lane; j < 12 * nb; j += 32) d.s_tgt[3 * d.body_row[b0 + j / 12] + j % 12] = src[j];
  if (lane == 0) {
    begin_step_counters(d, e);
    ENVI(d, e, I_RUN) = 1;
  }
}

// after the Newton iteration: the Newton cap ends a step as not converged;
// ENDNOW marks the envs whose step ended in this iteration
__global__ void k_roll_end(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  ENVI(d, e, I_BEGIN) = 0;
  int end = 0;
  if (ENVI(d, e, I_RUN)) {
    // the Newton cap applies once the iteration's solve and decision are done
    if (ENVI(d, e, I_ACTIVE) && !ENVI(d, e, I_PCG) && ENVI(d, e, I_NEWTON) >= d.newton_max) {
      ENVI(d, e, I_ACTIVE) = 0;
      if (ENVI(d, e, I_STATUS) == IPC_OK) ENVI(d, e, I_STATUS) = IPC_ENOTCONV;
    }
    end = !ENVI(d, e, I_ACTIVE);
  }
  ENVI(d, e, I_ENDNOW) = end;
}

// envs whose step ended: counters into the rollout sums, next step (unless
// it failed or was the last); LIVE = running or beginning
__global__ void k_roll_advance(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  if (ENVI(d, e, I_ENDNOW)) {
    ENVI(d, e, I_RNEWTON) += ENVI(d, e, I_NEWTON);
    ENVI(d, e, I_RNEWTONMAX) = max(ENVI(d, e, I_RNEWTONMAX), ENVI(d, e, I_NEWTON));
    ENVI(d, e, I_RAL) += ENVI(d, e, I_AL);
    ENVI(d, e, I_RPCG) += ENVI(d, e, I_PCGTOT);
    ENVI(d, e, I_RLS) += ENVI(d, e, I_LSTOT);
    ENVI(d, e, I_RCCDCUT) += ENVI(d, e, I_CCDCUT);
    ENVI(d, e, I_RACCDIT) += ENVI(d, e, I_ACCDIT);
    ENVI(d, e, I_RACCDMAX) = max(ENVI(d, e, I_RACCDMAX), ENVI(d, e, I_ACCDMAX));
    ENVI(d, e, I_RPAIR) += ENVI(d, e, I_PAIRTOT);
    ENVI(d, e, I_RSWEPT) += ENVI(d, e, I_SWEPTTOT);
    ENVI(d, e, I_RPAIRSMAX) = max(ENVI(d, e, I_RPAIRSMAX), ENVI(d, e, I_NPAIRS));
    ENVS(d, e, S_RASUM) += ENVS(d, e, S_ASUM);
    ENVS(d, e, S_RAPCG) += ENVS(d, e, S_APCG);
    const int k = ++ENVI(d, e, I_RSTEP);
    ENVI(d, e, I_RUN) = 0;
    ENVI(d, e, I_ENDNOW) = 0;
    ENVI(d, e, I_BEGIN) = ENVI(d, e, I_STATUS) == IPC_OK && (unsigned long long)k < d.roll_ctl[1] &&
                          k < ENVI(d, e, I_RLIMIT);
  }
  ENVI(d, e, I_LIVE) = ENVI(d, e, I_RUN) || ENVI(d, e, I_BEGIN);
}

// the rollout loop's condition (one CTA): some env live and the loop below
// its cap (roll_ctl[2]); counts the loop iterations in step_ctl[0]
__global__ void k_roll_cond(Dev d, cudaGraphConditionalHandle h) {
  __shared__ int sh[32];
  int c = 0;
  for (int e = threadIdx.x; e < d.n_envs; e += blockDim.x) c += ENVI(d, e, I_LIVE) != 0;
  c = block_sum(c, sh);
  if (threadIdx.x != 0) return;
  d.step_ctl[2] = (unsigned)c;
  const unsigned k = ++d.step_ctl[0];
  cudaGraphSetConditional(h, (c > 0 && (unsigned long long)k < d.roll_ctl[2]) ? 1u : 0u);
}

// Loop control of the device-side step (one CTA): counts the envs whose
// `flag` is set into step_ctl[cnt]; with inc >= 0 also advances the loop
// counter step_ctl[inc] (and step_ctl[acc] when acc >= 0), with rst >= 0
// zeroes step_ctl[rst].  The condition is 1 while some env has the flag and
// (with inc >= 0) the counter is below `cap`; inside a graph it is set on the
// conditional handle h.
__global__ void k_flag_cond(Dev d, int flag, int cnt, int inc, int acc, int rst, unsigned cap,
                            cudaGraphConditionalHandle h, int use_cond) {
  __shared__ int sh[32];
  int c = 0;
  for (int e = threadIdx.x; e < d.n_envs; e += blockDim.x) c += ENVI(d, e, flag) != 0;
  c = block_sum(c, sh);
  if (threadIdx.x != 0) return;
  d.step_ctl[cnt] = (unsigned)c;
  if (rst >= 0) d.step_ctl[rst] = 0u;
  bool more = c > 0;
  if (inc >= 0) {
    const unsigned k = ++d.step_ctl[inc];
    if (acc >= 0) d.step_ctl[acc] += 1u;
    more = more && k < cap;
  }
  if (use_cond) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// pair-list overflow ends the env's step (state restored at finalize)
__global__ void k_check_overflow(Dev d) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_envs) return;
  if (ENVI(d, e, I_OVERFLOW) && ENVI(d, e, I_SEL) && ENVI(d, e, I_STATUS) != IPC_EOVERFLOW) {
    ENVI(d, e, I_STATUS) = IPC_EOVERFLOW;
    ENVI(d, e, I_ACTIVE) = 0;
    ENVI(d, e, I_LS) = 0;
    ENVI(d, e, I_NEWT) = 0;
  }
}

// min det F over tets of I_SEL envs -> S_MIND (as a sign flag: 0 if inverted)
__global__ void k_check_inverted(Dev d) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tets) return;
  int e = find_env(d.env_tet_off, d.n_envs, t);
  if (!ENVI(d, e, I_SEL)) return;
  const int* q = d.tets + 4 * (long long)t;
  D3 X[4];
  for (int k = 0; k < 4; ++k) X[k] = ld3(d.x, q[k]);
  double Dmi[9], F[9];
  for (int k = 0; k < 9; ++k) Dmi[k] = d.Dm_inv[9 * (long long)t + k];
  tet_deformation<double>(X, Dmi, F);
  if (!(det3<double>(F) > 0.0)) ENVI(d, e, I_FLAG) = 1;
}

// staged host targets [env][body][12] -> body target rows
__global__ void k_scatter_targets(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;  // (env, body, row k, component) flattened
  int per_env = d.max_bodies * 12;
  if (i >= d.n_envs * per_env) return;
  int e = i / per_env, j = i % per_env, b = j / 12, k = j % 12;
  int b0 = d.env_body_off[e];
  if (b >= d.env_body_off[e + 1] - b0) return;
  d.s_tgt[3 * d.body_row[b0 + b] + k] = d.tgt_stage[i];
}

// coated-surface rows -> contiguous staging buffer
__global__ void k_gather_coated(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_coated) return;
  st3(d.out_stage, i, ld3(d.x, d.coated_row[i]));
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define ROWGRID (d.n_rows / 128), 128, 0, s
#define ENVGRID nblk(d.n_envs, 128), 128, 0, s
int launch_predict(const Dev& d, int flag, cudaStream_t s) { k_predict<<<ROWGRID>>>(d, flag); return 1; }
int launch_attach_targets(const Dev& d, int flag, cudaStream_t s) { k_attach_targets<<<ROWGRID>>>(d, flag); return 1; }
int launch_tet(const Dev& d, cudaStream_t s) {
  if (d.prec) k_tet<float><<<nblk(d.n_tets, 64), 64, 0, s>>>(d);
  else k_tet<double><<<nblk(d.n_tets, 64), 64, 0, s>>>(d);
  return 1;
}
int launch_body(const Dev& d, cudaStream_t s) {
  if (!d.n_bodies) return 0;
  k_body<<<nblk(d.n_bodies, 4), 128, 0, s>>>(d);
  return 1;
}
int launch_assemble(const Dev& d, cudaStream_t s) {
  const int b = d.asm_block > 0 ? d.asm_block : 128;
  if (d.prec) k_assemble<float><<<nblk(32LL * d.n_chunks, b), b, 0, s>>>(d);
  else k_assemble<double><<<nblk(32LL * d.n_chunks, b), b, 0, s>>>(d);
  return 1;
}
int launch_grad(const Dev& d, cudaStream_t s) { k_grad<<<ROWGRID>>>(d); return 1; }
int launch_precond(const Dev& d, cudaStream_t s) {
  if (d.prec) k_precond_rows<float><<<ROWGRID>>>(d);
  else k_precond_rows<double><<<ROWGRID>>>(d);
  if (!d.n_bodies) return 1;
  k_precond_body<<<nblk(d.n_bodies, 4), 128, 0, s>>>(d);
  return 2;
}
int launch_newton_check(const Dev& d, cudaStream_t s) {
  k_newton_rows<<<ROWGRID>>>(d);
  return 1 + launch_pnorm_body(d, s);
}
int launch_newton_decide(const Dev& d, cudaStream_t s) { k_newton_decide<<<ENVGRID>>>(d); return 1; }
int launch_al_update(const Dev& d, cudaStream_t s) { k_al_update<<<ROWGRID>>>(d); return 1; }
int launch_ls_init(const Dev& d, cudaStream_t s) { k_ls_init<<<ENVGRID>>>(d); return 1; }
int launch_energy(const Dev& d, int use_alpha, int which, cudaStream_t s) {
  int n = 3;
  k_energy_tet<<<nblk(d.n_tets, 128), 128, 0, s>>>(d, use_alpha);
  k_energy_row<<<ROWGRID>>>(d, use_alpha);
  if (d.n_bodies) { k_energy_body<<<nblk(d.n_bodies, 32), 32, 0, s>>>(d, use_alpha); ++n; }
  n += launch_pair_energy(d, use_alpha, s);
  n += launch_fric_energy(d, use_alpha, s);
  k_env_energy<<<d.n_envs, 256, 0, s>>>(d, which);
  return n;
}
int launch_ls_decide(const Dev& d, cudaStream_t s) { k_ls_decide<<<ENVGRID>>>(d); return 1; }
int launch_ls_apply(const Dev& d, cudaStream_t s) {
  k_ls_apply<<<ROWGRID>>>(d);
  k_clear_accept<<<ENVGRID>>>(d);
  return 2;
}
int launch_finalize(const Dev& d, cudaStream_t s) {
  k_finalize_envs<<<ENVGRID>>>(d);
  k_finalize_rows<<<ROWGRID>>>(d, I_SEL);
  return 2;
}
int launch_roll_setup(const Dev& d, const double* table, int n_steps, unsigned long long cap, cudaStream_t s) {
  k_roll_setup<<<1, 1, 0, s>>>(d, table, n_steps, cap);
  return 1;
}
int launch_roll_init(const Dev& d, cudaStream_t s) { k_roll_init<<<ENVGRID>>>(d); return 1; }
int launch_roll_begin(const Dev& d, cudaStream_t s) {
  k_roll_begin<<<nblk(32LL * d.n_envs, 128), 128, 0, s>>>(d);
  k_predict<<<ROWGRID>>>(d, I_BEGIN);
  k_attach_targets<<<ROWGRID>>>(d, I_BEGIN);
  return 3;
}
int launch_roll_end(const Dev& d, cudaStream_t s) {
  k_roll_end<<<ENVGRID>>>(d);
  k_finalize_rows<<<ROWGRID>>>(d, I_ENDNOW);
  k_roll_advance<<<ENVGRID>>>(d);
  return 3;
}
int launch_roll_cond(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h) {
  k_roll_cond<<<1, 1024, 0, s>>>(d, h);
  return 1;
}
int launch_env_reset(const Dev& d, int what, cudaStream_t s) { k_env_reset<<<ENVGRID>>>(d, what); return 1; }
int launch_check_overflow(const Dev& d, cudaStream_t s) { k_check_overflow<<<ENVGRID>>>(d); return 1; }
int launch_flag_cond(const Dev& d, cudaStream_t s, int flag, int cnt, int inc, int acc, int rst, unsigned cap,
                     cudaGraphConditionalHandle h, int use_cond) {
  k_flag_cond<<<1, 256, 0, s>>>(d, flag, cnt, inc, acc, rst, cap, h, use_cond);
  return 1;
}
int launch_scatter_targets(const Dev& d, cudaStream_t s) {
  long long n = (long long)d.n_envs * d.max_bodies * 12;
  if (n == 0) return 0;
  k_scatter_targets<<<nblk(n, 256), 256, 0, s>>>(d);
  return 1;
}
int launch_gather_coated(const Dev& d, cudaStream_t s) {
  if (!d.n_coated) return 0;
  k_gather_coated<<<nblk(d.n_coated, 256), 256, 0, s>>>(d);
  return 1;
}
int launch_check_inverted(const Dev& d, cudaStream_t s) { k_check_inverted<<<nblk(d.n_tets, 128), 128, 0, s>>>(d); return 1; }

// ---------------------------------------------------------------------------
// element kernel on caller buffers
// ---------------------------------------------------------------------------
__global__ void k_elem_tet(int n, const double* x, const double* Dmi_all, const double* vol, double mu, double lam,
                           double* E, double* g, double* H, int project) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  D3 X[4];
  for (int a = 0; a < 4; ++a) X[a] = ld3(x + 12 * (long long)t, a);
  double Dmi[9], F[9];
  for (int k = 0; k < 9; ++k) Dmi[k] = Dmi_all[9 * (long long)t + k];
  tet_deformation<double>(X, Dmi, F);
  double e = nh_energy<double>(F, vol[t], mu, lam);
  if (E) E[t] = e;
  bool ok = det3<double>(F) > 0.0;
  if (g) {
    double gl[12];
    if (ok) nh_gradient<double>(F, Dmi, vol[t], mu, lam, gl);
    for (int k = 0; k < 12; ++k) g[12 * (long long)t + k] = ok ? gl[k] : NAN;
  }
  if (H) {
    double* Ht = H + 144 * (long long)t;
    if (!ok) {
      for (int k = 0; k < 144; ++k) Ht[k] = NAN;
    } else {
      nh_hessian_blocks<double>(
          F, Dmi, vol[t], mu, lam, [&](int a, int b, int i, int j, double v) { Ht[(3 * a + i) * 12 + 3 * b + j] = v; },
          project);
    }
  }
}

int launch_k_tet(int n, const double* x, const double* Dmi, const double* vol, double mu, double lam,
                 double* E, double* g, double* H, int project, cudaStream_t s) {
  if (n <= 0) return 0;
  k_elem_tet<<<nblk(n, 64), 64, 0, s>>>(n, x, Dmi, vol, mu, lam, E, g, H, project);
  return 1;
}

}  // namespace ipc
