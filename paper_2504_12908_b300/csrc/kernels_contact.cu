// Contact kernels: contact-vertex positions, object boxes, broad phase,
// barrier energy/gradient/Hessian (K1, K2), matrix-free contact mat-vec,
// additive CCD (K7) and pair energies for the line search.
#include "common.cuh"
#include "kernels.h"
#include "pcgvec.cuh"
#include "physics.cuh"

namespace ipc {

#define ENVI(d, e, k) (d).env_i[(e) * NUM_INTS + (k)]
#define ENVS(d, e, k) (d).env_s[(e) * NUM_SCALARS + (k)]

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// contact vertex positions: gel vertex -> x[row]; body vertex j -> p + A xbar_j
// (phi(y), Sec. 3.3).  With `with_disp` also the displacement along p.
// ---------------------------------------------------------------------------
__device__ __forceinline__ D3 body_point(const double* x, int br, D3 xb) {
  return ld3(x, br) + xb.x * ld3(x, br + 1) + xb.y * ld3(x, br + 2) + xb.z * ld3(x, br + 3);
}

__global__ void k_cv_pos(Dev d, int flag, int with_disp) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n_cv) return;
  int e = find_env(d.env_cv_off, d.n_envs, c);
  if (!ENVI(d, e, flag)) return;
  int row = d.cv_row[c];
  if (d.cv_body[c] < 0) {
    st3(d.cvx, c, ld3(d.x, row));
    if (with_disp) st3(d.cvp, c, ld3(d.p, row));
  } else {
    D3 xb = ld3(d.cv_xbar, c);
    st3(d.cvx, c, body_point(d.x, row, xb));
    if (with_disp) st3(d.cvp, c, body_point(d.p, row, xb));
  }
}

// Boxes of every contact primitive (swept: over both ends of the step).
// idx in [0, n_cv + n_tri + n_edge): points, then triangles, then edges.
__device__ __forceinline__ void grow(double* bx, D3 a) {
  bx[0] = fmin(bx[0], a.x); bx[1] = fmin(bx[1], a.y); bx[2] = fmin(bx[2], a.z);
  bx[3] = fmax(bx[3], a.x); bx[4] = fmax(bx[4], a.y); bx[5] = fmax(bx[5], a.z);
}

__global__ void k_prim_boxes(Dev d, int flag, int swept) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int n = d.n_cv + d.n_tri + d.n_edge;
  if (i >= n) return;
  int kind, j, e;
  if (i < d.n_cv) { kind = 0; j = i; e = find_env(d.env_cv_off, d.n_envs, j); }
  else if (i < d.n_cv + d.n_tri) { kind = 1; j = i - d.n_cv; e = find_env(d.env_tri_off, d.n_envs, j); }
  else { kind = 2; j = i - d.n_cv - d.n_tri; e = find_env(d.env_edge_off, d.n_envs, j); }
  if (!ENVI(d, e, flag)) return;
  int v[3], nv;
  if (kind == 0) { v[0] = j; nv = 1; }
  else if (kind == 1) { v[0] = d.tri[3 * j]; v[1] = d.tri[3 * j + 1]; v[2] = d.tri[3 * j + 2]; nv = 3; }
  else { v[0] = d.edge[2 * j]; v[1] = d.edge[2 * j + 1]; nv = 2; }
  double bx[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < nv; ++k) {
    D3 a = ld3(d.cvx, v[k]);
    grow(bx, a);
    if (swept) grow(bx, a + ld3(d.cvp, v[k]));
  }
  double* out = (kind == 0 ? d.cv_box : (kind == 1 ? d.tri_box : d.edge_box)) + 6 * (long long)j;
  for (int k = 0; k < 6; ++k) out[k] = bx[k];
}

// one CTA per object: box of its contact-vertex boxes
__global__ void k_obj_box(Dev d, int flag) {
  int o = blockIdx.x;
  int e = d.obj_env[o];
  if (!ENVI(d, e, flag)) return;
  __shared__ double sh[32];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int c = d.obj_cv_begin[o] + threadIdx.x; c < d.obj_cv_end[o]; c += blockDim.x) {
    const double* b = d.cv_box + 6 * (long long)c;
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], b[k]); hi[k] = fmax(hi[k], b[3 + k]); }
  }
  for (int k = 0; k < 3; ++k) {
    double m = -block_max(-lo[k], sh);
    if (threadIdx.x == 0) d.obj_box[6 * o + k] = m;
    double M = block_max(hi[k], sh);
    if (threadIdx.x == 0) d.obj_box[6 * o + 3 + k] = M;
  }
}

// widened overlap: lo_a <= hi_b + dhat and lo_b <= hi_a + dhat on every axis
__device__ __forceinline__ bool overlap6(const double* a, const double* b, double dh) {
  for (int k = 0; k < 3; ++k)
    if (!(a[k] <= b[3 + k] + dh) || !(b[k] <= a[3 + k] + dh)) return false;
  return true;
}

__device__ __forceinline__ bool bigger(const Dev& d, int A, int B) {
  int sa = d.obj_size[A], sb = d.obj_size[B];
  return sa > sb || (sa == sb && A < B);
}

__device__ void emit_pair(const Dev& d, int e, int4 v, int kind, double w, double eps) {
  int slot = atomicAdd(&ENVI(d, e, I_NPAIRS), 1);
  if (slot >= d.env_pair_cap[e]) {
    ENVI(d, e, I_OVERFLOW) = 1;
    return;
  }
  long long k = d.env_pair_off[e] + slot;
  d.pair_v[k] = v;
  d.pair_kind[k] = kind;
  d.pair_w[k] = w;
  d.pair_eps[k] = eps;
}

// Broad phase, stage 1: worklist of (query primitive, other object) items.
// Each unordered object pair {A, B} is handled from the bigger object's
// primitives, kept only when the primitive's box meets B's widened box:
//   QK = 0: points of A vs triangles of B   -> PT(point A, tri B)
//   QK = 1: triangles of A vs points of B   -> PT(point B, tri A)
//   QK = 2: edges of A vs edges of B        -> EE(lower object first)
// A self-contacting pad (its own exclusion bit clear) also gets the item
// (q, A) for its points and edges: QK = 0 covers its own PT pairs and
// QK = 2 its own EE pairs; QK = 1 would repeat the PT pairs.
// Items of one warp are written contiguously (one atomic per warp).
template <int QK>
__global__ void k_worklist(Dev d, int flag) {
  int n_q = QK == 0 ? d.n_cv : (QK == 1 ? d.n_tri : d.n_edge);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31;
  int cnt = 0, e = 0, A = 0;
  bool live = false;
  const double* qb = nullptr;
  unsigned long long ex = 0;
  if (i < n_q) {
    const int* qoff = QK == 0 ? d.env_cv_off : (QK == 1 ? d.env_tri_off : d.env_edge_off);
    e = find_env(qoff, d.n_envs, i);
    live = ENVI(d, e, flag) != 0;
    if (live) {
      A = QK == 0 ? d.cv_obj[i] : (QK == 1 ? d.tri_obj[i] : d.edge_obj[i]);
      qb = (QK == 0 ? d.cv_box : (QK == 1 ? d.tri_box : d.edge_box)) + 6 * (long long)i;
      ex = d.obj_exclude[A];
    }
  }
  // pass 1: count the objects this query meets; pass 2 (after the warp scan)
  // writes them, re-evaluating the same test
  auto keep = [&](int B) {
    if ((ex >> d.obj_local[B]) & 1ull) return false;
    if (B == A ? QK == 1 : !bigger(d, A, B)) return false;
    return overlap6(qb, d.obj_box + 6 * B, d.dhat);
  };
  if (live)
    for (int B = d.env_obj_off[e]; B < d.env_obj_off[e + 1]; ++B) cnt += keep(B) ? 1 : 0;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(d.bp_count, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  int pos = base + incl - cnt;
  if (live && cnt)
    for (int B = d.env_obj_off[e]; B < d.env_obj_off[e + 1]; ++B) {
      if (!keep(B)) continue;
      if (pos < d.bp_cap) d.bp_items[pos] = make_int4(QK, i, B, e);
      else *d.bp_overflow = 1;
      ++pos;
    }
}

// Broad-phase hierarchy refit.  Per object and primitive kind the
// primitives are kept in Morton order of their rest centroids; a cluster is
// 32 consecutive primitives of that order and a supercluster 32 consecutive
// clusters.  Their boxes are the unions of the current primitive boxes (the
// order is fixed at creation: the meshes deform but keep their topology, so
// clusters stay compact).  A union contains each of its boxes, so a box that
// meets the query meets every enclosing cluster and supercluster: pruning
// by them never drops a candidate.
__device__ __forceinline__ void prim_range(const Dev& d, int k, int o, int& b, int& e) {
  if (k == 0) { b = d.obj_cv_begin[o]; e = d.obj_cv_end[o]; }
  else if (k == 1) { b = d.obj_tri_begin[o]; e = d.obj_tri_end[o]; }
  else { b = d.obj_edge_begin[o]; e = d.obj_edge_end[o]; }
}
__device__ __forceinline__ const double* prim_boxes(const Dev& d, int k) {
  return k == 0 ? d.cv_box : (k == 1 ? d.tri_box : d.edge_box);
}

__global__ void k_bv_refit_cl(Dev d, int flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k = 0;
  while (k < 3 && c >= d.bv_n_cl[k]) c -= d.bv_n_cl[k++];
  if (k == 3) return;
  const int o = d.bv_cl_obj[k][c];
  if (!ENVI(d, d.obj_env[o], flag)) return;
  int pb, pe;
  prim_range(d, k, o, pb, pe);
  const int p0 = pb + 32 * (c - d.obj_cl_begin[k][o]), p1 = min(p0 + 32, pe);
  const double* pbox = prim_boxes(d, k);
  double bx[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int p = p0; p < p1; ++p) {
    const double* q = pbox + 6 * (long long)d.bv_perm[k][p];
    for (int j = 0; j < 3; ++j) { bx[j] = fmin(bx[j], q[j]); bx[3 + j] = fmax(bx[3 + j], q[3 + j]); }
  }
  double* out = d.bv_cl_box[k] + 6 * (long long)c;
  for (int j = 0; j < 6; ++j) out[j] = bx[j];
}

__global__ void k_bv_refit_sc(Dev d, int flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k = 0;
  while (k < 3 && c >= d.bv_n_sc[k]) c -= d.bv_n_sc[k++];
  if (k == 3) return;
  const int o = d.bv_sc_obj[k][c];
  if (!ENVI(d, d.obj_env[o], flag)) return;
  int pb, pe;
  prim_range(d, k, o, pb, pe);
  const int ncl = (pe - pb + 31) / 32;
  const int j0 = 32 * (c - d.obj_sc_begin[k][o]), j1 = min(j0 + 32, ncl);
  const double* cb = d.bv_cl_box[k] + 6 * (long long)d.obj_cl_begin[k][o];
  double bx[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int j = j0; j < j1; ++j)
    for (int q = 0; q < 3; ++q) { bx[q] = fmin(bx[q], cb[6 * j + q]); bx[3 + q] = fmax(bx[3 + q], cb[6 * j + 3 + q]); }
  double* out = d.bv_sc_box[k] + 6 * (long long)c;
  for (int j = 0; j < 6; ++j) out[j] = bx[j];
}

// Calls leaf(p) for every primitive p of kind k in object o whose
// supercluster and cluster boxes meet the query box qb (widened by dh); the
// leaf applies the exact box test itself.
template <class Leaf>
__device__ __forceinline__ void bv_query(const Dev& d, int k, int o, const double* qb, double dh, Leaf&& leaf) {
  int pb, pe;
  prim_range(d, k, o, pb, pe);
  const int ncl = (pe - pb + 31) / 32, nsc = (ncl + 31) / 32;
  const double* sb = d.bv_sc_box[k] + 6 * (long long)d.obj_sc_begin[k][o];
  const double* cb = d.bv_cl_box[k] + 6 * (long long)d.obj_cl_begin[k][o];
  const int* perm = d.bv_perm[k];
  for (int s = 0; s < nsc; ++s) {
    if (!overlap6(qb, sb + 6 * s, dh)) continue;
    const int j1 = min(32 * s + 32, ncl);
    for (int j = 32 * s; j < j1; ++j) {
      if (!overlap6(qb, cb + 6 * j, dh)) continue;
      const int p1 = min(pb + 32 * j + 32, pe);
      for (int p = pb + 32 * j; p < p1; ++p) leaf(perm[p]);
    }
  }
}

// Broad phase, stage 2: every item tests its query box against the boxes of
// the other object's primitives of the complementary kind, found through
// that object's cluster hierarchy (bv_query).  Within one
// (self-contacting) object: a point never pairs with a triangle it is a
// vertex of, and an edge pairs only with edges of higher index that share
// no vertex with it.
__global__ void k_pairs(Dev d) {
  const int n = min(*d.bp_count, d.bp_cap);
  const double dh = d.dhat;
  const double wscale = d.h * d.h * d.kappa;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    int4 item = d.bp_items[it];
    int qk = item.x, i = item.y, B = item.z, e = item.w;
    if (qk == 0) {
      const double* qb = d.cv_box + 6 * (long long)i;
      bool qfix = d.cv_fixed[i];
      const bool self = d.cv_obj[i] == B;
      bv_query(d, 1, B, qb, dh, [&](int t) {
        if (!overlap6(qb, d.tri_box + 6 * (long long)t, dh)) return;
        int t0 = d.tri[3 * t], t1 = d.tri[3 * t + 1], t2 = d.tri[3 * t + 2];
        if (self && (i == t0 || i == t1 || i == t2)) return;
        if (qfix && d.cv_fixed[t0] && d.cv_fixed[t1] && d.cv_fixed[t2]) return;
        emit_pair(d, e, make_int4(i, t0, t1, t2), 0, wscale * 0.5 * d.cv_area[i], 0.0);
      });
    } else if (qk == 1) {
      const double* qb = d.tri_box + 6 * (long long)i;
      int q0 = d.tri[3 * i], q1 = d.tri[3 * i + 1], q2 = d.tri[3 * i + 2];
      bool qfix = d.cv_fixed[q0] && d.cv_fixed[q1] && d.cv_fixed[q2];
      bv_query(d, 0, B, qb, dh, [&](int c) {
        if (!overlap6(qb, d.cv_box + 6 * (long long)c, dh)) return;
        if (qfix && d.cv_fixed[c]) return;
        emit_pair(d, e, make_int4(c, q0, q1, q2), 0, wscale * 0.5 * d.cv_area[c], 0.0);
      });
    } else {
      const double* qb = d.edge_box + 6 * (long long)i;
      int q0 = d.edge[2 * i], q1 = d.edge[2 * i + 1];
      bool qfix = d.cv_fixed[q0] && d.cv_fixed[q1];
      int A = d.edge_obj[i];
      const bool self = A == B;
      bv_query(d, 2, B, qb, dh, [&](int f) {
        if (self && f <= i) return;  // each unordered edge pair once
        if (!overlap6(qb, d.edge_box + 6 * (long long)f, dh)) return;
        int b0 = d.edge[2 * f], b1 = d.edge[2 * f + 1];
        if (self && (b0 == q0 || b0 == q1 || b1 == q0 || b1 == q1)) return;
        if (qfix && d.cv_fixed[b0] && d.cv_fixed[b1]) return;
        double w = wscale * 0.25 * (d.edge_area[i] + d.edge_area[f]);
        double eps = d.ee_moll * d.edge_len2[i] * d.edge_len2[f];
        int4 v = (A <= B) ? make_int4(q0, q1, b0, b1) : make_int4(b0, b1, q0, q1);
        emit_pair(d, e, v, 1, w, eps);
      });
    }
  }
}

__global__ void k_bp_reset(Dev d) {
  *d.bp_count = 0;
  *d.bp_overflow = 0;
}

// a worklist overflow marks every selected env as overflowed (conservative)
__global__ void k_bp_check(Dev d, int flag) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < d.n_envs && *d.bp_overflow && ENVI(d, e, flag)) ENVI(d, e, I_OVERFLOW) = 1;
}

// Exclusive scan of a per-env count over the envs (one CTA): the pair and
// friction kernels then walk a flat index space of real items only.
//   which 0: candidate pairs, min(I_NPAIRS, capacity), into pair_scan;
//   which 1: friction records of the envs still iterating, into fr_scan.
__global__ void k_env_scan(Dev d, int which) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  int* out = which == 0 ? d.pair_scan : d.fr_scan;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < d.n_envs; base += blockDim.x) {
    int e = base + threadIdx.x;
    int c = 0;
    if (e < d.n_envs) {
      if (which == 0) c = min(ENVI(d, e, I_NPAIRS), d.env_pair_cap[e]);
      else c = ENVI(d, e, I_ACTIVE) ? min(ENVI(d, e, I_NFRIC), d.env_pair_cap[e]) : 0;
    }
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
      int vi = v;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, vi, o);
        if (lane >= o) vi += t;
      }
      warp_tot[lane] = vi - v;  // exclusive warp offsets
    }
    __syncthreads();
    int excl = carry + warp_tot[wid] + incl - c;
    if (e < d.n_envs) out[e] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + c;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[d.n_envs] = carry;
}

// flat index f over real pairs -> (env, slot k in capacity space)
__device__ __forceinline__ int pair_at(const Dev& d, int f, int& e) {
  e = find_env(d.pair_scan, d.n_envs, f);
  return d.env_pair_off[e] + (f - d.pair_scan[e]);
}

#define FOR_PAIRS(d, f) for (int f = blockIdx.x * blockDim.x + threadIdx.x, _n = (d).pair_scan[(d).n_envs]; f < _n; \
                             f += gridDim.x * blockDim.x)

// env of pair slot k (segments of capacity env_pair_cap) and validity
__device__ __forceinline__ int pair_env(const Dev& d, int k, bool& valid) {
  int e = find_env(d.env_pair_off, d.n_envs, k);
  valid = (k - d.env_pair_off[e]) < min(ENVI(d, e, I_NPAIRS), d.env_pair_cap[e]);
  return e;
}

// ---------------------------------------------------------------------------
// barrier: energy, gradient (scattered into qc), PSD Hessian (stored), and the
// diagonal-block preconditioner contributions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scatter_cv(const Dev& d, double* dst, int cv, D3 gvec) {
  int row = d.cv_row[cv];
  if (d.cv_body[cv] < 0) {
    if (d.row_kind[row] == ROW_PINNED) return;
    atomic_add3(dst, row, gvec);
  } else {
    D3 xb = ld3(d.cv_xbar, cv);
    atomic_add3(dst, row, gvec);
    atomic_add3(dst, row + 1, xb.x * gvec);
    atomic_add3(dst, row + 2, xb.y * gvec);
    atomic_add3(dst, row + 3, xb.z * gvec);
  }
}

// tag the rows scatter_cv writes for contact vertex cv (the PCG update reads
// the contact accumulator only on tagged rows)
__device__ __forceinline__ void touch_cv(const Dev& d, int cv, uint8_t tag) {
  const int row = d.cv_row[cv];
  if (d.cv_body[cv] < 0) {
    if (d.row_kind[row] != ROW_PINNED) d.row_touch[row] = tag;
  } else {
    for (int k = 0; k < 4; ++k) d.row_touch[row + k] = tag;
  }
}

// HT: storage type of the pair Hessian (double: FP64 mode; float: mixed
// mode).  Distances, barrier derivatives and the projection are FP64 either way.
template <class HT>
__global__ void k_barrier(Dev d, int flag) {
  FOR_PAIRS(d, f) {
  int e;
  int k = pair_at(d, f, e);
  int cvs[4] = {0, 0, 0, 0};
  double E, g[12];
  HT H[144];
  bool act = false;
  if (ENVI(d, e, flag) &&
      IPC_CHECK(d.check_word, (unsigned)d.pair_v[k].x < (unsigned)d.n_cv && (unsigned)d.pair_v[k].y < (unsigned)d.n_cv &&
                (unsigned)d.pair_v[k].z < (unsigned)d.n_cv && (unsigned)d.pair_v[k].w < (unsigned)d.n_cv,
                CHK_PAIR_VERT, k)) {
    int4 v = d.pair_v[k];
    cvs[0] = v.x; cvs[1] = v.y; cvs[2] = v.z; cvs[3] = v.w;
    D3 X[4];
    for (int i = 0; i < 4; ++i) X[i] = ld3(d.cvx, cvs[i]);
    act = pair_barrier<HT>(X, d.pair_kind[k] == 1, d.pair_w[k], d.pair_eps[k], d.dhat, &E, g, H,
                           newton_filter(d, e));
    d.pair_act[k] = act ? 1 : 0;
  }
  // the active pairs of an env fill its slots env_pair_off[e] + [0, I_NACT)
  // in any order; the warp's lanes of one env take consecutive slots (one
  // atomic per env present in the warp)
  const unsigned wm = __activemask();
  const unsigned am = __ballot_sync(wm, act);
  if (!act) continue;
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(am, e);
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&ENVI(d, e, I_NACT), __popc(grp));
  base = __shfl_sync(grp, base, leader);
  const int slot = d.env_pair_off[e] + base + __popc(grp & ((1u << lane) - 1u));
  d.act_v[slot] = make_int4(cvs[0], cvs[1], cvs[2], cvs[3]);
  // interleaved by warp of slots so that the mat-vec's loads coalesce
  HT* Hs = reinterpret_cast<HT*>(d.pair_H) + (long long)(slot >> 5) * 78 * 32 + (slot & 31);
  for (int p = 0, o = 0; p < 12; ++p)
    for (int q = p; q < 12; ++q, ++o) Hs[o * 32] = H[p * 12 + q];
  const uint8_t tag = touch_tag(d, e);
  for (int i = 0; i < 4; ++i) touch_cv(d, cvs[i], tag);
  for (int i = 0; i < 4; ++i) scatter_cv(d, d.qc, cvs[i], D3{g[3 * i], g[3 * i + 1], g[3 * i + 2]});
  // preconditioner: diagonal 3x3 of gel vertices, body 12x12 self terms
  for (int i = 0; i < 4; ++i) {
    int cv = cvs[i];
    if (d.cv_body[cv] >= 0) continue;
    int row = d.cv_row[cv];
    if (d.row_kind[row] == ROW_PINNED) continue;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) atomicAdd(d.pc_acc + 9 * row + 3 * a + b, (double)H[(3 * i + a) * 12 + 3 * i + b]);
  }
  int done_body[4] = {-1, -1, -1, -1};
  for (int i = 0; i < 4; ++i) {
    int b = d.cv_body[cvs[i]];
    if (b < 0) continue;
    bool seen = false;
    for (int j = 0; j < i; ++j) seen |= (done_body[j] == b);
    done_body[i] = b;
    if (seen) continue;
    // M_kl (3x3 blocks k,l in 0..3) = sum_{i,j on b} w_ik w_jl H_ij, w = [1, xbar]
    HT wv[4][4];
    bool on[4];
    for (int m = 0; m < 4; ++m) {
      on[m] = d.cv_body[cvs[m]] == b;
      D3 xb = ld3(d.cv_xbar, cvs[m]);
      wv[m][0] = HT(1); wv[m][1] = (HT)xb.x; wv[m][2] = (HT)xb.y; wv[m][3] = (HT)xb.z;
    }
    for (int kk = 0; kk < 4; ++kk)
      for (int ll = 0; ll < 4; ++ll)
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) {
            HT s = 0;
            for (int m = 0; m < 4; ++m) {
              if (!on[m]) continue;
              for (int n = 0; n < 4; ++n) {
                if (!on[n]) continue;
                s += wv[m][kk] * wv[n][ll] * H[(3 * m + a) * 12 + 3 * n + c];
              }
            }
            atomicAdd(d.body_pc_acc + 144 * b + (3 * kk + a) * 12 + 3 * ll + c, (double)s);
          }
  }
  }
}

// ACCD time of impact per swept pair; env bound = min over its pairs
// ACCD (additive CCD): per swept pair a conservative time of impact; the
// env's step bound is the minimum over its pairs (S_ACCD, a running min).
// Phase 1 (one pair per thread): the sequential advancement, at most
// kAccdSeq iterations.  Pairs still advancing after that (sliding contacts
// at small distance take ~l_p / d iterations) continue in phase 2, where one
// warp advances one pair 32 certified intervals at a time.  A pair whose
// sequential run ends within kAccdSeq iterations gets exactly the
// sequential result.
constexpr int kAccdSeq = 64;

struct AccdPair {
  D3 X[4], P[4];
  double lp, gap;
  bool ee;
};

__device__ __forceinline__ void accd_setup(const Dev& d, int k, double s, AccdPair& a) {
  int4 v = d.pair_v[k];
  int cvs[4] = {v.x, v.y, v.z, v.w};
  for (int i = 0; i < 4; ++i) { a.X[i] = ld3(d.cvx, cvs[i]); a.P[i] = ld3(d.cvp, cvs[i]); }
  a.ee = d.pair_kind[k] == 1;
  D3 pm = 0.25 * (a.P[0] + a.P[1] + a.P[2] + a.P[3]);
  double nq[4];
  for (int i = 0; i < 4; ++i) nq[i] = sqrt(norm2(a.P[i] - pm));
  a.lp = a.ee ? fmax(nq[0], nq[1]) + fmax(nq[2], nq[3]) : nq[0] + fmax(nq[1], fmax(nq[2], nq[3]));
  a.gap = s * sqrt(pair_sqdist(a.X, a.ee));
}

__device__ __forceinline__ double accd_dist_at(const AccdPair& a, double t) {
  D3 Y[4];
  for (int i = 0; i < 4; ++i) Y[i] = a.X[i] + t * a.P[i];
  return sqrt(pair_sqdist(Y, a.ee));
}

__global__ void k_accd(Dev d) {
  FOR_PAIRS(d, f) {
  int e;
  int k = pair_at(d, f, e);
  if (!ENVI(d, e, I_LS)) continue;
  int4 v = d.pair_v[k];
  int cvs[4] = {v.x, v.y, v.z, v.w};
  D3 X[4], P[4];
  for (int i = 0; i < 4; ++i) { X[i] = ld3(d.cvx, cvs[i]); P[i] = ld3(d.cvp, cvs[i]); }
  const int seq_cap = min(d.accd_max, kAccdSeq);
  int its = 0;
  bool more = false;
  double t = accd_toi(X, P, d.pair_kind[k] == 1, d.accd_s, 1.0, seq_cap, &its, &ENVS(d, e, S_ACCD), &more);
  // still advancing after the sequential budget (below t = 1)
  if (more && d.accd_max > seq_cap) {
    unsigned slot = atomicAdd(&d.accd_tail_ctl[0], 1u);
    d.accd_tail[slot] = make_int4(k, e, its, 0);
    d.accd_tail_t[slot] = t;
    continue;
  }
  atomic_min_nonneg(&ENVS(d, e, S_ACCD), t);
  atomicAdd(&ENVI(d, e, I_ACCDIT), its);
  atomicMax(&ENVI(d, e, I_ACCDMAX), its);
  }
}

// Phase 2, one warp per pair.  From a certified time t with distance
// d_t >= gap, lane j evaluates the distance at t_j = t + (j + 1) D,
// D = 1.8 (d_t - gap) / l_p (clamped to t_j <= 1).  |d'| <= l_p, so on
// [t_{j-1}, t_j] the distance is at least (d_{j-1} + d_j - l_p D) / 2; the
// warp advances to the end of the longest prefix of intervals whose bound is
// >= gap.  When even the first interval fails, one sequential ACCD step is
// taken instead (step 0.9 d_t / l_p, stop if the distance there is below
// gap).  Each round counts 32 iterations against accd_max.  Guarantee as in
// the sequential form: no contact on [0, t] and distance >= gap at t.
__global__ void k_accd_tail(Dev d) {
  const unsigned n_tail = d.accd_tail_ctl[0];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned w = warp; w < n_tail; w += n_warps) {
    int4 ent = d.accd_tail[w];
    const int k = ent.x, e = ent.y;
    int its = ent.z;
    double t = d.accd_tail_t[w];
    AccdPair a;
    accd_setup(d, k, d.accd_s, a);
    double dt = accd_dist_at(a, t);
    while (t < 1.0 && its < d.accd_max) {
      const double cap = __shfl_sync(0xffffffffu, *(volatile double*)&ENVS(d, e, S_ACCD), 0);
      if (t >= cap) break;
      const double D = 1.8 * (dt - a.gap) / a.lp;
      const double tj = fmin(1.0, t + (lane + 1) * D);
      const double dj = accd_dist_at(a, tj);
      double dprev = __shfl_up_sync(0xffffffffu, dj, 1);
      double tprev = __shfl_up_sync(0xffffffffu, tj, 1);
      if (lane == 0) { dprev = dt; tprev = t; }
      const bool ok = (tj > tprev) ? (0.5 * (dprev + dj - a.lp * (tj - tprev)) >= a.gap) : true;
      const unsigned bad = __ballot_sync(0xffffffffu, !ok);
      its += 32;
      if (bad == 0u) {
        t = __shfl_sync(0xffffffffu, tj, 31);
        dt = __shfl_sync(0xffffffffu, dj, 31);
        continue;
      }
      const int first = __ffs(bad) - 1;
      if (first > 0) {
        t = __shfl_sync(0xffffffffu, tj, first - 1);
        dt = __shfl_sync(0xffffffffu, dj, first - 1);
        continue;
      }
      // no interval certified: one sequential step
      const double tn = fmin(1.0, t + 0.9 * dt / a.lp);
      const double dn = accd_dist_at(a, tn);
      if (dn < a.gap) break;
      t = tn;
      dt = dn;
    }
    if (t >= 1.0) t = 1.0;
    if (lane == 0) {
      atomic_min_nonneg(&ENVS(d, e, S_ACCD), t);
      atomicAdd(&ENVI(d, e, I_ACCDIT), its);
      atomicMax(&ENVI(d, e, I_ACCDMAX), its);
    }
  }
  // the last CTA to finish clears the list for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned done = atomicAdd(&d.accd_tail_ctl[1], 1u);
    if (done == gridDim.x - 1) {
      d.accd_tail_ctl[0] = 0u;
      d.accd_tail_ctl[1] = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// Lagged friction (App. A.3): the objective carries h^2 sum_k mu lambda_k^n
// f0(|u_k|), f0' = f1 = -y^2/(eps_v h)^2 + 2 y/(eps_v h) below eps_v h, 1 above.
// Lagged at x^n for every static pair within dhat: the closest-point weights
// w (r = sum_i w_i x_i, the difference of the closest points), the tangent
// basis T of the plane normal to r (first axis: the coordinate axis least
// aligned with r, made orthogonal), lambda = kappa A c |b'(d)| (c: edge-edge
// mollifier) and r(x^n).  u = T^T (r(x) - r(x^n)).  In the tangent frame the
// Hessian mu lambda [g I + g'/y u u^T], g = f1/y, has eigenvalues g and f1',
// both >= 0: no projection.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fr_f0(double y, double eh) {
  return y >= eh ? y : (-y * y * y / (3.0 * eh * eh) + y * y / eh + eh / 3.0);
}
__device__ __forceinline__ double fr_g(double y, double eh) {  // f1(y) / y
  return y >= eh ? 1.0 / y : (-y / (eh * eh) + 2.0 / eh);
}
__device__ __forceinline__ double fr_dg_y(double y, double eh) {  // g'(y) / y
  if (!(y > 0.0)) return 0.0;
  return y >= eh ? -1.0 / (y * y * y) : -1.0 / (eh * eh * y);
}

__device__ void fr_basis(D3 n, D3& t1, D3& t2) {
  double an[3] = {fabs(n.x), fabs(n.y), fabs(n.z)};
  int k = 0;
  if (an[1] < an[k]) k = 1;
  if (an[2] < an[k]) k = 2;
  D3 a{k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
  t1 = a - dot(a, n) * n;
  t1 = (1.0 / sqrt(norm2(t1))) * t1;
  t2 = cross(n, t1);
}

// the 4 contact points of a record at positions cvx + alpha cvp
__device__ __forceinline__ void fr_points(const Dev& d, int4 v, double alpha, D3* X) {
  int cvs[4] = {v.x, v.y, v.z, v.w};
  for (int i = 0; i < 4; ++i) X[i] = ld3(d.cvx, cvs[i]) + alpha * ld3(d.cvp, cvs[i]);
}

// u = T^T (sum_i w_i X_i - r_n)
__device__ __forceinline__ void fr_u(const Dev& d, int j, const D3* X, double& u0, double& u1, D3& t1, D3& t2) {
  const double* w = d.fr_w + 4 * (long long)j;
  D3 s = w[0] * X[0] + w[1] * X[1] + w[2] * X[2] + w[3] * X[3] - ld3(d.fr_rn, j);
  const double* T = d.fr_T + 6 * (long long)j;
  t1 = D3{T[0], T[1], T[2]};
  t2 = D3{T[3], T[4], T[5]};
  u0 = dot(t1, s);
  u1 = dot(t2, s);
}

// The first Newton iteration of an env's step (x = x^n): one record per
// static pair within dhat, in the env's segment (I_NFRIC was zeroed when
// the step began).  Envs may be at different iterations of their steps.
__global__ void k_fric_setup(Dev d) {
  FOR_PAIRS(d, f) {
  int e;
  int k = pair_at(d, f, e);
  if (!ENVI(d, e, I_NEWT) || ENVI(d, e, I_NEWTON) != 1) continue;
  int4 v = d.pair_v[k];
  D3 X[4];
  fr_points(d, v, 0.0, X);
  const bool ee = d.pair_kind[k] == 1;
  Closest cl;
  classify(X, ee, cl);
  const double dist = sqrt(cl.D);
  if (!(dist > 0.0) || dist >= d.dhat) continue;
  double c = 1.0;
  if (ee) {
    const double xm = ee_cross2(X, nullptr, nullptr), eps = d.pair_eps[k];
    if (xm < eps) c = (-xm / eps + 2.0) * xm / eps;
  }
  double b, b1, b2;
  barrier_d(dist, d.dhat, b, b1, b2);
  const double lam = d.pair_w[k] / (d.h * d.h) * c * fabs(b1);  // pair_w = h^2 kappa A
  if (!(lam > 0.0)) continue;
  int slot = atomicAdd(&ENVI(d, e, I_NFRIC), 1);
  if (slot >= d.env_pair_cap[e]) {
    ENVI(d, e, I_OVERFLOW) = 1;
    continue;
  }
  const int j = d.env_pair_off[e] + slot;
  d.fr_v[j] = v;
  for (int i = 0; i < 4; ++i) d.fr_w[4 * (long long)j + i] = cl.w[i];
  D3 t1, t2;
  fr_basis((1.0 / dist) * cl.r, t1, t2);
  double* T = d.fr_T + 6 * (long long)j;
  T[0] = t1.x; T[1] = t1.y; T[2] = t1.z; T[3] = t2.x; T[4] = t2.y; T[5] = t2.z;
  st3(d.fr_rn, j, cl.r);
  d.fr_ml[j] = d.fr_mu * lam;
  }
}

// flat index li over the records of the envs still iterating (fr_scan) ->
// (env e, record j)
#define FOR_FRIC(d, li) for (int li = blockIdx.x * blockDim.x + threadIdx.x, _nf = (d).fr_scan[(d).n_envs]; li < _nf; \
                             li += gridDim.x * blockDim.x)
__device__ __forceinline__ int fric_at(const Dev& d, int li, int& e) {
  e = find_env(d.fr_scan, d.n_envs, li);
  return d.env_pair_off[e] + (li - d.fr_scan[e]);
}

// Each Newton iteration: gradient (into the contact accumulator qc, like the
// barrier), the 3x3 matrix S = h^2 mu lambda T M T^T of the record, and the
// preconditioner blocks w_i w_j S.
__global__ void k_fric_assemble(Dev d) {
  FOR_FRIC(d, li) {
  int e;
  const int j = fric_at(d, li, e);
  if (!ENVI(d, e, I_NEWT)) continue;
  const int4 v = d.fr_v[j];
  const int cvs[4] = {v.x, v.y, v.z, v.w};
  D3 X[4];
  fr_points(d, v, 0.0, X);
  double u0, u1;
  D3 t1, t2;
  fr_u(d, j, X, u0, u1, t1, t2);
  const double y = sqrt(u0 * u0 + u1 * u1);
  const double sc = d.h * d.h * d.fr_ml[j];
  const double g = fr_g(y, d.fr_eh), gy = fr_dg_y(y, d.fr_eh);
  const D3 Tu = u0 * t1 + u1 * t2;
  const double* w = d.fr_w + 4 * (long long)j;
  for (int i = 0; i < 4; ++i) scatter_cv(d, d.qc, cvs[i], (sc * g * w[i]) * Tu);
  const uint8_t tag = touch_tag(d, e);
  for (int i = 0; i < 4; ++i) touch_cv(d, cvs[i], tag);
  // M = g I + gy u u^T (2x2) -> S = sc T M T^T = sc (g (t1 t1^T + t2 t2^T) + gy Tu Tu^T)
  double S[3][3];
  const double ta[3] = {t1.x, t1.y, t1.z}, tb[3] = {t2.x, t2.y, t2.z}, tu[3] = {Tu.x, Tu.y, Tu.z};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) S[a][c] = sc * (g * (ta[a] * ta[c] + tb[a] * tb[c]) + gy * tu[a] * tu[c]);
  double* Sp = d.fr_S + 6 * (long long)j;
  Sp[0] = S[0][0]; Sp[1] = S[0][1]; Sp[2] = S[0][2]; Sp[3] = S[1][1]; Sp[4] = S[1][2]; Sp[5] = S[2][2];
  for (int i = 0; i < 4; ++i) {
    int cv = cvs[i];
    if (d.cv_body[cv] >= 0) continue;
    int row = d.cv_row[cv];
    if (d.row_kind[row] == ROW_PINNED) continue;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) atomicAdd(d.pc_acc + 9 * row + 3 * a + c, w[i] * w[i] * S[a][c]);
  }
  int done_body[4] = {-1, -1, -1, -1};
  for (int i = 0; i < 4; ++i) {
    int b = d.cv_body[cvs[i]];
    if (b < 0) continue;
    bool seen = false;
    for (int m = 0; m < i; ++m) seen |= (done_body[m] == b);
    done_body[i] = b;
    if (seen) continue;
    // body blocks: sum over points m, n on b of J_m^T (w_m w_n S) J_n
    double wv[4][4];
    bool on[4];
    for (int m = 0; m < 4; ++m) {
      on[m] = d.cv_body[cvs[m]] == b;
      D3 xb = ld3(d.cv_xbar, cvs[m]);
      wv[m][0] = w[m]; wv[m][1] = w[m] * xb.x; wv[m][2] = w[m] * xb.y; wv[m][3] = w[m] * xb.z;
    }
    for (int kk = 0; kk < 4; ++kk)
      for (int ll = 0; ll < 4; ++ll) {
        double cw = 0.0;
        for (int m = 0; m < 4; ++m) {
          if (!on[m]) continue;
          for (int n = 0; n < 4; ++n)
            if (on[n]) cw += wv[m][kk] * wv[n][ll];
        }
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) atomicAdd(d.body_pc_acc + 144 * b + (3 * kk + a) * 12 + 3 * ll + c, cw * S[a][c]);
      }
  }
  }
}

// PCG mat-vec, after the SELL / pair mat-vec of the same iteration (which
// wrote this iteration's direction): q_c += w_i S (sum_j w_j d_j) per record
// (pinned gel rows read as zero and are never written), and the record's
// a^T S a (a = sum_j w_j d_j) into the env's contact part of d.q.
__global__ void k_fric_spmv(Dev d) {
  const int nb = pcg_new_buf(d);
  FOR_FRIC(d, li) {
  int e;
  const int j = fric_at(d, li, e);
  if (!ENVI(d, e, I_PCG)) continue;
  const int4 v = d.fr_v[j];
  const int cvs[4] = {v.x, v.y, v.z, v.w};
  const double* w = d.fr_w + 4 * (long long)j;
  D3 a{0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    int cv = cvs[i], row = d.cv_row[cv];
    D3 u;
    if (d.cv_body[cv] < 0) u = (d.row_kind[row] == ROW_PINNED) ? D3{0, 0, 0} : dir_row(d, row, nb);
    else u = dir_body_point(d, row, ld3(d.cv_xbar, cv), nb);
    a = a + w[i] * u;
  }
  const double* S = d.fr_S + 6 * (long long)j;
  D3 t{S[0] * a.x + S[1] * a.y + S[2] * a.z, S[1] * a.x + S[3] * a.y + S[4] * a.z,
       S[2] * a.x + S[4] * a.y + S[5] * a.z};
  for (int i = 0; i < 4; ++i) scatter_cv(d, d.qc, cvs[i], w[i] * t);
  atomicAdd(&ENVS(d, e, S_DQC), dot(a, t));
  }
}

// line-search energy of each record: h^2 mu lambda f0(|u|) at x + alpha p
__global__ void k_fric_energy(Dev d, int use_alpha) {
  FOR_FRIC(d, li) {
  int e;
  const int j = fric_at(d, li, e);
  if (!ENVI(d, e, I_LS)) continue;
  const double a = use_alpha ? ENVS(d, e, S_ALPHA) : 0.0;
  D3 X[4];
  fr_points(d, d.fr_v[j], a, X);
  double u0, u1;
  D3 t1, t2;
  fr_u(d, j, X, u0, u1, t1, t2);
  d.fr_E[j] = d.h * d.h * d.fr_ml[j] * fr_f0(sqrt(u0 * u0 + u1 * u1), d.fr_eh);
  }
}

// barrier energy of each swept pair at x + alpha p (+inf if touching)
__global__ void k_pair_energy(Dev d, int use_alpha) {
  FOR_PAIRS(d, f) {
  int e;
  int k = pair_at(d, f, e);
  if (!ENVI(d, e, I_LS)) continue;
  double a = use_alpha ? ENVS(d, e, S_ALPHA) : 0.0;
  int4 v = d.pair_v[k];
  int cvs[4] = {v.x, v.y, v.z, v.w};
  D3 X[4];
  for (int i = 0; i < 4; ++i) X[i] = ld3(d.cvx, cvs[i]) + a * ld3(d.cvp, cvs[i]);
  double D = pair_sqdist(X, d.pair_kind[k] == 1);
  double E = 0.0;
  if (!(D > 0.0)) E = INFINITY;
  else pair_barrier<double>(X, d.pair_kind[k] == 1, d.pair_w[k], d.pair_eps[k], d.dhat, &E, nullptr, nullptr);
  d.pair_E[k] = E;
  }
}

// min distance over the listed pairs (diagnostics / set_state check)
__global__ void k_min_dist(Dev d, int flag) {
  FOR_PAIRS(d, f) {
  int e;
  int k = pair_at(d, f, e);
  if (!ENVI(d, e, flag)) continue;
  int4 v = d.pair_v[k];
  int cvs[4] = {v.x, v.y, v.z, v.w};
  D3 X[4];
  for (int i = 0; i < 4; ++i) X[i] = ld3(d.cvx, cvs[i]);
  double D = pair_sqdist(X, d.pair_kind[k] == 1);
  atomic_min_nonneg(&ENVS(d, e, S_MIND), sqrt(fmax(D, 0.0)));
  }
}

// ---------------------------------------------------------------------------
// crossing surfaces (set_state): an edge of one contact object passing
// through a triangle of another (or, in a self-contacting pad, through a
// triangle of its own that shares no vertex with it) sets I_FLAG = 2.
// One thread per edge; boxes first (through the other object's triangle
// hierarchy, refitted by the candidate search), then the exact-sign test: segment PQ
// meets triangle ABC iff P and Q are not strictly on one side of ABC's plane
// and the line PQ passes on the same side of the three triangle edges.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double orient3(D3 a, D3 b, D3 c, D3 d) { return dot(cross(b - a, c - a), d - a); }

__device__ bool segment_meets_triangle(D3 p, D3 q, D3 a, D3 b, D3 c) {
  const double sp = orient3(a, b, c, p), sq = orient3(a, b, c, q);
  if ((sp > 0.0 && sq > 0.0) || (sp < 0.0 && sq < 0.0)) return false;
  if (sp == 0.0 && sq == 0.0) return false;  // coplanar: left to the distance check
  const double s0 = orient3(p, q, a, b), s1 = orient3(p, q, b, c), s2 = orient3(p, q, c, a);
  return (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) || (s0 <= 0.0 && s1 <= 0.0 && s2 <= 0.0);
}

__global__ void k_cross_check(Dev d, int flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_edge) return;
  const int e = find_env(d.env_edge_off, d.n_envs, i);
  if (!ENVI(d, e, flag)) return;
  const int A = d.edge_obj[i];
  const int q0 = d.edge[2 * i], q1 = d.edge[2 * i + 1];
  const D3 P = ld3(d.cvx, q0), Q = ld3(d.cvx, q1);
  double bx[6] = {fmin(P.x, Q.x), fmin(P.y, Q.y), fmin(P.z, Q.z), fmax(P.x, Q.x), fmax(P.y, Q.y), fmax(P.z, Q.z)};
  const unsigned long long ex = d.obj_exclude[A];
  bool hit = false;
  for (int B = d.env_obj_off[e]; B < d.env_obj_off[e + 1] && !hit; ++B) {
    if ((ex >> d.obj_local[B]) & 1ull) continue;   // excluded object pair (or a pad without self-contact)
    bv_query(d, 1, B, bx, 0.0, [&](int t) {
      if (hit || !overlap6(bx, d.tri_box + 6 * (long long)t, 0.0)) return;
      const int t0 = d.tri[3 * t], t1 = d.tri[3 * t + 1], t2 = d.tri[3 * t + 2];
      if (B == A && (t0 == q0 || t0 == q1 || t1 == q0 || t1 == q1 || t2 == q0 || t2 == q1)) return;
      hit = segment_meets_triangle(P, Q, ld3(d.cvx, t0), ld3(d.cvx, t1), ld3(d.cvx, t2));
    });
  }
  if (hit && ENVI(d, e, I_FLAG) == 0) ENVI(d, e, I_FLAG) = 2;  // an inverted tet (1) takes precedence
}

// |J_j p_b|_inf over body vertices into S_PNORM; |J_j (y_b - s_b)|_inf of
// driven bodies into S_CRES
__global__ void k_pnorm_body(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n_cv) return;
  int b = d.cv_body[c];
  if (b < 0) return;
  int e = d.body_env[b];
  if (!ENVI(d, e, I_DEC)) return;
  int row = d.cv_row[c];
  D3 xb = ld3(d.cv_xbar, c);
  D3 u = body_point(d.p, row, xb);
  atomic_max_nonneg(&ENVS(d, e, S_PNORM), fmax(fabs(u.x), fmax(fabs(u.y), fabs(u.z))));
  if (d.body_driven[b]) {
    D3 r = body_point(d.x, row, xb) - body_point(d.s_tgt, row, xb);
    atomic_max_nonneg(&ENVS(d, e, S_CRES), fmax(fabs(r.x), fmax(fabs(r.y), fabs(r.z))));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_cv_pos(const Dev& d, int flag, bool with_disp, cudaStream_t s) {
  if (!d.n_cv) return 0;
  k_cv_pos<<<nblk(d.n_cv, 256), 256, 0, s>>>(d, flag, with_disp ? 1 : 0);
  return 1;
}
// primitive boxes + object boxes (the object boxes feed the worklist)
int launch_obj_box(const Dev& d, int flag, bool swept, cudaStream_t s) {
  long long n = (long long)d.n_cv + d.n_tri + d.n_edge;
  if (!n) return 0;
  k_prim_boxes<<<nblk(n, 256), 256, 0, s>>>(d, flag, swept ? 1 : 0);
  k_obj_box<<<d.n_obj, 256, 0, s>>>(d, flag);
  return 2;
}
int launch_broad(const Dev& d, int flag, bool swept, cudaStream_t s) {
  (void)swept;  // boxes already include the sweep
  k_bp_reset<<<1, 1, 0, s>>>(d);
  int n = 1;
  if (d.n_cv) { k_worklist<0><<<nblk(d.n_cv, 128), 128, 0, s>>>(d, flag); ++n; }
  if (d.n_tri) { k_worklist<1><<<nblk(d.n_tri, 128), 128, 0, s>>>(d, flag); ++n; }
  if (d.n_edge) { k_worklist<2><<<nblk(d.n_edge, 128), 128, 0, s>>>(d, flag); ++n; }
  {
    const int ncl = d.bv_n_cl[0] + d.bv_n_cl[1] + d.bv_n_cl[2], nsc = d.bv_n_sc[0] + d.bv_n_sc[1] + d.bv_n_sc[2];
    if (ncl) { k_bv_refit_cl<<<nblk(ncl, 128), 128, 0, s>>>(d, flag); ++n; }
    if (nsc) { k_bv_refit_sc<<<nblk(nsc, 128), 128, 0, s>>>(d, flag); ++n; }
  }
  k_pairs<<<d.pairs_grid > 0 ? d.pairs_grid : 148 * 8, 128, 0, s>>>(d);
  k_bp_check<<<nblk(d.n_envs, 128), 128, 0, s>>>(d, flag);
  k_env_scan<<<1, 1024, 0, s>>>(d, 0);
  return n + 3;
}
// pair kernels grid-stride over the real pairs (count on the device)
#define PAIR_GRID 148 * 8, 128, 0, s
int launch_barrier(const Dev& d, int flag, cudaStream_t s) {
  if (!d.n_pairs_cap) return 0;
  if (d.prec) k_barrier<float><<<PAIR_GRID>>>(d, flag);
  else k_barrier<double><<<PAIR_GRID>>>(d, flag);
  return 1;
}
int launch_fric_setup(const Dev& d, cudaStream_t s) {
  if (!(d.fr_mu > 0.0) || !d.n_pairs_cap) return 0;
  k_fric_setup<<<PAIR_GRID>>>(d);
  k_env_scan<<<1, 1024, 0, s>>>(d, 1);
  return 2;
}
int launch_fric_assemble(const Dev& d, cudaStream_t s) {
  if (!(d.fr_mu > 0.0) || !d.n_pairs_cap) return 0;
  k_fric_assemble<<<PAIR_GRID>>>(d);
  return 1;
}
int launch_fric_spmv(const Dev& d, cudaStream_t s) {
  if (!(d.fr_mu > 0.0) || !d.n_pairs_cap) return 0;
  k_fric_spmv<<<PAIR_GRID>>>(d);
  return 1;
}
int launch_fric_energy(const Dev& d, int use_alpha, cudaStream_t s) {
  if (!(d.fr_mu > 0.0) || !d.n_pairs_cap) return 0;
  k_fric_energy<<<PAIR_GRID>>>(d, use_alpha);
  return 1;
}
int launch_accd(const Dev& d, cudaStream_t s) {
  if (!d.n_pairs_cap) return 0;
  k_accd<<<PAIR_GRID>>>(d);
  k_accd_tail<<<148 * 4, 256, 0, s>>>(d);
  return 2;
}
int launch_pair_energy(const Dev& d, int use_alpha, cudaStream_t s) {
  if (!d.n_pairs_cap) return 0;
  k_pair_energy<<<PAIR_GRID>>>(d, use_alpha);
  return 1;
}
int launch_cross_check(const Dev& d, int flag, cudaStream_t s) {
  if (!d.n_edge) return 0;
  k_cross_check<<<nblk(d.n_edge, 128), 128, 0, s>>>(d, flag);
  return 1;
}
int launch_min_dist(const Dev& d, int flag, cudaStream_t s) {
  if (!d.n_pairs_cap) return 0;
  k_min_dist<<<PAIR_GRID>>>(d, flag);
  return 1;
}
int launch_pnorm_body(const Dev& d, cudaStream_t s) {
  if (!d.n_cv) return 0;
  k_pnorm_body<<<nblk(d.n_cv, 256), 256, 0, s>>>(d);
  return 1;
}

// ---------------------------------------------------------------------------
// element kernels on caller buffers
// ---------------------------------------------------------------------------
__global__ void k_elem_barrier(int n, const double* X, const int* is_ee, const double* w, const double* eps,
                               double dhat, double* E, double* g, double* H, int project) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  D3 P[4];
  for (int i = 0; i < 4; ++i) P[i] = ld3(X + 12 * (long long)k, i);
  double e = 0, gl[12];
  double* Hk = H ? H + 144 * (long long)k : nullptr;
  const int filt = project & 3;
  bool act;
  if (project & 8) {  // the mixed mode's FP32 Hessian, widened on output
    float Hf[144];
    act = pair_barrier<float>(P, is_ee[k] != 0, w[k], eps ? eps[k] : 0.0, dhat, &e, g ? gl : nullptr,
                              Hk ? Hf : nullptr, filt);
    if (Hk && act)
      for (int i = 0; i < 144; ++i) Hk[i] = (double)Hf[i];
  } else {
    act = pair_barrier<double>(P, is_ee[k] != 0, w[k], eps ? eps[k] : 0.0, dhat, &e, g ? gl : nullptr, Hk, filt);
  }
  if (E) E[k] = e;
  if (g)
    for (int i = 0; i < 12; ++i) g[12 * (long long)k + i] = act ? gl[i] : 0.0;
  if (Hk && !act)
    for (int i = 0; i < 144; ++i) Hk[i] = 0.0;
}

__global__ void k_elem_accd(int n, const double* X0, const double* P, const int* is_ee, double sfrac,
                            int max_iter, double* toi, int* iters) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  D3 A[4], B[4];
  for (int i = 0; i < 4; ++i) { A[i] = ld3(X0 + 12 * (long long)k, i); B[i] = ld3(P + 12 * (long long)k, i); }
  int it = 0;
  toi[k] = accd_toi(A, B, is_ee[k] != 0, sfrac, 1.0, max_iter, &it);
  if (iters) iters[k] = it;
}

int launch_k_barrier(int n, const double* X, const int* is_ee, const double* w, const double* eps,
                     double dhat, double* E, double* g, double* H, int project, cudaStream_t s) {
  if (n <= 0) return 0;
  k_elem_barrier<<<nblk(n, 64), 64, 0, s>>>(n, X, is_ee, w, eps, dhat, E, g, H, project);
  return 1;
}
int launch_k_accd(int n, const double* X0, const double* P, const int* is_ee, double sfrac, int max_iter,
                  double* toi, int* iters, cudaStream_t s) {
  if (n <= 0) return 0;
  k_elem_accd<<<nblk(n, 128), 128, 0, s>>>(n, X0, P, is_ee, sfrac, max_iter, toi, iters);
  return 1;
}

}  // namespace ipc
