// Block-Jacobi preconditioned conjugate gradients on H p = -g (K6), the
// step the paper names as its main cost (Limitations).
//
// Every form works over a device-side work list of the envs still
// iterating, in items: 128 consecutive rows of one env (one row per
// thread), a group of 8 active pairs (16 lanes per pair) or of 128 friction
// records (one per thread).  The per-item work is shared:
//   matvec_rows: d_k = z_k + beta_k d_{k-1} (formed on the fly, written to
//     the other direction buffer), q = A d_k over the SELL-32 matrix, d_k.q
//     summed per env by CTA partials;
//   matvec_pairs / matvec_fric: the contact and friction terms of d_k
//     (matrix-free, added to the accumulator qc) and their part of d_k.q;
//   update_rows: alpha = r.z / d.q, p += alpha d, r -= alpha q, z = P^-1 r,
//     r.z and r.r per env -> beta and the stop test.
// Three forms run them:
//   k_pcg_multi (the default): W iterations per persistent launch, each
//     env's items waiting only for its own earlier ones;
//   k_pcg_iter: one iteration per launch (inside rollout windows);
//   k_pcg_matvec + k_pcg_pairs (beside it) + k_fric_spmv, then
//     k_pcg_update (ipc_params.pcg_fused = 0).
// The grid's last CTA of each launch rebuilds the work list when stopped
// envs hold a quarter of its items and (inside a CUDA graph) sets the
// loop's condition, so the whole solve runs without the host.
#include "common.cuh"
#include "fpconv.cuh"
#include "kernels.h"
#include "pcgvec.cuh"

namespace ipc {

#define ENVI(d, e, k) (d).env_i[(e) * NUM_INTS + (k)]
#define ENVS(d, e, k) (d).env_s[(e) * NUM_SCALARS + (k)]

namespace {

// C_NEXT: next pair / mat-vec item of the fused kernel; C_ABORT: a wait
// gave up; C_RALLOC / C_RTAKE: slots of the ready update items allocated /
// taken; C_LIVEROWS: row items of the envs solving at the launch's start;
// C_STOPROWS: row items of the envs that stopped during the launch
enum PcgCtl {
  C_ARRIVED = 0, C_ITER, C_LEN, C_DEAD, C_LIVE, C_NEXT, C_ABORT, C_RALLOC, C_RTAKE, C_LIVEROWS, C_STOPROWS,
  C_COUNT
};

// component c of a 3-vector of either precision
template <class T>
__device__ __forceinline__ T comp3(V3<T> v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

__device__ __forceinline__ bool row_is_body(uint8_t k) { return k == ROW_BODY || k == ROW_BODY_DRIVEN; }


__device__ __forceinline__ int env_row_ctas(const Dev& d, int e) { return (d.env_row_off[e + 1] - d.env_row_off[e]) >> 7; }
__device__ __forceinline__ int env_active_pairs(const Dev& d, int e) { return min(ENVI(d, e, I_NACT), d.env_pair_cap[e]); }
// friction records of env e in PCG (records of this step; none without friction)
__device__ __forceinline__ int env_fric(const Dev& d, int e) {
  return d.fr_mu > 0.0 ? min(ENVI(d, e, I_NFRIC), d.env_pair_cap[e]) : 0;
}
// the fused kernels' product items of env e per iteration: row items, groups
// of 8 active pairs and (FR: the kernel variant for runs with friction)
// groups of 128 friction records
template <bool FR>
__device__ __forceinline__ int env_products(const Dev& d, int e) {
  if constexpr (FR) return env_row_ctas(d, e) + (env_active_pairs(d, e) + 7) / 8 + (env_fric(d, e) + 127) / 128;
  return env_row_ctas(d, e) + (env_active_pairs(d, e) + 7) / 8;
}

// Rebuild the work list from the envs' I_PCG flags (one CTA, blockDim a
// multiple of 32): list order is env order; per listed env the prefix of
// its 128-row items and of its groups of 8 active pairs.
__device__ void build_list(const Dev& d) {
  __shared__ int wsum[4][32];
  __shared__ int carry[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x < 4) carry[threadIdx.x] = 0;
  __syncthreads();
  for (int base = 0; base < d.n_envs; base += blockDim.x) {
    const int e = base + threadIdx.x;
    const bool on = e < d.n_envs && ENVI(d, e, I_PCG) != 0;
    int v[4];
    v[0] = on ? 1 : 0;
    v[1] = on ? env_row_ctas(d, e) : 0;
    v[2] = on ? (env_active_pairs(d, e) + 7) / 8 : 0;
    v[3] = on ? (env_fric(d, e) + 127) / 128 : 0;
    int inc[4];
    for (int k = 0; k < 4; ++k) {
      inc[k] = v[k];
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc[k], o);
        if (lane >= o) inc[k] += t;
      }
      if (lane == 31) wsum[k][wid] = inc[k];
    }
    __syncthreads();
    if (wid == 0)
      for (int k = 0; k < 4; ++k) {
        const int w = lane < nw ? wsum[k][lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, wi, o);
          if (lane >= o) wi += t;
        }
        wsum[k][lane] = wi - w;  // exclusive warp offsets
      }
    __syncthreads();
    int ex[4];
    for (int k = 0; k < 4; ++k) ex[k] = carry[k] + wsum[k][wid] + inc[k] - v[k];
    if (on) {
      d.pcg_list[ex[0]] = e;
      d.pcg_row_off[ex[0]] = ex[1];
      d.pcg_pair_off[ex[0]] = ex[2];
      d.pcg_fric_off[ex[0]] = ex[3];
      // per item its env and global row CTA / pair group, so that a kernel
      // finds its item with one load instead of a search over the list
      const int cta0 = d.env_row_off[e] >> 7;
      ENVI(d, e, I_LISTROW) = ex[1];
      ENVI(d, e, I_UPDK) = 0;
      for (int j = 0; j < v[1]; ++j) d.pcg_item[ex[1] + j] = make_int2(e, cta0 + j);
      for (int j = 0; j < v[2]; ++j) d.pcg_pitem[ex[2] + j] = make_int2(e, j);
      for (int j = 0; j < v[3]; ++j) d.pcg_fitem[ex[3] + j] = make_int2(e, j);
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1)
      for (int k = 0; k < 4; ++k) carry[k] = ex[k] + v[k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d.pcg_row_off[carry[0]] = carry[1];
    d.pcg_pair_off[carry[0]] = carry[2];
    d.pcg_fric_off[carry[0]] = carry[3];
    d.pcg_ctl[C_LEN] = carry[0];
    d.pcg_ctl[C_LIVE] = carry[0];
    d.pcg_ctl[C_DEAD] = 0;
    d.pcg_ctl[C_LIVEROWS] = carry[1];
    d.pcg_ctl[C_STOPROWS] = 0;
  }
  __syncthreads();
}

// ---- block-Jacobi preconditioner application
// z = P^{-1} r for row r.  Body rows read the 4 sub-rows of their body (all
// of them sit in the same warp) and apply the body's 12x12 inverse in FP64.
template <bool CG = false>
__device__ __forceinline__ D3 apply_pc_body(const Dev& d, int r) {
  const int b = d.row_body[r];
  const int br = d.body_row[b];
  const int kk = r - br;
  const double* Pi = d.body_pc + 144 * (long long)b;
  double o[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 12; ++j) o[i] += Pi[(3 * kk + i) * 12 + j] * (CG ? __ldcg(d.r + 3 * br + j) : d.r[3 * br + j]);
  return D3{o[0], o[1], o[2]};
}

// FP64 mode: gel rows apply the 6 stored entries of the symmetric 3x3 inverse
template <bool CG = false>
__device__ __forceinline__ D3 apply_pc64(const Dev& d, int r, uint8_t kr, D3 x) {
  if (row_is_body(kr)) return apply_pc_body<CG>(d, r);
  if (kr == ROW_PAD) return D3{0, 0, 0};
  const double* P = reinterpret_cast<const double*>(d.pc) + 6 * (long long)r;
  const double a = P[0], b = P[1], c = P[2], e = P[3], f = P[4], g = P[5];
  return D3{a * x.x + b * x.y + c * x.z, b * x.x + e * x.y + f * x.z, c * x.x + f * x.y + g * x.z};
}

// mixed mode: FP32 inverse applied to the FP32-rounded residual of the row
template <bool CG = false>
__device__ __forceinline__ float4 apply_pc32(const Dev& d, int r, uint8_t kr, float3 x) {
  if (row_is_body(kr)) {
    const D3 z = apply_pc_body<CG>(d, r);
    return make_float4(d2f_bits(z.x), d2f_bits(z.y), d2f_bits(z.z), 0.0f);
  }
  if (kr == ROW_PAD) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float* P = reinterpret_cast<const float*>(d.pc) + 6 * (long long)r;
  const float a = P[0], b = P[1], c = P[2], e = P[3], f = P[4], g = P[5];
  return make_float4(a * x.x + b * x.y + c * x.z, b * x.x + e * x.y + f * x.z, c * x.x + f * x.y + g * x.z, 0.0f);
}

__device__ __forceinline__ float3 round_row(D3 v) { return make_float3(d2f_bits(v.x), d2f_bits(v.y), d2f_bits(v.z)); }
__device__ __forceinline__ D3 widen_row(float4 v) { return D3{f2d_bits(v.x), f2d_bits(v.y), f2d_bits(v.z)}; }

// d_k of one row from z_k and d_{k-1}: the same fused operations wherever a
// row's direction is formed (its own row, a gathered column, a pair point)
__device__ __forceinline__ float dk32(float z, float b, float dold) { return __fmaf_rn(b, dold, z); }
__device__ __forceinline__ double dk64(double z, double b, double dold) { return __fma_rn(b, dold, z); }

// CG: z and d_{k-1} read through L2 (the multi-iteration kernel, where
// other CTAs of the same launch wrote them)
template <class HT> struct Dk;
template <> struct Dk<float> {
  template <bool CG = false>
  static __device__ __forceinline__ V3<float> row(const Dev& d, int c, float b, int ob) {
    const V3<float> z = PV<float>::gather_z<CG>(d, c), o = PV<float>::gather_dir<CG>(d, c, ob);
    return V3<float>{dk32(z.x, b, o.x), dk32(z.y, b, o.y), dk32(z.z, b, o.z)};
  }
};
template <> struct Dk<double> {
  template <bool CG = false>
  static __device__ __forceinline__ V3<double> row(const Dev& d, int c, double b, int ob) {
    const V3<double> z = PV<double>::gather_z<CG>(d, c), o = PV<double>::gather_dir<CG>(d, c, ob);
    return V3<double>{dk64(z.x, b, o.x), dk64(z.y, b, o.y), dk64(z.z, b, o.z)};
  }
};

// ---- mat-vec item: 128 rows of SELL-32, U slots in flight per lane
template <class HT, int U, bool CG = false>
__device__ __forceinline__ void matvec_rows(const Dev& d, int e, int cta, HT beta, int ob, int nb) {
  const int r = cta * 128 + threadIdx.x;
  const int ch = r >> 5, lane = r & 31;
  const int slots = d.chunk_slots[ch];
  const long long base = d.chunk_ptr[ch];
  const HT* __restrict__ val = reinterpret_cast<const HT*>(d.sell_val) + base * 9 + lane;
  const int* __restrict__ colp = d.sell_col + base + lane;
  HT ax = 0, ay = 0, az = 0;
  int sl = 0;
  // the column indices of the next group of U slots are loaded one group
  // ahead, so that a group's gathers go out together with its value loads
  // (one memory round trip per group instead of a column -> gather chain)
  int cn[U];
  if (U <= slots) {
#pragma unroll
    for (int u = 0; u < U; ++u) cn[u] = colp[u * 32];
  }
  for (; sl + U <= slots; sl += U) {
    int c[U];
    HT A[U][9];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = cn[u];
      if (!IPC_CHECK(d.check_word, (unsigned)c[u] < (unsigned)d.n_rows, CHK_SELL_COL, c[u])) c[u] = r;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < 9; ++k) A[u][k] = val[(long long)(sl + u) * 288 + k * 32];
    if (sl + 2 * U <= slots) {
#pragma unroll
      for (int u = 0; u < U; ++u) cn[u] = colp[(sl + U + u) * 32];
    }
    V3<HT> w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = Dk<HT>::template row<CG>(d, c[u], beta, ob);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ax += A[u][0] * w[u].x + A[u][1] * w[u].y + A[u][2] * w[u].z;
      ay += A[u][3] * w[u].x + A[u][4] * w[u].y + A[u][5] * w[u].z;
      az += A[u][6] * w[u].x + A[u][7] * w[u].y + A[u][8] * w[u].z;
    }
  }
  for (; sl < slots; ++sl) {
    int c = colp[sl * 32];
    if (!IPC_CHECK(d.check_word, (unsigned)c < (unsigned)d.n_rows, CHK_SELL_COL, c)) c = r;
    const HT* A = val + (long long)sl * 288;
    const V3<HT> w = Dk<HT>::template row<CG>(d, c, beta, ob);
    ax += A[0] * w.x + A[32] * w.y + A[64] * w.z;
    ay += A[96] * w.x + A[128] * w.y + A[160] * w.z;
    az += A[192] * w.x + A[224] * w.y + A[256] * w.z;
  }
  const V3<HT> own = Dk<HT>::template row<CG>(d, r, beta, ob);
  double out[1];
  bool last;
  if constexpr (sizeof(HT) == 4) {
    PV<float>::dbuf(d, nb)[r] = make_float4(own.x, own.y, own.z, 0.0f);
    d.q4[r] = make_float4(ax, ay, az, 0.0f);
    last = env_reduce<1, float>(d, e, 1, cta, own.x * ax + own.y * ay + own.z * az, nullptr, out);
  } else {
    st3(PV<double>::dbuf(d, nb), r, D3{own.x, own.y, own.z});
    st3(d.q, r, D3{ax, ay, az});
    last = env_reduce<1>(d, e, 1, cta, own.x * ax + own.y * ay + own.z * az, nullptr, out);
  }
  if (last) ENVS(d, e, S_DQ) = out[0];
}

// index of (p, q), p <= q, in the packed upper triangle of a 12x12 matrix
__device__ __forceinline__ int ut12(int p, int q) { return p * 12 - p * (p - 1) / 2 + (q - p); }

// ---- mat-vec item: contact terms of 8 active pairs of env e (group g)
// q_c += H_k d_k per pair (pinned gel rows are eliminated: read as zero,
// never written); sum_k d_k^T H_k d_k -> S_DQC.  H_k is stored as its
// packed upper triangle, interleaved by warp of slots.  16 lanes per pair:
// lane j < 12 owns coordinate j = 3 m + c (point m, component c); it forms
// that component of the pair's direction, the group shares the 12 values by
// shuffles, lane j computes row j of H_k d and scatters it: gel points
// directly, body points as J^T (H_k d) on the body's 4 sub-rows (merged with
// the warp's other pair when both touch the same single body).
template <class HT, bool CG = false>
__device__ __forceinline__ void matvec_pairs(const Dev& d, int e, int g, HT beta, int ob) {
  __shared__ double sdq[4];
  const int lane = threadIdx.x & 31, j = lane & 15, half = lane >> 4;
  const int m = j / 3, c = j - 3 * m;
  const int local = 8 * g + (threadIdx.x >> 4);
  const int i = d.env_pair_off[e] + local;       // slot of this half-warp's pair
  bool live = local < env_active_pairs(d, e) &&
              IPC_CHECK(d.check_word, (long long)i < d.n_pairs_cap, CHK_ACT_SLOT, i);
  int4 v = live ? d.act_v[i] : make_int4(0, 0, 0, 0);
  if (live && !IPC_CHECK(d.check_word, (unsigned)v.x < (unsigned)d.n_cv && (unsigned)v.y < (unsigned)d.n_cv &&
                         (unsigned)v.z < (unsigned)d.n_cv && (unsigned)v.w < (unsigned)d.n_cv, CHK_ACT_SLOT, i)) {
    live = false;
    v = make_int4(0, 0, 0, 0);
  }
  const int cv = m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w));
  int b_pt = -1, row = 0;
  double xb[3] = {0, 0, 0};
  HT dj = 0;
  if (live && j < 12) {
    row = d.cv_row[cv];
    b_pt = d.cv_body[cv];
    if (b_pt < 0) {
      dj = (d.row_kind[row] == ROW_PINNED) ? (HT)0 : comp3(Dk<HT>::template row<CG>(d, row, beta, ob), c);
    } else {
      const D3 x3 = ld3(d.cv_xbar, cv);
      xb[0] = x3.x; xb[1] = x3.y; xb[2] = x3.z;
      const HT d0 = comp3(Dk<HT>::template row<CG>(d, row, beta, ob), c),
               d1 = comp3(Dk<HT>::template row<CG>(d, row + 1, beta, ob), c),
               d2 = comp3(Dk<HT>::template row<CG>(d, row + 2, beta, ob), c),
               d3 = comp3(Dk<HT>::template row<CG>(d, row + 3, beta, ob), c);
      dj = (HT)((double)d0 + xb[0] * (double)d1 + xb[1] * (double)d2 + xb[2] * (double)d3);
    }
  }
  HT oj = 0;
  const HT* H = reinterpret_cast<const HT*>(d.pair_H) + (long long)(i >> 5) * 78 * 32 + (i & 31);
  for (int q = 0; q < 12; ++q) {
    const HT dq = __shfl_sync(0xffffffffu, dj, (lane & 16) + q);
    if (live && j < 12) {
      const int lo = min(j, q), hi = max(j, q);
      oj += H[ut12(lo, hi) * 32] * dq;
    }
  }
  // d_k^T H_k d_k of the CTA's pairs (all of env e): one atomic per CTA
  double part = (live && j < 12) ? (double)(dj * oj) : 0.0;
  part = warp_sum(part);
  if (lane == 0) sdq[threadIdx.x >> 5] = part;
  const double o = (double)oj;
  if (live && j < 12 && b_pt < 0 && d.row_kind[row] != ROW_PINNED) atomicAdd(d.qc + 3 * row + c, o);
  int bm[4];
  for (int mm = 0; mm < 4; ++mm) bm[mm] = __shfl_sync(0xffffffffu, b_pt, (lane & 16) + 3 * mm);
  int body = -2;
  for (int mm = 0; mm < 4; ++mm)
    if (bm[mm] >= 0) body = (body == -2 || body == bm[mm]) ? bm[mm] : -1;
  if (!live) body = -2;
  const int s4 = j / 3;
  double jb = 0.0;
  for (int mm = 0; mm < 4; ++mm) {
    const int src = (lane & 16) + 3 * mm;
    const double om = __shfl_sync(0xffffffffu, o, src + c);
    const double x0 = __shfl_sync(0xffffffffu, xb[0], src);
    const double x1 = __shfl_sync(0xffffffffu, xb[1], src);
    const double x2 = __shfl_sync(0xffffffffu, xb[2], src);
    const double xs = s4 == 0 ? 1.0 : (s4 == 1 ? x0 : (s4 == 2 ? x1 : x2));
    if (body >= 0 && bm[mm] == body) jb += xs * om;
  }
  const int other = __shfl_xor_sync(0xffffffffu, body, 16);
  const double jb_other = __shfl_xor_sync(0xffffffffu, jb, 16);
  if (body >= 0 && j < 12) {
    if (other == body) {
      if (half == 0) atomicAdd(d.qc + 3 * d.body_row[body] + j, jb + jb_other);
    } else {
      atomicAdd(d.qc + 3 * d.body_row[body] + j, jb);
    }
  }
  if (body == -1 && j < 12 && b_pt >= 0) {
    const int br = d.body_row[b_pt];
    atomicAdd(d.qc + 3 * br + c, o);
    for (int s = 0; s < 3; ++s) atomicAdd(d.qc + 3 * (br + 1 + s) + c, xb[s] * o);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(&ENVS(d, e, S_DQC), sdq[0] + sdq[1] + sdq[2] + sdq[3]);
  __syncthreads();
}

template <class HT>
__device__ __forceinline__ D3 widen3(V3<HT> v) { return D3{(double)v.x, (double)v.y, (double)v.z}; }

// ---- mat-vec item of the fused kernels: the lagged friction terms of 128
// records of env e (group g), one thread per record (Sec. 3.2, App. A.3):
// u = sum_i w_i d_k(point i), q_c += w_i S u per point, d_k.q part u.S.u.
// d_k of the points is formed on the fly from z_k and d_{k-1} (the same
// fused operation the mat-vec writes, so the same values the separate
// friction kernel reads from the new direction buffer).
template <class HT, bool CG = false>
__device__ __forceinline__ void matvec_fric(const Dev& d, int e, int g, HT beta, int ob) {
  __shared__ double sdq[32];
  const int local = 128 * g + threadIdx.x;
  double part = 0.0;
  if (local < env_fric(d, e)) {
    const int j = d.env_pair_off[e] + local;
    const int4 v = d.fr_v[j];
    const int cvs[4] = {v.x, v.y, v.z, v.w};
    const double* w = d.fr_w + 4 * (long long)j;
    D3 a{0, 0, 0};
    for (int i = 0; i < 4; ++i) {
      const int cv = cvs[i], row = d.cv_row[cv];
      D3 u;
      if (d.cv_body[cv] < 0) {
        u = (d.row_kind[row] == ROW_PINNED) ? D3{0, 0, 0} : widen3(Dk<HT>::template row<CG>(d, row, beta, ob));
      } else {
        const D3 xb = ld3(d.cv_xbar, cv);
        u = widen3(Dk<HT>::template row<CG>(d, row, beta, ob)) +
            xb.x * widen3(Dk<HT>::template row<CG>(d, row + 1, beta, ob)) +
            xb.y * widen3(Dk<HT>::template row<CG>(d, row + 2, beta, ob)) +
            xb.z * widen3(Dk<HT>::template row<CG>(d, row + 3, beta, ob));
      }
      a = a + w[i] * u;
    }
    const double* S = d.fr_S + 6 * (long long)j;
    const D3 t{S[0] * a.x + S[1] * a.y + S[2] * a.z, S[1] * a.x + S[3] * a.y + S[4] * a.z,
               S[2] * a.x + S[4] * a.y + S[5] * a.z};
    for (int i = 0; i < 4; ++i) {
      const int cv = cvs[i], row = d.cv_row[cv];
      const D3 gv = w[i] * t;
      if (d.cv_body[cv] < 0) {
        if (d.row_kind[row] != ROW_PINNED) atomic_add3(d.qc, row, gv);
      } else {
        const D3 xb = ld3(d.cv_xbar, cv);
        atomic_add3(d.qc, row, gv);
        atomic_add3(d.qc, row + 1, xb.x * gv);
        atomic_add3(d.qc, row + 2, xb.y * gv);
        atomic_add3(d.qc, row + 3, xb.z * gv);
      }
    }
    part = dot(a, t);
  }
  part = block_sum(part, sdq);
  if (threadIdx.x == 0) atomicAdd(&ENVS(d, e, S_DQC), part);
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// PCG start: p = 0, r = -g, z = P^-1 r, d_{-1} = 0, beta = 0; r.z, r.r
template <class HT>
__global__ void k_pcg_init(Dev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_NEWT)) return;
  const uint8_t kr = d.row_kind[r];
  const D3 rv = (kr == ROW_PINNED || kr == ROW_PAD) ? D3{0, 0, 0} : -1.0 * ld3(d.g, r);
  st3(d.r, r, rv);
  st3(d.p, r, D3{0, 0, 0});
  __syncwarp();
  const double rr = dot(rv, rv);
  double out[2];
  bool last;
  if constexpr (sizeof(HT) == 4) {
    const float3 rf = round_row(rv);
    const float4 z = apply_pc32(d, r, kr, rf);
    d.z4[r] = z;
    d.d4[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    last = env_reduce<2, float>(d, e, 0, r >> 7, rf.x * z.x + rf.y * z.y + rf.z * z.z, &rr, out);
  } else {
    const D3 z = apply_pc64(d, r, kr, rv);
    PV<double>::set_z(d, r, z);
    PV<double>::set_dir(d, r, 0, D3{0, 0, 0});
    last = env_reduce<2>(d, e, 0, r >> 7, dot(rv, z), &rr, out);
  }
  if (last) {
    ENVS(d, e, S_PBETA) = 0.0;
    ENVS(d, e, S_RZ) = out[0];
    ENVS(d, e, S_RR0) = out[1];
    ENVS(d, e, S_RR) = out[1];
    ENVS(d, e, S_DQC) = 0.0;
    ENVI(d, e, I_PCGIT) = 0;
    ENVI(d, e, I_PCG) = out[1] > 0.0 ? 1 : 0;
    ENVI(d, e, I_DEC) = out[1] > 0.0 ? 0 : 1;   // nothing to solve: the decision follows
  }
}

// work list of the envs whose I_PCG flag is set; iteration counter 0; sets
// the solve loop's condition when launched inside a graph
__global__ void k_pcg_begin(Dev d, cudaGraphConditionalHandle h, int use_cond) {
  if (threadIdx.x == 0) {
    d.pcg_ctl[C_ARRIVED] = 0;
    d.pcg_ctl[C_ITER] = 0;
    d.pcg_ctl[C_NEXT] = 0;
    d.pcg_ctl[C_ABORT] = 0;
    d.pcg_ctl[C_RALLOC] = 0;
    d.pcg_ctl[C_RTAKE] = 0;
  }
  build_list(d);
  if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(h, d.pcg_ctl[C_LIVE] > 0 ? 1u : 0u);
}


template <class HT, int U>
__global__ void __launch_bounds__(128) k_pcg_matvec(Dev d) {
  // the item's env, row CTA and beta, read by thread 0 and shared (keeps
  // the per-thread registers of the row loop at the kernel's occupancy)
  __shared__ int s_e, s_cta;
  __shared__ double s_beta;
  const int n_list = (int)d.pcg_ctl[C_LEN];
  const int n_items = d.pcg_row_off[n_list];
  const int nb = pcg_new_buf(d), ob = nb ^ 1;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    __syncthreads();  // the previous item is done with the shared item data
    if (threadIdx.x == 0) {
      const int2 it = d.pcg_item[item];                // (env, row CTA)
      const bool in = IPC_CHECK(d.check_word, (unsigned)it.x < (unsigned)d.n_envs &&
                                (unsigned)it.y < (unsigned)(d.n_rows >> 7), CHK_PCG_ITEM, item);
      s_e = in && ENVI(d, it.x, I_PCG) ? it.x : -1;    // stopped envs stay listed until a rebuild
      s_cta = it.y;
      s_beta = ENVS(d, it.x, S_PBETA);
    }
    __syncthreads();
    const int e = s_e;
    if (e < 0) continue;
    matvec_rows<HT, U>(d, e, s_cta, (HT)s_beta, ob, nb);
  }
}

// the contact terms of the listed envs' active pairs, beside the SELL
// mat-vec (both form d_k on the fly from z_k and d_{k-1})
template <class HT>
__global__ void __launch_bounds__(128) k_pcg_pairs(Dev d) {
  const int n_list = (int)d.pcg_ctl[C_LEN];
  const int n_items = d.pcg_pair_off[n_list];
  const int ob = pcg_new_buf(d) ^ 1;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int2 it = d.pcg_pitem[item];                 // (env, group of 8 active pairs)
    if (!IPC_CHECK(d.check_word, (unsigned)it.x < (unsigned)d.n_envs, CHK_PCG_ITEM, item)) continue;
    if (!ENVI(d, it.x, I_PCG)) continue;
    matvec_pairs<HT>(d, it.x, it.y, (HT)ENVS(d, it.x, S_PBETA), ob);
  }
}

// ---- update item: 128 rows of env e.  alpha = r.z / (d.q + its contact
// part), p += alpha d_k, r -= alpha q, z = P^-1 r, r.z and r.r of the env
// (its last CTA: beta, the stop test).  q, d_k, the contact accumulator
// and the env's d.q are read through L2: in the fused iteration kernel
// they were written by other CTAs of the same launch.
// MULTI: the multi-iteration kernel, where the previous iteration's p, r, z
// and the env's scalars were written by other CTAs of the same launch (read
// through L2; the env's last CTA then counts the iteration in I_UPDK, which
// the env's next products wait for).
template <class HT, bool MULTI = false>
__device__ __forceinline__ void update_rows(const Dev& d, int e, int cta, double dq, double al, uint8_t tag,
                                            int nb) {
  const int r = cta * 128 + threadIdx.x;
  const uint8_t kr = d.row_kind[r];
  // contact part of q on the rows this iteration's contact terms write
  D3 qcv{0, 0, 0};
  const bool touched = d.row_touch[r] == tag;
  if (touched) {
    qcv = D3{__ldcg(d.qc + 3 * r), __ldcg(d.qc + 3 * r + 1), __ldcg(d.qc + 3 * r + 2)};
    st3(d.qc, r, D3{0, 0, 0});
  }
  double out[2];
  bool last;
  if constexpr (sizeof(HT) == 4) {
    const float4 dd = __ldcg(PV<float>::dbuf(d, nb) + r), qq = __ldcg(d.q4 + r);
    st3(d.p, r, (MULTI ? ld3cg(d.p, r) : ld3(d.p, r)) + al * widen_row(dd));
    const D3 rv = (MULTI ? ld3cg(d.r, r) : ld3(d.r, r)) - al * (touched ? widen_row(qq) + qcv : widen_row(qq));
    st3(d.r, r, rv);
    __syncwarp();
    const double rr = dot(rv, rv);
    const float3 rf = round_row(rv);
    const float4 z = apply_pc32<MULTI>(d, r, kr, rf);
    d.z4[r] = z;
    last = env_reduce<2, float>(d, e, 0, cta, rf.x * z.x + rf.y * z.y + rf.z * z.z, &rr, out);
  } else {
    const double* db = PV<double>::dbuf(d, nb) + 3 * r;
    const double* qv = d.q + 3 * r;
    const D3 dd{__ldcg(db), __ldcg(db + 1), __ldcg(db + 2)}, qq{__ldcg(qv), __ldcg(qv + 1), __ldcg(qv + 2)};
    st3(d.p, r, (MULTI ? ld3cg(d.p, r) : ld3(d.p, r)) + al * dd);
    const D3 rv = (MULTI ? ld3cg(d.r, r) : ld3(d.r, r)) - al * (touched ? qq + qcv : qq);
    st3(d.r, r, rv);
    __syncwarp();
    const double rr = dot(rv, rv);
    const D3 z = apply_pc64<MULTI>(d, r, kr, rv);
    PV<double>::set_z(d, r, z);
    last = env_reduce<2>(d, e, 0, cta, dot(rv, z), &rr, out);
  }
  if (last) {
    const double rz_old = __ldcg(&ENVS(d, e, S_RZ));
    ENVS(d, e, S_PBETA) = rz_old > 0.0 ? out[0] / rz_old : 0.0;
    ENVS(d, e, S_RZ) = out[0];
    ENVS(d, e, S_RR) = out[1];
    ENVS(d, e, S_DQC) = 0.0;
    if constexpr (!MULTI) ENVI(d, e, I_PHASE) = 0;   // the multi kernel counts across its iterations
    const int it = atomicAdd(&ENVI(d, e, I_PCGIT), 1) + 1;
    atomicAdd(&ENVI(d, e, I_PCGTOT), 1);
    const double tol2 = d.pcg_tol * d.pcg_tol * ENVS(d, e, S_RR0);
    if (out[1] <= tol2 || it >= d.pcg_max || !(dq > 0.0)) {
      ENVI(d, e, I_PCG) = 0;
      ENVI(d, e, I_DEC) = 1;
      atomicAdd(d.pcg_ctl + C_DEAD, (unsigned)(env_row_ctas(d, e) + (env_active_pairs(d, e) + 7) / 8));
      atomicAdd(d.pcg_ctl + C_STOPROWS, (unsigned)env_row_ctas(d, e));
      atomicSub(d.pcg_ctl + C_LIVE, 1u);
    }
    if constexpr (MULTI) {
      __threadfence();
      atomicAdd(&ENVI(d, e, I_UPDK), 1);
    }
  }
}

// thread 0: the update item's env (-1: skip), row CTA, d.q, alpha and row tag
__device__ __forceinline__ void update_item_info(const Dev& d, int item, int* s_e, int* s_cta, double* s_dq,
                                                 double* s_al, uint8_t* s_tag) {
  int2 iv = d.pcg_item[item];                        // (env, row CTA)
  const bool in = IPC_CHECK(d.check_word, (unsigned)iv.x < (unsigned)d.n_envs &&
                            (unsigned)iv.y < (unsigned)(d.n_rows >> 7), CHK_PCG_ITEM, item);
  if (!in) iv = make_int2(0, 0);
  const int e = iv.x;
  *s_e = in && ENVI(d, e, I_PCG) ? e : -1;           // stopped envs stay listed until a rebuild
  *s_cta = iv.y;
  const double dq = __ldcg(&ENVS(d, e, S_DQ)) + __ldcg(&ENVS(d, e, S_DQC));
  *s_dq = dq;
  *s_al = dq > 0.0 ? ENVS(d, e, S_RZ) / dq : 0.0;    // alpha, once per item
  *s_tag = touch_tag(d, e);
}

// the grid's last CTA after an iteration: next iteration, list upkeep,
// loop condition.  Every CTA of the grid calls it once, after its items.
// iters: PCG iterations the launch ran; multi: the multi-iteration kernel
// (its per-env iteration and product counts are reset for the next launch)
__device__ void pcg_iteration_end(const Dev& d, cudaGraphConditionalHandle h, int use_cond, unsigned window,
                                  unsigned iters = 1u, bool multi = false) {
  __shared__ bool s_last;
  __shared__ bool s_rebuild;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(d.pcg_ctl + C_ARRIVED, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    d.pcg_ctl[C_ARRIVED] = 0;
    d.pcg_ctl[C_NEXT] = 0;
    d.pcg_ctl[C_RALLOC] = 0;
    d.pcg_ctl[C_RTAKE] = 0;
    d.pcg_ctl[C_LIVEROWS] -= d.pcg_ctl[C_STOPROWS];
    d.pcg_ctl[C_STOPROWS] = 0;
    d.pcg_ctl[C_ITER] += iters;
    d.step_ctl[4] += 1u;   // PCG launches
    const unsigned len = d.pcg_ctl[C_LEN];
    const unsigned dead = d.pcg_ctl[C_DEAD];
    const unsigned items = len ? (unsigned)(d.pcg_row_off[len] + d.pcg_pair_off[len]) : 0u;
    s_rebuild = dead > 0 && 4u * dead >= items;
  }
  __syncthreads();
  if (multi) {
    const int n_list = (int)d.pcg_ctl[C_LEN];
    for (int i = threadIdx.x; i < n_list; i += blockDim.x) {
      const int e = d.pcg_list[i];
      ENVI(d, e, I_PHASE) = 0;
      ENVI(d, e, I_UPDK) = 0;
    }
    __syncthreads();
  }
  if (d.pcg_ctl[C_ABORT]) {
    // a wait of the fused kernel gave up (never expected): the envs still
    // solving end their step with IPC_ECUDA, their reductions and the
    // ready slots reset
    const int n_list = (int)d.pcg_ctl[C_LEN];
    for (int i = threadIdx.x; i < (d.n_rows >> 7); i += blockDim.x) d.pcg_ritem[i] = -1;
    for (int i = threadIdx.x; i < n_list; i += blockDim.x) {
      const int e = d.pcg_list[i];
      if (!ENVI(d, e, I_PCG)) continue;
      ENVI(d, e, I_PCG) = 0;
      ENVI(d, e, I_ACTIVE) = 0;
      ENVI(d, e, I_STATUS) = IPC_ECUDA;
      ENVI(d, e, I_PHASE) = 0;
      d.env_cnt[2 * e] = 0;
      d.env_cnt[2 * e + 1] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      d.pcg_ctl[C_ABORT] = 0;
      d.pcg_ctl[C_LIVE] = 0;
      d.pcg_ctl[C_DEAD] = 0;
      d.pcg_ctl[C_LEN] = 0;
      d.pcg_ctl[C_LIVEROWS] = 0;
    }
    __syncthreads();
  } else if (s_rebuild) {
    build_list(d);
  }
  if (threadIdx.x == 0 && use_cond) {
    // window: iterations of this solve loop (solves still running carry
    // over to the next one; the direction buffers alternate by iteration,
    // so an even window leaves a carried solve's d_{k-1} in buffer 0,
    // where the next loop's first iteration reads it)
    const bool more = d.pcg_ctl[C_LIVE] > 0 && d.pcg_ctl[C_ITER] <= (unsigned)d.pcg_max + 1u &&
                      d.pcg_ctl[C_ITER] < window;
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

template <class HT>
__global__ void __launch_bounds__(128) k_pcg_update(Dev d, cudaGraphConditionalHandle h, int use_cond,
                                                     unsigned window) {
  const int n_list = (int)d.pcg_ctl[C_LEN];
  const int n_items = d.pcg_row_off[n_list];
  const int nb = pcg_new_buf(d);
  __shared__ double s_dq, s_al;
  __shared__ int s_e, s_cta;
  __shared__ uint8_t s_tag;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    __syncthreads();  // the previous item is done with the shared item data
    if (threadIdx.x == 0) update_item_info(d, item, &s_e, &s_cta, &s_dq, &s_al, &s_tag);
    __syncthreads();
    if (s_e < 0) continue;
    update_rows<HT>(d, s_e, s_cta, s_dq, s_al, s_tag, nb);
  }
  pcg_iteration_end(d, h, use_cond, window);
}

// ---- the fused PCG iteration: contact terms, SELL mat-vec and update of
// every listed env in one persistent launch.  CTAs first take the pair
// groups and then the mat-vec row items in order from a device counter
// (C_NEXT).  Each of these items ends with a fence and an increment of its
// env's I_PHASE; the CTA that completes the count publishes the env's
// update row items into the ready slots (pcg_ritem, allocated by C_RALLOC).
// CTAs that find the pair and mat-vec items all taken take ready slots in
// order (C_RTAKE) up to the row items of the envs solving (C_LIVEROWS), so
// an update item starts when its own env is ready, in the order the envs
// become ready (no item waits behind another env's).  A CTA waits only for
// its slot to be written: when it waits, every pair and mat-vec item has
// been taken by a running CTA that waits on nothing, so every solving env
// publishes and every slot below C_LIVEROWS is written.  The wait is
// bounded all the same: after kWaitCycles (about a second) the CTA raises
// C_ABORT, the other waits give up at once, and the grid's last CTA ends
// the envs still solving with IPC_ECUDA.
constexpr long long kWaitCycles = 2000000000ll;

// end of a pair or mat-vec item of env e (every thread calls it); rq: the
// ready-slot order (the env's last product publishes its update items)
template <bool FR>
__device__ __forceinline__ void phase_signal(const Dev& d, int e, bool rq) {
  __shared__ int s_pub;
  __threadfence();   // every thread: its stores and atomics of the item before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    const int need = env_products<FR>(d, e);
    const int old = atomicAdd(&ENVI(d, e, I_PHASE), 1);
    s_pub = rq && old == need - 1 ? (int)atomicAdd(d.pcg_ctl + C_RALLOC, (unsigned)env_row_ctas(d, e)) : -1;
  }
  __syncthreads();
  const int base = s_pub;
  if (base >= 0) {
    // the env's last product: its update row items become ready
    const int n = env_row_ctas(d, e), first = ENVI(d, e, I_LISTROW);
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      if (IPC_CHECK(d.check_word, (unsigned)(base + j) < (unsigned)(d.n_rows >> 7), CHK_PCG_ITEM, base + j))
        atomicExch(d.pcg_ritem + base + j, first + j);
  }
}

// thread 0, env order: waits until env e's pair and mat-vec items are
// done (they were taken before this update item by running CTAs that wait
// on nothing); false on abort
template <bool FR>
__device__ __forceinline__ bool phase_wait(const Dev& d, int e) {
  const int need = env_products<FR>(d, e);
  volatile int* ph = &ENVI(d, e, I_PHASE);
  volatile unsigned* ab = d.pcg_ctl + C_ABORT;
  if (*ph < need) {
    const long long t0 = clock64();
    while (*ph < need) {
      if (*ab) return false;
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(d.pcg_ctl + C_ABORT, 1u);
        return false;
      }
      __nanosleep(100);
    }
  }
  __threadfence();
  return true;
}

// thread 0, ready-slot order: the next ready update item (its index in the
// row item table), -1 when none is left or on abort
__device__ __forceinline__ int take_ready(const Dev& d, unsigned n_upd) {
  const unsigned t = atomicAdd(d.pcg_ctl + C_RTAKE, 1u);
  if (t >= n_upd) return -1;
  volatile int* slot = d.pcg_ritem + t;
  volatile unsigned* ab = d.pcg_ctl + C_ABORT;
  int v = *slot;
  if (v < 0) {
    const long long t0 = clock64();
    while ((v = *slot) < 0) {
      if (*ab) return -1;
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(d.pcg_ctl + C_ABORT, 1u);
        return -1;
      }
      __nanosleep(100);
    }
  }
  *slot = -1;  // the slot is free for the next launch
  __threadfence();
  return v;
}

// B = 1 bounds the registers so that the mat-vec items keep the separate
// mat-vec kernel's occupancy (12 CTAs per SM in FP32, 6 in FP64; the pair
// path spills a few words), B = 0 gives the pair path its registers (9
// CTAs per SM in FP32, 5 in FP64); ipc_autotune picks one.  FR: the
// variant for runs with friction (friction record groups among the
// products).
template <class HT, int U, int B, bool FR>
__global__ void __launch_bounds__(128, sizeof(HT) == 4 ? (B ? 12 : 9) : (B ? 6 : 5))
    k_pcg_iter(Dev d, cudaGraphConditionalHandle h, int use_cond, unsigned window) {
  __shared__ int s_item, s_e, s_cta;
  __shared__ double s_beta, s_dq, s_al;
  __shared__ uint8_t s_tag;
  const int n_list = (int)d.pcg_ctl[C_LEN];
  const int n_rows = d.pcg_row_off[n_list];
  const int n_pairs = d.pcg_pair_off[n_list];
  const int n_fric = FR ? d.pcg_fric_off[n_list] : 0;
  const int n_pf = n_pairs + n_fric;                 // pair groups, then friction groups, then rows
  const int n_a = n_pf + n_rows;
  const unsigned n_upd = d.pcg_ctl[C_LIVEROWS];
  const bool rq = d.pcg_fused == 1;    // 1: ready-slot order, 2: env order
  const int nb = pcg_new_buf(d), ob = nb ^ 1;
  bool products_left = true;
  for (;;) {
    __syncthreads();  // the previous item is done with the shared item data
    if (threadIdx.x == 0) {
      int it = n_a;
      if (products_left || !rq) it = (int)atomicAdd(d.pcg_ctl + C_NEXT, 1u);
      if (rq) {
        if (it >= n_a) {
          const int v = take_ready(d, n_upd);
          it = v < 0 ? -1 : n_a + v;
        }
      } else if (it >= n_a + n_rows) {
        it = -1;
      } else if (it >= n_a) {
        // env order: the update item waits for its own env's products
        update_item_info(d, it - n_a, &s_e, &s_cta, &s_dq, &s_al, &s_tag);
        if (s_e >= 0) {
          if (phase_wait<FR>(d, s_e)) {
            const double dq = __ldcg(&ENVS(d, s_e, S_DQ)) + __ldcg(&ENVS(d, s_e, S_DQC));
            s_dq = dq;
            s_al = dq > 0.0 ? ENVS(d, s_e, S_RZ) / dq : 0.0;
          } else {
            s_e = -1;
          }
        }
      }
      s_item = it;
    }
    __syncthreads();
    const int item = s_item;
    if (item < 0) break;
    if (item < n_pairs) {
      const int2 it = d.pcg_pitem[item];               // (env, group of 8 active pairs)
      if (!IPC_CHECK(d.check_word, (unsigned)it.x < (unsigned)d.n_envs, CHK_PCG_ITEM, item)) continue;
      if (!ENVI(d, it.x, I_PCG)) continue;
      matvec_pairs<HT>(d, it.x, it.y, (HT)ENVS(d, it.x, S_PBETA), ob);
      phase_signal<FR>(d, it.x, rq);
    } else if (item < n_pf) {
      if constexpr (FR) {
        const int2 it = d.pcg_fitem[item - n_pairs];   // (env, group of 128 friction records)
        if (!IPC_CHECK(d.check_word, (unsigned)it.x < (unsigned)d.n_envs, CHK_PCG_ITEM, item)) continue;
        if (!ENVI(d, it.x, I_PCG)) continue;
        matvec_fric<HT>(d, it.x, it.y, (HT)ENVS(d, it.x, S_PBETA), ob);
        phase_signal<FR>(d, it.x, rq);
      }
    } else if (item < n_a) {
      if (threadIdx.x == 0) {
        const int2 it = d.pcg_item[item - n_pf];       // (env, row CTA)
        const bool in = IPC_CHECK(d.check_word, (unsigned)it.x < (unsigned)d.n_envs &&
                                  (unsigned)it.y < (unsigned)(d.n_rows >> 7), CHK_PCG_ITEM, item);
        s_e = in && ENVI(d, it.x, I_PCG) ? it.x : -1;
        s_cta = it.y;
        s_beta = ENVS(d, it.x, S_PBETA);
      }
      __syncthreads();
      const int e = s_e;
      if (e < 0) continue;
      matvec_rows<HT, U>(d, e, s_cta, (HT)s_beta, ob, nb);
      phase_signal<FR>(d, e, rq);
    } else {
      products_left = false;
      // an update item whose env's products are all in (ready slot; in env
      // order thread 0 has waited above)
      if (rq) {
        if (threadIdx.x == 0) update_item_info(d, item - n_a, &s_e, &s_cta, &s_dq, &s_al, &s_tag);
        __syncthreads();
      }
      if (s_e < 0) continue;
      update_rows<HT>(d, s_e, s_cta, s_dq, s_al, s_tag, nb);
    }
  }
  pcg_iteration_end(d, h, use_cond, window);
}

// ---- several PCG iterations in one launch (ipc_params.pcg_iters_per_launch
// = W > 1, no rollout window): the per-env dataflow of k_pcg_iter carried
// across iterations, so that envs do not line up on iteration boundaries.
// Items are W rounds of [pair groups, mat-vec row items, update row items],
// each env after env, taken in order from C_NEXT.  Env e's products of
// iteration k wait until its update of iteration k - 1 is done (I_UPDK >= k,
// counted by the env's last update CTA after a fence); its update items of
// iteration k wait until its products of rounds 0..k are in (I_PHASE >=
// (k + 1) x its pair groups and row items; I_PHASE counts across the
// launch).  Every wait is on items with smaller indices, taken by running
// CTAs, so every wait ends; an env that stops ends the waits of its later
// items (they see I_PCG = 0 and skip).  Within the launch z, the direction
// buffers, p, r and the env's scalars are written by other CTAs and read
// again, so these reads go through L2 (the CG / MULTI forms of the shared
// device functions).  Waits are bounded as in k_pcg_iter.
__device__ __forceinline__ bool multi_wait(const Dev& d, int e, int which, int need) {
  volatile int* pcg = &ENVI(d, e, I_PCG);
  volatile int* cnt = &ENVI(d, e, which);
  volatile unsigned* ab = d.pcg_ctl + C_ABORT;
  if (!*pcg) return false;
  if (*cnt < need) {
    const long long t0 = clock64();
    while (*cnt < need) {
      if (!*pcg || *ab) return false;
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(d.pcg_ctl + C_ABORT, 1u);
        return false;
      }
      __nanosleep(100);
    }
  }
  __threadfence();
  return *pcg != 0;   // an env that stopped in the iteration waited for skips
}

template <class HT, int U, bool FR>
__global__ void __launch_bounds__(128, sizeof(HT) == 4 ? 12 : 6)
    k_pcg_multi(Dev d, cudaGraphConditionalHandle h, int use_cond, unsigned window, int W) {
  __shared__ int s_kind, s_e, s_cta, s_nb;
  __shared__ double s_beta, s_dq, s_al;
  __shared__ uint8_t s_tag;
  const int n_list = (int)d.pcg_ctl[C_LEN];
  const int n_rows = d.pcg_row_off[n_list];
  const int n_pairs = d.pcg_pair_off[n_list];
  const int n_fric = FR ? d.pcg_fric_off[n_list] : 0;
  const int n_pf = n_pairs + n_fric;
  const int per = n_pf + 2 * n_rows;                 // a round: pairs, friction, rows, updates
  const unsigned n_total = (unsigned)W * (unsigned)per;
  const unsigned it0 = d.pcg_ctl[C_ITER];
  enum { K_PAIRS = 0, K_FRIC, K_ROWS, K_UPDATE, K_SKIP };
  for (;;) {
    __syncthreads();  // the previous item is done with the shared item data
    if (threadIdx.x == 0) {
      const unsigned it = atomicAdd(d.pcg_ctl + C_NEXT, 1u);
      int kind = -1;
      if (it < n_total) {
        const int k = (int)(it / (unsigned)per), j = (int)(it % (unsigned)per);
        s_nb = (int)((it0 + (unsigned)k + 1u) & 1u);
        int2 iv;
        if (j < n_pairs) {
          iv = d.pcg_pitem[j];                         // (env, group of 8 active pairs)
          kind = K_PAIRS;
        } else if (j < n_pf) {
          iv = d.pcg_fitem[j - n_pairs];               // (env, group of 128 friction records)
          kind = K_FRIC;
        } else {
          iv = d.pcg_item[j < n_pf + n_rows ? j - n_pf : j - n_pf - n_rows];   // (env, row CTA)
          kind = j < n_pf + n_rows ? K_ROWS : K_UPDATE;
        }
        if (!IPC_CHECK(d.check_word, (unsigned)iv.x < (unsigned)d.n_envs, CHK_PCG_ITEM, (long long)it)) {
          kind = K_SKIP;
        } else {
          const int e = iv.x;
          s_e = e;
          s_cta = iv.y;
          const bool product = kind != K_UPDATE;
          if (!multi_wait(d, e, product ? I_UPDK : I_PHASE, product ? k : (k + 1) * env_products<FR>(d, e))) {
            kind = K_SKIP;                             // the env stopped (or a wait gave up)
          } else if (product) {
            s_beta = __ldcg(&ENVS(d, e, S_PBETA));
          } else {
            const double dq = __ldcg(&ENVS(d, e, S_DQ)) + __ldcg(&ENVS(d, e, S_DQC));
            s_dq = dq;
            s_al = dq > 0.0 ? __ldcg(&ENVS(d, e, S_RZ)) / dq : 0.0;
            s_tag = touch_tag(d, e);
          }
        }
      }
      s_kind = kind;
    }
    __syncthreads();
    const int kind = s_kind;
    if (kind < 0) break;
    if (kind == K_SKIP) continue;
    const int e = s_e, nb = s_nb, ob = nb ^ 1;
    if (kind == K_PAIRS) {
      matvec_pairs<HT, true>(d, e, s_cta, (HT)s_beta, ob);
      phase_signal<FR>(d, e, false);
    } else if (kind == K_FRIC) {
      if constexpr (FR) {
        matvec_fric<HT, true>(d, e, s_cta, (HT)s_beta, ob);
        phase_signal<FR>(d, e, false);
      }
    } else if (kind == K_ROWS) {
      matvec_rows<HT, U, true>(d, e, s_cta, (HT)s_beta, ob, nb);
      phase_signal<FR>(d, e, false);
    } else {
      update_rows<HT, true>(d, e, s_cta, s_dq, s_al, s_tag, nb);
    }
  }
  pcg_iteration_end(d, h, use_cond, window, (unsigned)W, true);
}

// diagnostics: env e's count of completed update rounds set to v (-1: its
// first products wait for a round that nothing completes, so the bounded
// waits of the multi-iteration kernel run out)
__global__ void k_debug_set_updk(Dev d, int e, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ENVI(d, e, I_UPDK) = v;
}

// diagnostics: the direction v (FP64 rows staged in Dev::z) as z with
// beta = 0 and d_{-1} = 0, so that one mat-vec item computes H v
template <class HT>
__global__ void k_debug_dir_from_rows(Dev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_PCG)) return;
  const D3 v = ld3(d.z, r);
  PV<HT>::set_z(d, r, v);
  PV<HT>::set_dir(d, r, 0, D3{0, 0, 0});
  if (r == d.env_row_off[e]) {
    ENVS(d, e, S_PBETA) = 0.0;
    ENVS(d, e, S_DQC) = 0.0;
  }
}
// q = A v + contact part back to FP64 rows in Dev::q; qc cleared
template <class HT>
__global__ void k_debug_q_to_rows(Dev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = d.cta_env[r >> 7];
  if (!ENVI(d, e, I_PCG)) return;
  D3 q = PV<HT>::q(d, r);
  if (d.row_touch[r] == touch_tag(d, e)) {
    q = q + ld3(d.qc, r);
    st3(d.qc, r, D3{0, 0, 0});
  }
  st3(d.q, r, q);
}

// ---------------------------------------------------------------------------
// launchers

int launch_pcg_init(const Dev& d, cudaStream_t s) {
  if (d.prec) k_pcg_init<float><<<d.n_rows / 128, 128, 0, s>>>(d);
  else k_pcg_init<double><<<d.n_rows / 128, 128, 0, s>>>(d);
  return 1;
}
int launch_pcg_begin(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  k_pcg_begin<<<1, 1024, 0, s>>>(d, h, use_cond);
  return 1;
}
int launch_pcg_matvec(const Dev& d, cudaStream_t s) {
  const int u = d.spmv_unroll ? d.spmv_unroll : 2;
  const int g = d.pcg_grid;
  if (d.prec) {
    if (u == 2) k_pcg_matvec<float, 2><<<g, 128, 0, s>>>(d);
    else if (u == 8) k_pcg_matvec<float, 8><<<g, 128, 0, s>>>(d);
    else k_pcg_matvec<float, 4><<<g, 128, 0, s>>>(d);
  } else {
    if (u == 4) k_pcg_matvec<double, 4><<<g, 128, 0, s>>>(d);
    else if (u == 8) k_pcg_matvec<double, 8><<<g, 128, 0, s>>>(d);
    else k_pcg_matvec<double, 2><<<g, 128, 0, s>>>(d);
  }
  return 1;
}
int launch_pcg_pairs(const Dev& d, cudaStream_t s) {
  if (d.prec) k_pcg_pairs<float><<<d.pcg_grid_pairs, 128, 0, s>>>(d);
  else k_pcg_pairs<double><<<d.pcg_grid_pairs, 128, 0, s>>>(d);
  return 1;
}
int launch_pcg_update(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond, unsigned window) {
  if (d.prec) k_pcg_update<float><<<d.pcg_grid, 128, 0, s>>>(d, h, use_cond, window);
  else k_pcg_update<double><<<d.pcg_grid, 128, 0, s>>>(d, h, use_cond, window);
  return 1;
}
int launch_debug_dir_from_rows(const Dev& d, cudaStream_t s) {
  if (d.prec) k_debug_dir_from_rows<float><<<d.n_rows / 128, 128, 0, s>>>(d);
  else k_debug_dir_from_rows<double><<<d.n_rows / 128, 128, 0, s>>>(d);
  return 1;
}
int launch_debug_q_to_rows(const Dev& d, cudaStream_t s) {
  if (d.prec) k_debug_q_to_rows<float><<<d.n_rows / 128, 128, 0, s>>>(d);
  else k_debug_q_to_rows<double><<<d.n_rows / 128, 128, 0, s>>>(d);
  return 1;
}

// resident CTAs per SM of the persistent PCG kernels (the smaller of the two)
// the fused kernels' variants: slots in flight 2 or 4 (an 8-slot choice of
// the mat-vec runs the fused kernels with 4), register bound on or off
// (single-iteration kernel), friction items or none (runs with friction)
template <class HT, bool FR>
static const void* pcg_iter_fn_t(bool u4, int bound) {
  if (bound) return u4 ? (const void*)k_pcg_iter<HT, 4, 1, FR> : (const void*)k_pcg_iter<HT, 2, 1, FR>;
  return u4 ? (const void*)k_pcg_iter<HT, 4, 0, FR> : (const void*)k_pcg_iter<HT, 2, 0, FR>;
}
template <class HT, bool FR>
static const void* pcg_multi_fn_t(bool u4) {
  return u4 ? (const void*)k_pcg_multi<HT, 4, FR> : (const void*)k_pcg_multi<HT, 2, FR>;
}
static bool unroll4(int unroll) { return unroll == 4 || unroll == 8; }

template <class HT, bool FR>
static void launch_iter_t(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                          unsigned window) {
  const bool u4 = unroll4(d.spmv_unroll);
  if (pcg_iters_per_launch(d, window) > 1) {
    const int g = d.pcg_grid_multi, w = d.pcg_multi;
    if (u4) k_pcg_multi<HT, 4, FR><<<g, 128, 0, s>>>(d, h, use_cond, window, w);
    else k_pcg_multi<HT, 2, FR><<<g, 128, 0, s>>>(d, h, use_cond, window, w);
    return;
  }
  const int g = d.pcg_grid_fused;
  if (d.pcg_iter_bound) {
    if (u4) k_pcg_iter<HT, 4, 1, FR><<<g, 128, 0, s>>>(d, h, use_cond, window);
    else k_pcg_iter<HT, 2, 1, FR><<<g, 128, 0, s>>>(d, h, use_cond, window);
  } else {
    if (u4) k_pcg_iter<HT, 4, 0, FR><<<g, 128, 0, s>>>(d, h, use_cond, window);
    else k_pcg_iter<HT, 2, 0, FR><<<g, 128, 0, s>>>(d, h, use_cond, window);
  }
}

int launch_debug_set_updk(const Dev& d, int env, int v, cudaStream_t s) {
  k_debug_set_updk<<<1, 32, 0, s>>>(d, env, v);
  return 1;
}

int launch_pcg_iter(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond, unsigned window) {
  const bool fr = d.fr_mu > 0.0;
  if (d.prec) {
    if (fr) launch_iter_t<float, true>(d, s, h, use_cond, window);
    else launch_iter_t<float, false>(d, s, h, use_cond, window);
  } else {
    if (fr) launch_iter_t<double, true>(d, s, h, use_cond, window);
    else launch_iter_t<double, false>(d, s, h, use_cond, window);
  }
  return 1;
}

// PCG iterations one launch of the fused kernel runs: pcg_multi, or 1
// inside a rollout window (which counts single iterations)
int pcg_iters_per_launch(const Dev& d, unsigned window) {
  return (d.pcg_fused && d.pcg_multi > 1 && window == 0xffffffffu) ? d.pcg_multi : 1;
}

// resident CTAs per SM of the multi-iteration kernel (fr: the friction variant)
int pcg_multi_ctas_per_sm(int prec, int unroll, bool fr) {
  int a = 0;
  const bool u4 = unroll4(unroll);
  const void* f = prec ? (fr ? pcg_multi_fn_t<float, true>(u4) : pcg_multi_fn_t<float, false>(u4))
                       : (fr ? pcg_multi_fn_t<double, true>(u4) : pcg_multi_fn_t<double, false>(u4));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, f, 128, 0);
  return a > 0 ? a : 1;
}

// resident CTAs per SM of the single-iteration fused kernel
int pcg_iter_ctas_per_sm(int prec, int unroll, int bound, bool fr) {
  int a = 0;
  const bool u4 = unroll4(unroll);
  const void* f = prec ? (fr ? pcg_iter_fn_t<float, true>(u4, bound) : pcg_iter_fn_t<float, false>(u4, bound))
                       : (fr ? pcg_iter_fn_t<double, true>(u4, bound) : pcg_iter_fn_t<double, false>(u4, bound));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, f, 128, 0);
  return a > 0 ? a : 1;
}

int pcg_ctas_per_sm(int prec, int unroll) {
  int a = 0, b = 0;
  const int u = unroll ? unroll : 2;
  if (prec) {
    if (u == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<float, 2>, 128, 0);
    else if (u == 8) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<float, 8>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<float, 4>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_update<float>, 128, 0);
  } else {
    if (u == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<double, 4>, 128, 0);
    else if (u == 8) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<double, 8>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg_matvec<double, 2>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_update<double>, 128, 0);
  }
  const int m = a < b ? a : b;
  return m > 0 ? m : 1;
}

}  // namespace ipc
