// PCG vectors z (preconditioned residual), d (search direction) and q
// (= A d) per row: FP64 rows (Dev::z, d / db, q) in FP64 mode, 16-byte FP32
// rows (Dev::z4, d4 / d4b, q4) in mixed mode, where the matrix and its
// mat-vec are FP32 too.  The residual r, the Newton direction p, the dot
// products and the step lengths alpha / beta stay FP64 in both modes.
//
// The direction is double-buffered (buffer 0: d / d4, buffer 1: db / d4b).
// PCG iteration k (Dev::pcg_ctl[1]) reads d_{k-1} from buffer k % 2 and
// writes d_k = z_k + beta_k d_{k-1} into buffer (k + 1) % 2, so that the
// mat-vec can form d_k of its neighbours on the fly while it writes its own.
#pragma once

#include "common.cuh"
#include "ctx.h"

namespace ipc {

template <class HT> struct PV;

// a row of three doubles through L2 only
__device__ __forceinline__ D3 ld3cg(const double* p, int i) {
  return D3{__ldcg(p + 3 * i), __ldcg(p + 3 * i + 1), __ldcg(p + 3 * i + 2)};
}

template <> struct PV<double> {
  static __device__ __forceinline__ double* dbuf(const Dev& d, int b) { return b ? d.db : d.d; }
  static __device__ __forceinline__ D3 z(const Dev& d, int r) { return ld3(d.z, r); }
  static __device__ __forceinline__ void set_z(const Dev& d, int r, D3 v) { st3(d.z, r, v); }
  static __device__ __forceinline__ D3 dir(const Dev& d, int r, int b) { return ld3(dbuf(d, b), r); }
  static __device__ __forceinline__ void set_dir(const Dev& d, int r, int b, D3 v) { st3(dbuf(d, b), r, v); }
  static __device__ __forceinline__ D3 q(const Dev& d, int r) { return ld3(d.q, r); }
  static __device__ __forceinline__ void set_q(const Dev& d, int r, D3 v) { st3(d.q, r, v); }
  // z and the previous direction of column c as the mat-vec gathers them
  // (CG: through L2 only, for rows that other CTAs of the same launch wrote)
  template <bool CG = false>
  static __device__ __forceinline__ V3<double> gather_z(const Dev& d, int c) {
    if constexpr (CG) return ld3cg(d.z, c);
    return ld3(d.z, c);
  }
  template <bool CG = false>
  static __device__ __forceinline__ V3<double> gather_dir(const Dev& d, int c, int b) {
    if constexpr (CG) return ld3cg(dbuf(d, b), c);
    return ld3(dbuf(d, b), c);
  }
};

template <> struct PV<float> {
  static __device__ __forceinline__ float4* dbuf(const Dev& d, int b) { return b ? d.d4b : d.d4; }
  static __device__ __forceinline__ D3 f4(float4 v) { return D3{v.x, v.y, v.z}; }
  static __device__ __forceinline__ float4 to4(D3 v) {
    return make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f);
  }
  static __device__ __forceinline__ D3 z(const Dev& d, int r) { return f4(d.z4[r]); }
  static __device__ __forceinline__ void set_z(const Dev& d, int r, D3 v) { d.z4[r] = to4(v); }
  static __device__ __forceinline__ D3 dir(const Dev& d, int r, int b) { return f4(dbuf(d, b)[r]); }
  static __device__ __forceinline__ void set_dir(const Dev& d, int r, int b, D3 v) { dbuf(d, b)[r] = to4(v); }
  static __device__ __forceinline__ D3 q(const Dev& d, int r) { return f4(d.q4[r]); }
  static __device__ __forceinline__ void set_q(const Dev& d, int r, D3 v) { d.q4[r] = to4(v); }
  template <bool CG = false>
  static __device__ __forceinline__ V3<float> gather_z(const Dev& d, int c) {
    const float4 v = CG ? __ldcg(d.z4 + c) : __ldg(d.z4 + c);
    return V3<float>{v.x, v.y, v.z};
  }
  template <bool CG = false>
  static __device__ __forceinline__ V3<float> gather_dir(const Dev& d, int c, int b) {
    const float4 v = CG ? __ldcg(dbuf(d, b) + c) : __ldg(dbuf(d, b) + c);
    return V3<float>{v.x, v.y, v.z};
  }
};

// buffer that receives the direction of the current PCG iteration
__device__ __forceinline__ int pcg_new_buf(const Dev& d) { return (int)((*(volatile unsigned int*)(d.pcg_ctl + 1) + 1u) & 1u); }

// direction row with the precision decided at run time (kernels that are
// not templated on it)
__device__ __forceinline__ D3 dir_row(const Dev& d, int r, int b) {
  return d.prec ? PV<float>::dir(d, r, b) : PV<double>::dir(d, r, b);
}

// J w of a body point: the direction on the body's 4 sub-rows [p, a0, a1, a2]
__device__ __forceinline__ D3 dir_body_point(const Dev& d, int br, D3 xb, int b) {
  return dir_row(d, br, b) + xb.x * dir_row(d, br + 1, b) + xb.y * dir_row(d, br + 2, b) +
         xb.z * dir_row(d, br + 3, b);
}

// tag of the rows the contact terms of env e write in its current Newton iteration
__device__ __forceinline__ uint8_t touch_tag(const Dev& d, int e) {
  return (uint8_t)(1 + (d.env_i[e * NUM_INTS + I_GEN] % 255));
}

// Deterministic per-env reduction of CTA partials: every row CTA of the env
// writes `n` partials; the last CTA to arrive sums them in CTA order.
// cta: the row CTA (row / 128), which is not blockIdx.x when a kernel walks
// a list of CTAs.  Returns true in thread 0 of the last CTA, with the sums
// in out[0..n).  Every thread of the 128-thread CTA must call it.
// T0: type in which the first value (v0) is summed within the CTA (FP32 for
// the FP32 products r.z and d.q of mixed mode); the other n - 1 values are
// FP64, and the CTA partials are summed in FP64.
template <int n, class T0 = double>
__device__ bool env_reduce(const Dev& d, int e, int which, int cta, T0 v0, const double* rest /* n - 1 */,
                           double* out) {
  __shared__ double sh[128];
  __shared__ float shf[32];
  __shared__ bool last;
  double part[n];
  if constexpr (sizeof(T0) == 4) part[0] = (double)block_sum(v0, shf);
  else part[0] = block_sum128(v0, sh);
  for (int j = 1; j < n; ++j) part[j] = block_sum128(rest[j - 1], sh);
  if (threadIdx.x == 0) {
    for (int j = 0; j < n; ++j) d.cta_part[4 * cta + j] = part[j];
    __threadfence();
    unsigned int t = atomicAdd(&d.env_cnt[2 * e + which], 1u);
    int ncta = (d.env_row_off[e + 1] - d.env_row_off[e]) >> 7;
    last = (t == (unsigned)(ncta - 1));
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  int c0 = d.env_row_off[e] >> 7, c1 = d.env_row_off[e + 1] >> 7;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) s += __ldcg(d.cta_part + 4 * c + j);
    out[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) d.env_cnt[2 * e + which] = 0;
  return threadIdx.x == 0;
}

}  // namespace ipc
