// PCG vectors z (preconditioned residual), d (search direction) and q
// (= A d) per row: FP64 rows (Dev::z, d, q) in FP64 mode, 16-byte FP32 rows
// (Dev::z4, d4, q4) in mixed mode, where the matrix and its mat-vec are FP32
// too.  The residual r, the Newton direction p, the dot products and the
// step lengths alpha / beta stay FP64 in both modes.
#pragma once

#include "common.cuh"
#include "ctx.h"

namespace ipc {

template <class HT> struct PV;

template <> struct PV<double> {
  static __device__ __forceinline__ D3 z(const Dev& d, int r) { return ld3(d.z, r); }
  static __device__ __forceinline__ void set_z(const Dev& d, int r, D3 v) { st3(d.z, r, v); }
  static __device__ __forceinline__ D3 dir(const Dev& d, int r) { return ld3(d.d, r); }
  static __device__ __forceinline__ void set_dir(const Dev& d, int r, D3 v) { st3(d.d, r, v); }
  static __device__ __forceinline__ D3 q(const Dev& d, int r) { return ld3(d.q, r); }
  static __device__ __forceinline__ void set_q(const Dev& d, int r, D3 v) { st3(d.q, r, v); }
  // the direction of column c as the SpMV gathers it
  static __device__ __forceinline__ V3<double> gather(const Dev& d, int c) { return ld3(d.d, c); }
};

template <> struct PV<float> {
  static __device__ __forceinline__ D3 f4(float4 v) { return D3{v.x, v.y, v.z}; }
  static __device__ __forceinline__ float4 to4(D3 v) {
    return make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f);
  }
  static __device__ __forceinline__ D3 z(const Dev& d, int r) { return f4(d.z4[r]); }
  static __device__ __forceinline__ void set_z(const Dev& d, int r, D3 v) { d.z4[r] = to4(v); }
  static __device__ __forceinline__ D3 dir(const Dev& d, int r) { return f4(d.d4[r]); }
  static __device__ __forceinline__ void set_dir(const Dev& d, int r, D3 v) { d.d4[r] = to4(v); }
  static __device__ __forceinline__ D3 q(const Dev& d, int r) { return f4(d.q4[r]); }
  static __device__ __forceinline__ void set_q(const Dev& d, int r, D3 v) { d.q4[r] = to4(v); }
  static __device__ __forceinline__ V3<float> gather(const Dev& d, int c) {
    float4 v = __ldg(d.d4 + c);
    return V3<float>{v.x, v.y, v.z};
  }
};

// direction of one row with the precision decided at run time (kernels that
// are not templated on it)
__device__ __forceinline__ D3 dir_row(const Dev& d, int r) {
  return d.prec ? PV<float>::dir(d, r) : PV<double>::dir(d, r);
}

// J w of a body point: the direction on the body's 4 sub-rows [p, a0, a1, a2]
__device__ __forceinline__ D3 dir_body_point(const Dev& d, int br, D3 xb) {
  return dir_row(d, br) + xb.x * dir_row(d, br + 1) + xb.y * dir_row(d, br + 2) + xb.z * dir_row(d, br + 3);
}

}  // namespace ipc
