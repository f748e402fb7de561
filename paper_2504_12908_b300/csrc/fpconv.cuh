// FP32 <-> FP64 conversions built from the IEEE-754 binary32 / binary64 bit
// layouts with integer operations.
//
// B300 issues FP64 instructions, conversions to and from FP64 included, at a
// small fraction of its FP32 and integer rates.  The mixed-precision PCG row
// kernels keep z, d and q in FP32 and r, p in FP64, so every row converts
// several values per iteration; on the integer pipe those conversions no
// longer compete with the FP64 updates that must stay FP64.
//
// f2d_bits: exact for zeros, normal numbers, infinities and NaNs; FP32
//   subnormals (|x| < 2^-126) become a zero of the same sign.
// d2f_bits: rounds to the nearest FP32 value, ties away from zero (IEEE
//   rounds ties to even: the two differ only when the 29 dropped bits are
//   exactly 1000...0); results below 2^-126 in magnitude flush to a signed
//   zero, results above the FP32 range give infinity, NaN stays NaN.
//
// The header compiles as plain C++ too, so the host tests check it against
// the compiler's own conversions.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define IPC_FPC __host__ __device__ __forceinline__
#else
#define IPC_FPC inline
#endif

namespace ipc {

IPC_FPC uint32_t fpc_bits32(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
IPC_FPC float fpc_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
IPC_FPC uint64_t fpc_bits64(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}
IPC_FPC double fpc_double(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

// binary32 -> binary64: exponent bias 127 -> 1023, 23 -> 52 fraction bits
IPC_FPC double f2d_bits(float f) {
  const uint32_t u = fpc_bits32(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint32_t ex64 = ex == 0xffu ? 0x7ffu : ex + 896u;  // 1023 - 127
  uint32_t hi = sign | (ex64 << 20) | ((u & 0x7fffffu) >> 3);
  uint32_t lo = u << 29;
  if (ex == 0) {  // zero (and subnormal): signed zero
    hi = sign;
    lo = 0;
  }
  return fpc_double(hi, lo);
}

// binary64 -> binary32, nearest with ties away from zero
IPC_FPC float d2f_bits(double x) {
  const uint64_t b = fpc_bits64(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t mag = b & 0x7fffffffffffffffull;
  if (mag > 0x7ff0000000000000ull) return fpc_float(sign | 0x7fc00000u);  // NaN
  // adding half of the 29 dropped fraction bits rounds; a carry out of the
  // fraction moves into the exponent field, which is the correct result
  const uint64_t m = mag + (1ull << 28);
  const int32_t e32 = (int32_t)(m >> 52) - 896;
  uint32_t u;
  if (e32 <= 0) u = sign;                         // below the normal range
  else if (e32 >= 255) u = sign | 0x7f800000u;    // above it (and infinity)
  else u = sign | ((uint32_t)e32 << 23) | ((uint32_t)(m >> 29) & 0x7fffffu);
  return fpc_float(u);
}

}  // namespace ipc
