// Device-side helpers shared by the ABD-IPC kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define IPC_HD __host__ __device__ __forceinline__
#define IPC_D __host__ __device__ __forceinline__
#define IPC_DEV __device__ __forceinline__

namespace ipc {

constexpr int WARP = 32;
constexpr int ROWS_PER_CTA = 128;     // row kernels: 4 warps, one row per thread
constexpr int CHUNK = 32;             // SELL chunk height (one warp)

// ---------------------------------------------------------------- vec3
template <class T>
struct V3 {
  T x, y, z;
};

template <class T> IPC_HD V3<T> v3(T a, T b, T c) { return V3<T>{a, b, c}; }
template <class T> IPC_HD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> IPC_HD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> IPC_HD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> IPC_HD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> IPC_HD V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> IPC_HD T norm2(V3<T> a) { return dot(a, a); }

using D3 = V3<double>;

IPC_D D3 ld3(const double* p, int i) { return D3{p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
IPC_D void st3(double* p, int i, D3 v) { p[3 * i] = v.x; p[3 * i + 1] = v.y; p[3 * i + 2] = v.z; }
IPC_DEV void atomic_add3(double* p, int i, D3 v) {
  atomicAdd(p + 3 * i, v.x);
  atomicAdd(p + 3 * i + 1, v.y);
  atomicAdd(p + 3 * i + 2, v.z);
}
IPC_D double comp(D3 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

// ---------------------------------------------------------------- debug checks
// Bounds-checked builds (-DIPC_CHECKS): IPC_CHECK(word, cond, code, index)
// is false when cond fails, after recording (code, index) as the first
// violation in word[0..1] (atomic, first one wins); the caller then skips
// the access.  Release builds compile it to `true`.
IPC_DEV bool check_record(unsigned long long* word, bool cond, unsigned code, long long index) {
  if (cond) return true;
  if (atomicCAS(word, 0ull, (unsigned long long)code) == 0ull) word[1] = (unsigned long long)index;
  return false;
}
#ifdef IPC_CHECKS
#define IPC_CHECK(word, cond, code, index) ::ipc::check_record((word), (cond), (code), (long long)(index))
#else
#define IPC_CHECK(word, cond, code, index) true
#endif
// codes of IPC_CHECK
enum CheckCode : unsigned {
  CHK_SELL_COL = 1,   // a SELL column outside the row space
  CHK_TET_VERT = 2,   // a tet vertex outside the row space
  CHK_PAIR_VERT = 3,  // a pair's contact vertex outside the contact vertices
  CHK_PCG_ITEM = 4,   // a PCG work item outside the envs / row CTAs
  CHK_ACT_SLOT = 5,   // an active-pair slot or vertex outside its range
  CHK_ASM_SRC = 6,    // an assembly source outside the element blocks
};

// ---------------------------------------------------------------- atomics
// min / max of non-negative doubles through their (monotone) bit patterns
IPC_DEV void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
IPC_DEV void atomic_min_nonneg(double* addr, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------- reductions
template <class T> IPC_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T> IPC_DEV T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block sum in a fixed order (deterministic); blockDim.x multiple of 32, <= 1024.
template <class T> IPC_DEV T block_sum(T v, T* sh /* >= 32 */) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (w == 0) r = warp_sum(r);
  return r;  // valid in thread 0
}
// FP64 sum over a 128-thread CTA with few FP64 instructions (B300 issues
// FP64 at a small fraction of its FP32 rate): two halving steps through
// shared memory (3 warp-wide adds) before one warp's shuffle tree, instead
// of a shuffle tree in every warp (25 warp-wide adds).  Fixed order
// (deterministic).  Valid in thread 0.
IPC_DEV double block_sum128(double v, double* sh /* >= 128 */) {
  __syncthreads();  // a previous use of sh may still be read
  sh[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 64) sh[threadIdx.x] = v + sh[threadIdx.x + 64];
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) r = warp_sum(sh[threadIdx.x] + sh[threadIdx.x + 32]);
  return r;
}
template <class T> IPC_DEV T block_max(T v, T* sh) {
  v = warp_max(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(-INFINITY);
  if (w == 0) r = warp_max(r);
  return r;
}

// env index of item i given prefix offsets off[0..n_envs] (off[e] <= i < off[e+1])
IPC_DEV int find_env(const int* off, int n_envs, int i) {
  int lo = 0, hi = n_envs;  // invariant off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- small dense
// Jacobi stopping threshold on (off-diagonal / diagonal) squared norms: far
// below FP64 rounding, and at FP32 rounding for float (sweeps beyond it
// only rotate rounding noise).
template <class T> struct JacobiTol;
template <> struct JacobiTol<double> { static constexpr double v = 1e-30; };
template <> struct JacobiTol<float> { static constexpr float v = 1e-12f; };

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix in place:
// on return A's diagonal holds the eigenvalues, V (row-major, columns =
// eigenvectors).  Bounded number of sweeps.
template <int n, class T>
IPC_HD void jacobi_eigen(T* A, T* V, int max_sweeps = 12) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = 0, diag = 0;
    for (int i = 0; i < n; ++i) {
      diag += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= JacobiTol<T>::v * diag || off == T(0)) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        T apq = A[p * n + q];
        if (apq == T(0)) continue;
        T app = A[p * n + p], aqq = A[q * n + q];
        T theta = (aqq - app) / (T(2) * apq);
        T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
        T c = T(1) / sqrt(t * t + T(1));
        T s = t * c;
        for (int k = 0; k < n; ++k) {
          T akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          T apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          T vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

// In-place PSD projection of a symmetric n x n matrix (row-major): negative
// eigenvalues clamped to zero, or replaced by their absolute values when
// `absval` is set.  Uses `work` of 2 n^2 elements.
template <int n, class T>
IPC_HD void psd_project(T* H, T* work, bool absval = false) {
  T* A = work;
  T* V = work + n * n;
  for (int i = 0; i < n * n; ++i) A[i] = H[i];
  jacobi_eigen<n, T>(A, V);
  bool neg = false;
  for (int k = 0; k < n; ++k) neg |= (A[k * n + k] < T(0));
  if (!neg) return;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      T s = 0;
      for (int k = 0; k < n; ++k) {
        T l = A[k * n + k];
        if (absval) l = fabs(l);
        if (l > T(0)) s += V[i * n + k] * l * V[j * n + k];
      }
      H[i * n + j] = s;
      H[j * n + i] = s;
    }
}

// True when the symmetric n x n matrix is positive definite (Cholesky runs
// to the end with positive pivots).  work: n * n.
template <int n, class T>
IPC_HD bool is_pos_def(const T* A, T* work) {
  T* L = work;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      T s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (!(s > T(0))) return false;
        L[i * n + i] = sqrt(s);
      } else {
        L[i * n + j] = s / L[j * n + j];
      }
    }
  return true;
}

// Inverse of a symmetric positive definite n x n matrix by Gauss-Jordan with
// partial pivoting (small n).  Returns false if singular.
template <int n, class T>
IPC_HD bool invert_small(const T* A, T* Ainv, T* work /* n*2n */) {
  T* M = work;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? T(1) : T(0));
  for (int c = 0; c < n; ++c) {
    int piv = c;
    T best = fabs(M[c * 2 * n + c]);
    for (int r = c + 1; r < n; ++r) {
      T v = fabs(M[r * 2 * n + c]);
      if (v > best) { best = v; piv = r; }
    }
    if (best == T(0)) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        T t = M[c * 2 * n + j]; M[c * 2 * n + j] = M[piv * 2 * n + j]; M[piv * 2 * n + j] = t;
      }
    T inv = T(1) / M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      T f = M[r * 2 * n + c];
      if (f == T(0)) continue;
      for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

// 3x3 inverse via cofactors; returns determinant.
template <class T>
IPC_HD T inv3(const T* a, T* r) {
  T c00 = a[4] * a[8] - a[5] * a[7];
  T c01 = a[5] * a[6] - a[3] * a[8];
  T c02 = a[3] * a[7] - a[4] * a[6];
  T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  T id = T(1) / det;
  r[0] = c00 * id;
  r[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  r[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  r[3] = c01 * id;
  r[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  r[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  r[6] = c02 * id;
  r[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  r[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return det;
}

}  // namespace ipc
