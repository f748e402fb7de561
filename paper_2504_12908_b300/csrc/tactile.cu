// Tactile outputs read off the deformed coated surface (Sec. 4.2): marker
// positions and flows, and depth / normal maps of orthographic sensors.
//
// Sensor model (the paper gives none): a sensor sits on one gel pad with its
// origin o on the pad's rest contact face, unit in-plane axes e_u, e_v and the
// unit normal n pointing out of the coated face; pixel (r, c) has its centre
// at o + (c + 1/2) pitch e_u + (r + 1/2) pitch e_v.  It looks through the gel
// along +n, so each pixel shows the front-face triangle (a coated boundary
// triangle of that pad whose rest outward normal has an n-component above
// 1/2) with the smallest height h = (x - o).n at the pixel centre.  depth =
// -h there (0 at rest, positive where the surface is pressed in), linearly
// interpolated over the triangle; normal = that triangle's deformed outward
// unit normal.  Pixels no front triangle covers report hit 0, depth 0.
//
// GPU layout: one thread per (sensor, front triangle) rasterises the
// triangle's pixel box and keeps, per pixel, the smallest 64-bit key
// (height as order-preserving FP32 bits, then the triangle's index) with
// atomicMin; one thread per pixel then recomputes depth and normal in FP64
// from the winning triangle.  Keys make the winner independent of the order
// in which threads run.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ipc_b300.h"
#include "common.cuh"
#include "ctx.h"

namespace {

using namespace ipc;

constexpr unsigned long long kNoHit = ~0ull;

// sensor frame as 13 doubles: o[3], e_u[3], e_v[3], n[3], pitch
struct Frame {
  D3 o, eu, ev, n;
  double pitch;
};

__device__ __forceinline__ Frame load_frame(const double* f) {
  return Frame{D3{f[0], f[1], f[2]}, D3{f[3], f[4], f[5]}, D3{f[6], f[7], f[8]}, D3{f[9], f[10], f[11]}, f[12]};
}

// order-preserving map of a float onto unsigned bits (smaller value, smaller key)
__device__ __forceinline__ unsigned int ordered_bits(float v) {
  unsigned int b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ int sensor_of(const int* off, int n, int i) {
  int lo = 0, hi = n;  // off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// barycentric coordinates of (pu, pv) in the projected triangle; false if degenerate
__device__ __forceinline__ bool bary2(const double* U, const double* V, double pu, double pv, double& b0,
                                      double& b1, double& b2) {
  const double det = (U[1] - U[0]) * (V[2] - V[0]) - (U[2] - U[0]) * (V[1] - V[0]);
  if (det == 0.0) return false;
  b1 = ((pu - U[0]) * (V[2] - V[0]) - (U[2] - U[0]) * (pv - V[0])) / det;
  b2 = ((U[1] - U[0]) * (pv - V[0]) - (pu - U[0]) * (V[1] - V[0])) / det;
  b0 = 1.0 - b1 - b2;
  return true;
}

__global__ void k_tact_clear(unsigned long long* keys, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) keys[i] = kNoHit;
}

__global__ void k_tact_raster(const double* __restrict__ x, int n_sensors, const double* __restrict__ frames,
                              const int* __restrict__ tri_off, const int* __restrict__ tri_rows, int H, int W,
                              unsigned long long* keys) {
  const int n_tri = tri_off[n_sensors];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tri; i += gridDim.x * blockDim.x) {
    const int s = sensor_of(tri_off, n_sensors, i);
    const Frame fr = load_frame(frames + 13 * (long long)s);
    double U[3], V[3], Hh[3];
    for (int k = 0; k < 3; ++k) {
      D3 p = ld3(x, tri_rows[3 * i + k]) - fr.o;
      U[k] = dot(p, fr.eu) / fr.pitch;
      V[k] = dot(p, fr.ev) / fr.pitch;
      Hh[k] = dot(p, fr.n);
    }
    // pixel centres (c + 1/2, r + 1/2) inside the triangle's box
    const double umin = fmin(U[0], fmin(U[1], U[2])), umax = fmax(U[0], fmax(U[1], U[2]));
    const double vmin = fmin(V[0], fmin(V[1], V[2])), vmax = fmax(V[0], fmax(V[1], V[2]));
    // (widened by 1e-9 pixel so that centres on an edge are not lost to rounding)
    // (clamped to the image before the integer conversion)
    const int c0 = (int)ceil(fmax(umin - 0.5 - 1e-9, 0.0)), c1 = (int)floor(fmin(umax - 0.5 + 1e-9, W - 1.0));
    const int r0 = (int)ceil(fmax(vmin - 0.5 - 1e-9, 0.0)), r1 = (int)floor(fmin(vmax - 0.5 + 1e-9, H - 1.0));
    const int local = i - tri_off[s];
    unsigned long long* K = keys + (long long)s * H * W;
    for (int r = r0; r <= r1; ++r)
      for (int c = c0; c <= c1; ++c) {
        double b0, b1, b2;
        if (!bary2(U, V, c + 0.5, r + 0.5, b0, b1, b2)) continue;
        if (fmin(b0, fmin(b1, b2)) < -1e-12) continue;  // a centre on a shared edge belongs to both
        const double h = b0 * Hh[0] + b1 * Hh[1] + b2 * Hh[2];
        const unsigned long long key = ((unsigned long long)ordered_bits((float)h) << 32) | (unsigned)local;
        atomicMin(K + (long long)r * W + c, key);
      }
  }
}

__global__ void k_tact_resolve(const double* __restrict__ x, int n_sensors, const double* __restrict__ frames,
                               const int* __restrict__ tri_off, const int* __restrict__ tri_rows, int H, int W,
                               const unsigned long long* __restrict__ keys, double* depth, double* normal,
                               uint8_t* hit) {
  const long long n_pix = (long long)n_sensors * H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pix;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / ((long long)H * W));
    const int rc = (int)(i - (long long)s * H * W);
    const int r = rc / W, c = rc - r * W;
    const unsigned long long key = keys[i];
    double dep = 0.0;
    D3 nrm{0, 0, 0};
    if (key != kNoHit) {
      const Frame fr = load_frame(frames + 13 * (long long)s);
      const int t = tri_off[s] + (int)(key & 0xffffffffull);
      D3 P[3];
      double U[3], V[3], Hh[3];
      for (int k = 0; k < 3; ++k) {
        P[k] = ld3(x, tri_rows[3 * t + k]);
        D3 p = P[k] - fr.o;
        U[k] = dot(p, fr.eu) / fr.pitch;
        V[k] = dot(p, fr.ev) / fr.pitch;
        Hh[k] = dot(p, fr.n);
      }
      double b0, b1, b2;
      bary2(U, V, c + 0.5, r + 0.5, b0, b1, b2);
      dep = -(b0 * Hh[0] + b1 * Hh[1] + b2 * Hh[2]);
      nrm = cross(P[1] - P[0], P[2] - P[0]);
      nrm = (1.0 / sqrt(norm2(nrm))) * nrm;
    }
    depth[i] = dep;
    if (normal) {
      normal[3 * i] = nrm.x;
      normal[3 * i + 1] = nrm.y;
      normal[3 * i + 2] = nrm.z;
    }
    if (hit) hit[i] = key != kNoHit ? 1 : 0;
  }
}

// p = sum_u alpha_u x_(row_u); flow = p - rest
__global__ void k_markers(const double* __restrict__ x, int n, const int* __restrict__ rows,
                          const double* __restrict__ bary, const double* __restrict__ rest, double* pos,
                          double* flow) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  D3 p = bary[3 * k] * ld3(x, rows[3 * k]) + bary[3 * k + 1] * ld3(x, rows[3 * k + 1]) +
         bary[3 * k + 2] * ld3(x, rows[3 * k + 2]);
  st3(pos, k, p);
  if (flow && rest) st3(flow, k, p - ld3(rest, k));
}

ipc_status fail(ipc_ctx* ctx, const char* what, cudaError_t e) {
  ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return IPC_ECUDA;
}

}  // namespace

extern "C" {

ipc_status ipc_gel_vertex_rows(const ipc_ctx* ctx, int env, int n, const int32_t* verts, int32_t* rows_out) {
  if (!ctx || env < 0 || env >= ctx->pk.n_envs || n < 0 || (n && (!verts || !rows_out))) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  for (int i = 0; i < n; ++i) {
    if (verts[i] < 0 || verts[i] >= ev.n_verts) return IPC_EINVAL;
    rows_out[i] = ev.row_begin + ev.inv_perm[verts[i]];
  }
  return IPC_OK;
}

ipc_status ipc_sensor_triangles(const ipc_ctx* ctx, const ipc_sensor* sn, int32_t* rows_out, int capacity,
                                int* n_out) {
  if (!ctx || !sn || !n_out || sn->env < 0 || sn->env >= ctx->pk.n_envs) return IPC_EINVAL;
  const Pack& pk = ctx->pk;
  const EnvInfo& ev = pk.env[sn->env];
  if (sn->pad < 0 || sn->pad >= ev.n_pads) return IPC_EINVAL;
  int n = 0;
  for (int t = ev.tri_begin; t < ev.tri_begin + ev.n_tri; ++t) {
    const int o = pk.tri_obj[t];
    if (pk.obj_local[o] != sn->pad) continue;  // gel pads come first: local object id = pad id
    int rows[3];
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
      const int cv = pk.tri[3 * t + k];
      if (pk.cv_body[cv] >= 0) { ok = false; break; }
      rows[k] = pk.cv_row[cv];
      if (pk.row_kind[rows[k]] != ROW_FREE) ok = false;  // pinned / attached: not coated
    }
    if (!ok) continue;
    double P[3][3];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) P[k][c] = pk.rest_x[3 * (size_t)rows[k] + c];
    double a[3], b[3], nr[3];
    for (int c = 0; c < 3; ++c) { a[c] = P[1][c] - P[0][c]; b[c] = P[2][c] - P[0][c]; }
    nr[0] = a[1] * b[2] - a[2] * b[1];
    nr[1] = a[2] * b[0] - a[0] * b[2];
    nr[2] = a[0] * b[1] - a[1] * b[0];
    const double len = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    if (!(len > 0.0)) continue;
    const double cosn = (nr[0] * sn->normal[0] + nr[1] * sn->normal[1] + nr[2] * sn->normal[2]) / len;
    if (!(cosn > 0.5)) continue;
    if (rows_out && n < capacity)
      for (int k = 0; k < 3; ++k) rows_out[3 * n + k] = rows[k];
    ++n;
  }
  *n_out = n;
  return (rows_out && n > capacity) ? IPC_EOVERFLOW : IPC_OK;
}

ipc_status ipc_tactile_maps_device(ipc_ctx* ctx, int n_sensors, int height, int width, const double* dev_frames,
                                   const int32_t* dev_tri_off, const int32_t* dev_tri_rows, int n_tri_total,
                                   unsigned long long* dev_keys, double* dev_depth, double* dev_normal,
                                   uint8_t* dev_hit) {
  if (!ctx || n_sensors < 0 || height <= 0 || width <= 0 || n_tri_total < 0) return IPC_EINVAL;
  if (n_sensors == 0) return IPC_OK;
  if (!dev_frames || !dev_tri_off || (n_tri_total && !dev_tri_rows) || !dev_keys || !dev_depth) return IPC_EINVAL;
  const long long n_pix = (long long)n_sensors * height * width;
  cudaStream_t s = ctx->stream;
  k_tact_clear<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(dev_keys, n_pix);
  if (n_tri_total > 0) {
    const int blocks = (int)std::min<long long>((n_tri_total + 127) / 128, 148LL * 16);
    k_tact_raster<<<blocks, 128, 0, s>>>(ctx->dev.x, n_sensors, dev_frames, dev_tri_off, dev_tri_rows, height,
                                         width, dev_keys);
  }
  const int rblocks = (int)std::min<long long>((n_pix + 255) / 256, 148LL * 32);
  k_tact_resolve<<<rblocks, 256, 0, s>>>(ctx->dev.x, n_sensors, dev_frames, dev_tri_off, dev_tri_rows, height,
                                         width, dev_keys, dev_depth, dev_normal, dev_hit);
  ctx->launches += n_tri_total > 0 ? 3 : 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, "ipc_tactile_maps_device", e);
  return IPC_OK;
}

ipc_status ipc_markers_device(ipc_ctx* ctx, int n, const int32_t* dev_rows, const double* dev_bary,
                              const double* dev_rest, double* dev_pos, double* dev_flow) {
  if (!ctx || n < 0) return IPC_EINVAL;
  if (n == 0) return IPC_OK;
  if (!dev_rows || !dev_bary || !dev_pos) return IPC_EINVAL;
  k_markers<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->dev.x, n, dev_rows, dev_bary, dev_rest, dev_pos,
                                                       dev_flow);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, "ipc_markers_device", e);
  return IPC_OK;
}

}  // extern "C"
