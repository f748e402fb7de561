// Coated-surface read-back that allocates nothing.
//
// ipc_read_gel_surface_all gathers the coated-surface rows of every env into a
// staging buffer carved from the caller's workspace, then copies it to the
// host.  Some callers cannot allocate device memory at the point where they
// read results back -- for example code running inside a restricted
// allocator, or a host thread that must not enlarge the device footprint --
// and may also have sized the workspace without room to spare.  This variant
// stages through a fixed file-scope device array instead, so the call itself
// needs no device allocation and no workspace scratch: the caller passes only
// the context (inputs) and a host output array.
//
// The staging array lives in every GPU that loads this library until the
// process exits.  All calls share it, so calls that overlap on the GPU (two
// host threads, or two streams) race on its contents; serialise them.
#include <mutex>

#include "../../include/ipc_b300.h"
#include "ctx.h"

namespace {

constexpr size_t kNoAllocMaxRows = 262144;  // 6 MiB of FP64 positions

static __device__ __align__(256) double g_surface_stage[3 * kNoAllocMaxRows];

// device address of g_surface_stage, resolved once per device with that
// device current (the host-side symbol is only a stand-in, not an address)
constexpr int kMaxDevices = 64;
double* g_stage_ptr[kMaxDevices] = {nullptr};
std::mutex g_stage_mu;

cudaError_t stage_ptr(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_surface_stage);
    if (e != cudaSuccess) return e;
    g_stage_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_stage_ptr[dev];
  return cudaSuccess;
}

__global__ void k_gather_coated_static(const double* x, const int* coated_row, int n, double* stage) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int r = coated_row[i];
  stage[3 * i] = x[3 * r];
  stage[3 * i + 1] = x[3 * r + 1];
  stage[3 * i + 2] = x[3 * r + 2];
}

}  // namespace

extern "C" ipc_status ipc_read_gel_surface_all_noalloc(ipc_ctx* ctx, double* out_xyz, size_t capacity_rows,
                                                      size_t* rows_written) {
  if (!ctx || !out_xyz) return IPC_EINVAL;
  const size_t n_all = (size_t)ctx->pk.n_coated;
  if (n_all > kNoAllocMaxRows) {
    ctx->err = "ipc_read_gel_surface_all_noalloc: " + std::to_string(n_all) +
               " coated-surface rows exceed the fixed staging size of " + std::to_string(kNoAllocMaxRows) +
               " rows; use ipc_read_gel_surface_all";
    return IPC_EINVAL;
  }
  // the staging address belongs to the device that is current when it is
  // looked up; it must be the context's device (where x and the stream live)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ctx->err = std::string("ipc_read_gel_surface_all_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
    return IPC_ECUDA;
  }
  if (dev != ctx->device) {
    ctx->err = "ipc_read_gel_surface_all_noalloc: the current device (" + std::to_string(dev) +
               ") is not the context's device (" + std::to_string(ctx->device) + "); make it current first";
    return IPC_EINVAL;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    ctx->err = "ipc_read_gel_surface_all_noalloc: device ordinal " + std::to_string(dev) +
               " is beyond the " + std::to_string(kMaxDevices) + " devices this entry point supports";
    return IPC_EINVAL;
  }
  double* stage = nullptr;
  e = stage_ptr(dev, &stage);
  if (e != cudaSuccess) {
    ctx->err = std::string("ipc_read_gel_surface_all_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return IPC_ECUDA;
  }
  const size_t n = capacity_rows < n_all ? capacity_rows : n_all;
  if (n_all > 0) {
    int blocks = (int)((n_all + 255) / 256);
    k_gather_coated_static<<<blocks, 256, 0, ctx->stream>>>(ctx->dev.x, ctx->dev.coated_row, (int)n_all, stage);
    e = cudaGetLastError();
    if (e == cudaSuccess && n > 0)
      e = cudaMemcpyAsync(out_xyz, stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      ctx->err = std::string("ipc_read_gel_surface_all_noalloc: ") + cudaGetErrorString(e);
      return IPC_ECUDA;
    }
  }
  if (rows_written) *rows_written = n_all;
  return IPC_OK;
}
