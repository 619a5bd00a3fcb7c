// Field query at live points (warp -> hash encoding -> MLPs) that allocates nothing, for
// callers that cannot call cudaMalloc.  Same kernels and results as invr_query_points; the
// scratch they need between steps (canonical positions [3][n] and features [mlp_in][n])
// sits in one file-scope device array instead of stream-ordered allocations.
#include <mutex>

#include "invr.h"
#include "invr_internal.cuh"

namespace invr {
invr_status resolve_point_query(invr_ctx ctx, const invr_field_view* view, WarpDev& W, FieldDev& F, int& device,
                                int& num_sms, unsigned*& status, uint32_t& wait_limit);
invr_status record_error(invr_ctx ctx, invr_status st, const char* msg);
}  // namespace invr

using namespace invr;

namespace {

constexpr int64_t kMaxPoints = INVR_NOALLOC_MAX_POINTS;
constexpr int64_t kScratchFloats = (3 + kMaxIn) * kMaxPoints;  // 35 x 65536 floats = 9.2 MB

// One scratch array per device, held for the life of the process.  Host code must not use
// this name as an address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float g_query_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_addr[kMaxDevices];  // null until a lookup on that device succeeded
std::mutex g_scratch_mu;

// Device address of the scratch array on `dev` (which the caller has made current).  Only a
// successful lookup is kept, so a failed one (for example during a stream capture, or with
// an error pending) is retried by the next call.
cudaError_t scratch_on(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_query_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

// Called by invr_ctx_create with `dev` current.  The address lookup loads this file's module
// (and with it the scratch array), and the preloads load the kernels the query launches; with
// lazy module loading both would otherwise happen inside the first query, as allocations.
cudaError_t invr::noalloc_prepare(int dev) {
  float* p = nullptr;
  cudaError_t e = scratch_on(dev, &p);
  if (e == cudaSuccess) e = preload_warp_points();
  if (e == cudaSuccess) e = preload_encode_points();
  if (e == cudaSuccess) e = preload_mlp_points_f32();
  if (e == cudaSuccess) e = preload_mlp_points_tc();
  return e;
}

extern "C" invr_status invr_query_points_noalloc(invr_ctx ctx, const invr_field_view* view, int64_t n,
                                                 const float* p, float* out, invr_stream stream) {
  if (!ctx || !view || n < 0) return record_error(ctx, INVR_E_ARG, "bad query_points_noalloc arguments");
  if (n > kMaxPoints)
    return record_error(ctx, INVR_E_ARG,
                        "invr_query_points_noalloc: n exceeds INVR_NOALLOC_MAX_POINTS (65536); split the points");
  WarpDev W;
  FieldDev F;
  int dev = 0, sms = 0;
  unsigned* status = nullptr;
  uint32_t wait_limit = 0;
  invr_status st = resolve_point_query(ctx, view, W, F, dev, sms, status, wait_limit);
  if (st != INVR_OK) return st;
  if (n == 0) return INVR_OK;
  if (!p || !out) return record_error(ctx, INVR_E_ARG, "null pointer");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* scratch = nullptr;
  cudaError_t e = scratch_on(dev, &scratch);
  if (e == cudaSuccess) {
    float* vc = scratch;              // [3][n]
    float* feat = scratch + 3 * n;    // [mlp_in][n]
    e = launch_warp_points(W, n, p, vc, nullptr, s);
    if (e == cudaSuccess) e = launch_encode_points(F, n, vc, feat, nullptr, s);
    if (e == cudaSuccess)
      e = F.mlp_kind == kMlpF32 ? launch_mlp_points_f32(F, n, feat, out, sms, s)
                                : launch_mlp_points_tc(F, n, feat, out, status, wait_limit, sms, s);
  }
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) return record_error(ctx, INVR_E_CUDA, cudaGetErrorString(e));
  return INVR_OK;
}
