// Per-sample live -> canonical warp (Sec. 4.2, Eq. 4, and the object's rigid pose), shared by
// the warp kernels (k_warp.cu) and the fused warp + encoding kernel (k_encode.cu).  The
// search and the blend are described at the top of k_warp.cu.
#pragma once
#include "knn.cuh"

namespace invr {

__device__ __forceinline__ float3 rigid_inverse(const WarpDev& W, float3 p) {
  const float qx = p.x - W.t[0], qy = p.y - W.t[1], qz = p.z - W.t[2];
  return make_float3(W.R[0] * qx + W.R[3] * qy + W.R[6] * qz, W.R[1] * qx + W.R[4] * qy + W.R[7] * qz,
                     W.R[2] * qx + W.R[5] * qy + W.R[8] * qz);
}

// Normalised blend of unit dual quaternions -> inverse motion applied to p.
__device__ __forceinline__ float3 dq_inverse_apply(float4 br, float4 bd, float3 p) {
  const float inv = 1.0f / sqrtf(br.x * br.x + br.y * br.y + br.z * br.z + br.w * br.w);
  // stored as (w, x, y, z) in (x, y, z, w) slots of float4
  const float rw = br.x * inv, rx = br.y * inv, ry = br.z * inv, rz = br.w * inv;
  float dw = bd.x * inv, dx = bd.y * inv, dy = bd.z * inv, dz = bd.w * inv;
  const float dot = rw * dw + rx * dx + ry * dy + rz * dz;
  dw -= dot * rw;
  dx -= dot * rx;
  dy -= dot * ry;
  dz -= dot * rz;
  // t = 2 vec(q_d q_r^*), q_r^* = (rw, -rx, -ry, -rz)
  const float tx = 2.0f * (-dw * rx + dx * rw - dy * rz + dz * ry);
  const float ty = 2.0f * (-dw * ry + dx * rz + dy * rw - dz * rx);
  const float tz = 2.0f * (-dw * rz - dx * ry + dy * rx + dz * rw);
  const float R00 = 1.0f - 2.0f * (ry * ry + rz * rz), R01 = 2.0f * (rx * ry - rw * rz), R02 = 2.0f * (rx * rz + rw * ry);
  const float R10 = 2.0f * (rx * ry + rw * rz), R11 = 1.0f - 2.0f * (rx * rx + rz * rz), R12 = 2.0f * (ry * rz - rw * rx);
  const float R20 = 2.0f * (rx * rz - rw * ry), R21 = 2.0f * (ry * rz + rw * rx), R22 = 1.0f - 2.0f * (rx * rx + ry * ry);
  const float qx = p.x - tx, qy = p.y - ty, qz = p.z - tz;
  return make_float3(R00 * qx + R10 * qy + R20 * qz, R01 * qx + R11 * qy + R21 * qz, R02 * qx + R12 * qy + R22 * qz);
}

// Neighbour set from the tables (Sec. 4.2): the sample's live voxel (clamped into the
// grid) -> the canonical voxel stored there -> its K nodes, ordered by the live key; a
// hole (no canonical voxel landed there) falls back to the exact search.
template <int K>
__device__ __forceinline__ void lut_select(const WarpDev& W, float3 p, float (&keys)[K], int (&ids)[K]) {
  const int G = W.lut_res;
  const int64_t v = grid_cell(p.x, G) + (int64_t)G * (grid_cell(p.y, G) + (int64_t)G * grid_cell(p.z, G));
  const uint32_t k = __ldg(W.lut_live + v);
  if (k == kLutEmpty) {
    knn_select<K>(W, p, keys, ids);
    return;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    keys[j] = INFINITY;
    ids[j] = 0x7FFFFFFF;
  }
  const uint16_t* row = W.lut_canon + (int64_t)k * K;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int id = __ldg(row + j);
    knn_insert_any<K>(knn_key(p, __ldg(W.x_live + id)), id, keys, ids);  // ids arrive in canonical-key order
  }
}

// The blend of the K nearest nodes; cell and n from knn_locate (ignored with look-up tables);
// xs: the node positions the search reads (W.x_live, or its copy in shared memory if SMEM).
template <int K, bool SMEM = false>
__device__ __forceinline__ float3 dqb_warp_at(const WarpDev& W, const float4* xs, float3 p, int64_t cell,
                                              uint32_t n, int32_t* ids_out, int64_t ids_ld, int64_t i) {
  float keys[K];
  int ids[K];
  if (!SMEM && W.lut_live) {
    lut_select<K>(W, p, keys, ids);
  } else {
    knn_scan<K, SMEM>(W, xs, p, cell, n, keys, ids);
  }
  if (ids[0] < 0) return p;  // unreachable for finite p (every list holds >= K nodes)
  const float4 ref = __ldg(W.dq + 2 * ids[0]);
  float4 br = make_float4(0.f, 0.f, 0.f, 0.f), bd = br;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (ids[k] < 0) continue;
    const float4 r = __ldg(W.dq + 2 * ids[k]);
    const float4 du = __ldg(W.dq + 2 * ids[k] + 1);
    float w = expf(-(keys[k] - keys[0]) * W.inv_r2);
    if (r.x * ref.x + r.y * ref.y + r.z * ref.z + r.w * ref.w < 0.0f) w = -w;
    br.x += w * r.x; br.y += w * r.y; br.z += w * r.z; br.w += w * r.w;
    bd.x += w * du.x; bd.y += w * du.y; bd.z += w * du.z; bd.w += w * du.w;
    if (ids_out) ids_out[(int64_t)k * ids_ld + i] = ids[k];
  }
  return dq_inverse_apply(br, bd, p);
}

template <int K>
__device__ __forceinline__ float3 dqb_warp(const WarpDev& W, float3 p, int32_t* ids_out, int64_t ids_ld,
                                           int64_t i) {
  int64_t cell = 0;
  const uint32_t n = W.lut_live ? 0u : knn_locate(W, p, cell);
  return dqb_warp_at<K>(W, W.x_live, p, cell, n, ids_out, ids_ld, i);
}

// Views whose K is at most KMAX (the plan's largest): the instantiations for larger K are not
// compiled into the kernel, which keeps its registers (and so its occupancy) to what KMAX needs.
// SMEM: xs is a shared-memory copy of W.x_live (the caller has checked W.lut_live == null).
template <int KMAX, bool SMEM = false>
__device__ __forceinline__ float3 warp_point_upto(const WarpDev& W, const float4* xs, float3 p, int64_t cell,
                                                  uint32_t n) {
  if (W.mode == 0) return rigid_inverse(W, p);
  if constexpr (KMAX <= 4) {
    switch (W.K) {
      case 1: return dqb_warp_at<1, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 2: return dqb_warp_at<2, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 3: return dqb_warp_at<3, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      default: return dqb_warp_at<4, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
    }
  } else {
    switch (W.K) {
      case 1: return dqb_warp_at<1, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 2: return dqb_warp_at<2, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 3: return dqb_warp_at<3, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 4: return dqb_warp_at<4, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 5: return dqb_warp_at<5, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 6: return dqb_warp_at<6, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      case 7: return dqb_warp_at<7, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
      default: return dqb_warp_at<8, SMEM>(W, xs, p, cell, n, nullptr, 0, 0);
    }
  }
}

__device__ __forceinline__ float3 warp_point(const WarpDev& W, float3 p, int32_t* ids_out, int64_t ids_ld,
                                             int64_t i) {
  if (W.mode == 0) return rigid_inverse(W, p);
  switch (W.K) {
    case 1: return dqb_warp<1>(W, p, ids_out, ids_ld, i);
    case 2: return dqb_warp<2>(W, p, ids_out, ids_ld, i);
    case 3: return dqb_warp<3>(W, p, ids_out, ids_ld, i);
    case 4: return dqb_warp<4>(W, p, ids_out, ids_ld, i);
    case 5: return dqb_warp<5>(W, p, ids_out, ids_ld, i);
    case 6: return dqb_warp<6>(W, p, ids_out, ids_ld, i);
    case 7: return dqb_warp<7>(W, p, ids_out, ids_ld, i);
    default: return dqb_warp<8>(W, p, ids_out, ids_ld, i);
  }
}

}  // namespace invr
