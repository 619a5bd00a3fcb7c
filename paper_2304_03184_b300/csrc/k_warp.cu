// Live -> canonical warp of every sample (Sec. 4.2, Eq. 4, and the object's rigid pose).
//
// Human field: the K deformed nodes x_i^t nearest to the sample (exact; ties to the lower
// node index), Gaussian weights w_i = exp(-|p - x_i^t|^2 / r^2) (Eq. 2, shifted by the
// nearest node's squared distance, which the normalisation cancels), sign alignment to
// the nearest node's quaternion, dual-quaternion blend, normalisation, and the inverse
// rigid motion v_c = R^T (p - t) of the blend.
//
// Exact K-nearest search without scanning all N nodes: once per frame a 128^3 candidate
// grid over [-1,1]^3 is built.  For a cell with centre c and half-diagonal rho, let
// d_K(c) be the distance from c to its K-th nearest node.  Every point p of the cell has K
// nodes within d_K(c) + rho, so each of its K nearest nodes lies within d_K(c) + 2 rho of
// c.  The cell stores all nodes within that radius (times 1.001, plus 1e-4, covering
// single-precision rounding of the keys and of the cell assignment) in index order, so
// scanning the list with the same keys and tie rule as a scan of all nodes selects the
// same K nodes.  Cells whose list exceeds the capacity, and points outside the box, fall
// back to scanning all nodes.  This is the default; the approximate look-up tables of
// Sec. 4.2 ("On-the-fly Radiance Fields", built in k_lut.cu) replace the search when a
// graph has them.
//
// Bound: FP32 ALU (about 10 operations per candidate key) plus L1-resident node reads.
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

// (key, id) ascending insertion with the tie rule written out: the table's ids arrive in
// canonical-key order, not in index order.
template <int K>
__device__ __forceinline__ void lut_insert(float key, int id, float (&keys)[K], int (&ids)[K]) {
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const bool lt = key < keys[m] || (key == keys[m] && id < ids[m]);
    const float tk = lt ? keys[m] : key;
    const int ti = lt ? ids[m] : id;
    keys[m] = lt ? key : keys[m];
    ids[m] = lt ? id : ids[m];
    key = tk;
    id = ti;
  }
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
    lut_insert<K>(knn_key(p, __ldg(W.x_live + id)), id, keys, ids);
  }
}

template <int K>
__device__ __forceinline__ float3 dqb_warp(const WarpDev& W, float3 p, int32_t* ids_out, int64_t ids_ld,
                                           int64_t i) {
  float keys[K];
  int ids[K];
  if (W.lut_live) {
    lut_select<K>(W, p, keys, ids);
  } else {
    knn_select<K>(W, p, keys, ids);
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

__global__ void __launch_bounds__(256) k_warp(const __grid_constant__ Plan P) {
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const int g = P.ws.s_ray[s];
    float3 vc = make_float3(0.f, 0.f, 0.f);
    if (g >= 0) {
      const float3 p = make_float3(P.ws.s_pos[s], P.ws.s_pos[S_cap + s], P.ws.s_pos[2 * S_cap + s]);
      vc = warp_point(P.v[view_of_ray(P, g)].warp, p, nullptr, 0, 0);
    }
    P.ws.s_vc[s] = vc.x;
    P.ws.s_vc[S_cap + s] = vc.y;
    P.ws.s_vc[2 * S_cap + s] = vc.z;
  }
}

cudaError_t launch_warp(const Plan& P, int num_sms, cudaStream_t s) {
  k_warp<<<num_sms * P.tune.warp_ctas_per_sm, 256, 0, s>>>(P);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_warp_points(const __grid_constant__ WarpDev W, int64_t n,
                                                     const float* __restrict__ p, float* vc, int32_t* ids) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float3 q = make_float3(p[i], p[n + i], p[2 * n + i]);
    const float3 r = warp_point(W, q, ids, n, i);
    vc[i] = r.x;
    vc[n + i] = r.y;
    vc[2 * n + i] = r.z;
  }
}

cudaError_t launch_warp_points(const WarpDev& w, int64_t n, const float* p, float* vc, int32_t* ids,
                               cudaStream_t s) {
  if (n > 0) k_warp_points<<<min(ceil_div(n, 256), 65535), 256, 0, s>>>(w, n, p, vc, ids);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ per-frame setup
__global__ void k_graph_pack(const float* __restrict__ dq, const float* __restrict__ x, int n, float4* dq_out,
                             float4* x_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dq_out[2 * i] = make_float4(dq[i], dq[n + i], dq[2 * n + i], dq[3 * n + i]);
  dq_out[2 * i + 1] = make_float4(dq[4 * n + i], dq[5 * n + i], dq[6 * n + i], dq[7 * n + i]);
  x_out[i] = make_float4(x[i], x[n + i], x[2 * n + i], 0.0f);
}

cudaError_t launch_graph_pack(const float* dq_soa, const float* x_soa, int n, float4* dq_out, float4* x_out,
                              cudaStream_t s) {
  k_graph_pack<<<ceil_div(n, 256), 256, 0, s>>>(dq_soa, x_soa, n, dq_out, x_out);
  return cudaGetLastError();
}

// One warp per grid cell: K-th nearest distance from the cell centre, then every node
// within d_K + 2 rho (with margin), in index order.
template <int K>
__global__ void __launch_bounds__(256) k_knn_grid_build(const float4* __restrict__ x, int n, int cap,
                                                        uint16_t* cand, uint16_t* cand_n) {
  const int lane = threadIdx.x & 31;
  const int64_t n_cells = (int64_t)kKnnG * kKnnG * kKnnG;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = warp0; cell < n_cells; cell += n_warps) {
    const int ix = (int)(cell % kKnnG), iy = (int)((cell / kKnnG) % kKnnG), iz = (int)(cell / (kKnnG * kKnnG));
    const float cx = -1.0f + (ix + 0.5f) * kKnnH, cy = -1.0f + (iy + 0.5f) * kKnnH, cz = -1.0f + (iz + 0.5f) * kKnnH;
    float best[K];
#pragma unroll
    for (int k = 0; k < K; ++k) best[k] = INFINITY;
    for (int i = lane; i < n; i += 32) {
      const float4 p = __ldg(x + i);
      const float dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
      float d2 = dx * dx + dy * dy + dz * dz;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float lo = fminf(best[k], d2);
        d2 = fmaxf(best[k], d2);
        best[k] = lo;
      }
    }
    float kth = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float m = best[0];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const unsigned who = __ballot_sync(0xffffffffu, best[0] == m);
      if (lane == __ffs(who) - 1) {
#pragma unroll
        for (int j = 0; j + 1 < K; ++j) best[j] = best[j + 1];
        best[K - 1] = INFINITY;
      }
      kth = m;
    }
    const float rad = (sqrtf(kth) + 2.0f * kKnnRho) * 1.001f + 1e-4f;
    const float rad2 = rad * rad;
    int count = 0;
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      bool in = false;
      if (i < n) {
        const float4 p = __ldg(x + i);
        const float dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
        in = dx * dx + dy * dy + dz * dz <= rad2;
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = count + __popc(m & ((1u << lane) - 1u));
        if (pos < cap) cand[cell * cap + pos] = (uint16_t)i;
      }
      count += __popc(m);
    }
    if (lane == 0) cand_n[cell] = count <= cap ? (uint16_t)count : kKnnOverflow;
  }
}

cudaError_t launch_knn_grid_build(const float4* x_live, int n, int K, int cap, uint16_t* cand, uint16_t* cand_n,
                                  int num_sms, cudaStream_t s) {
  const int grid = num_sms * 8;
  switch (K) {
    case 1: k_knn_grid_build<1><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 2: k_knn_grid_build<2><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 3: k_knn_grid_build<3><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 4: k_knn_grid_build<4><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 5: k_knn_grid_build<5><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 6: k_knn_grid_build<6><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    case 7: k_knn_grid_build<7><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
    default: k_knn_grid_build<8><<<grid, 256, 0, s>>>(x_live, n, cap, cand, cand_n); break;
  }
  return cudaGetLastError();
}

}  // namespace invr
