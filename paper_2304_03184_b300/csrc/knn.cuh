// Exact K-nearest-node selection shared by the warp and the look-up-table builder: the
// FP32 key ((dx*dx)+(dy*dy))+(dz*dz), ties to the lower node index, candidates from the
// per-frame 128^3 candidate grid (or all nodes where a cell overflowed).
#pragma once
#include "invr_internal.cuh"

namespace invr {

// Insert (key, id) into the ascending list; equal keys keep the earlier (lower) id first.
// From the first slot whose key is larger, every later entry shifts down by one (an
// entry carried down is never compared again, so entries with equal keys keep their order).
template <int K>
__device__ __forceinline__ void knn_insert(float key, int id, float (&keys)[K], int (&ids)[K]) {
  if (!(key < keys[K - 1])) return;
  bool shift = false;
#pragma unroll
  for (int m = 0; m < K; ++m) {
    shift = shift || key < keys[m];
    const float tk = shift ? keys[m] : key;
    const int ti = shift ? ids[m] : id;
    keys[m] = shift ? key : keys[m];
    ids[m] = shift ? id : ids[m];
    key = tk;
    id = ti;
  }
}

// The candidate-grid cell of p and its list length, or n = kKnnOverflow where every node
// must be scanned (no grid, p outside the box, or the cell's list overflowed).
__device__ __forceinline__ uint32_t knn_locate(const WarpDev& W, float3 p, int64_t& cell) {
  cell = 0;
  if (W.cand_n && fabsf(p.x) <= 1.001f && fabsf(p.y) <= 1.001f && fabsf(p.z) <= 1.001f) {
    cell = grid_cell(p.x, kKnnG) + kKnnG * (grid_cell(p.y, kKnnG) + kKnnG * grid_cell(p.z, kKnnG));
    return __ldg(W.cand_n + cell);
  }
  return kKnnOverflow;
}

// The K nearest nodes of p from the located cell's list (or all nodes).
template <int K>
__device__ __forceinline__ void knn_scan(const WarpDev& W, float3 p, int64_t cell, uint32_t n, float (&keys)[K],
                                         int (&ids)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    keys[k] = INFINITY;
    ids[k] = -1;
  }
  if (n == kKnnOverflow) {
    for (int i = 0; i < W.n_nodes; ++i) knn_insert<K>(knn_key(p, __ldg(W.x_live + i)), i, keys, ids);
  } else {
    // the list in chunks of 8 ids (one 16-byte load; cap is a multiple of 8), whose 8 node
    // loads are issued together, then inserted in list order (= index order, as before)
    const uint16_t* list = W.cand + cell * W.cap;
    uint32_t c = 0;
    for (; c + 8 <= n; c += 8) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(list + c));
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
      float4 x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = __ldg(W.x_live + ((w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu));
#pragma unroll
      for (int j = 0; j < 8; ++j) knn_insert<K>(knn_key(p, x[j]), (int)((w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu), keys, ids);
    }
    for (; c < n; ++c) {
      const int i = __ldg(list + c);
      knn_insert<K>(knn_key(p, __ldg(W.x_live + i)), i, keys, ids);
    }
  }
}

template <int K>
__device__ __forceinline__ void knn_select(const WarpDev& W, float3 p, float (&keys)[K], int (&ids)[K]) {
  int64_t cell;
  const uint32_t n = knn_locate(W, p, cell);
  knn_scan<K>(W, p, cell, n, keys, ids);
}

}  // namespace invr
