// Exact K-nearest-node selection shared by the warp and the look-up-table builder: the
// FP32 key ((dx*dx)+(dy*dy))+(dz*dz), ties to the lower node index, candidates from the
// per-frame 128^3 candidate grid (or all nodes where a cell overflowed).
//
// A cell's candidate list is sorted by the nodes' distance r_i from the cell centre c, each
// entry holding the node id (low 16 bits) and a lower bound of r_i (high 16 bits, in units
// of 2^-14).  For a point p of the cell, every node j at or after list position i is at
// least r_i - |p - c| from p, so once that bound squared exceeds the current K-th key no
// later candidate can enter the K nearest and the scan stops.  The first kKnnHead entries of
// every list also sit in the cell's own 32-byte head (one sector, read without first reading
// a count: lists end with an end marker), so a scan that stops within them -- most do --
// touches one sector of a 64 MB array per frame (the occupied cells' heads stay in L2)
// instead of a row of the cap-entry array.
#pragma once
#include "invr_internal.cuh"

namespace invr {

constexpr float kKnnRUnit = 1.0f / 16384.0f;  // r bound units (r < 4 covers [-1,1]^3)

// Insert (key, id) into the ascending list; equal keys keep the earlier (lower) id first.
// From the first slot whose key is larger, every later entry shifts down by one (an
// entry carried down is never compared again, so entries with equal keys keep their order).
// For candidates arriving in index order.
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

// (key, id) ascending insertion with the tie rule written out, for candidates in any order.
template <int K>
__device__ __forceinline__ void knn_insert_any(float key, int id, float (&keys)[K], int (&ids)[K]) {
  if (!(key < keys[K - 1] || (key == keys[K - 1] && id < ids[K - 1]))) return;
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

// The candidate-grid cell of p (returns 0), or kKnnOverflow where every node must be scanned
// (no grid, or p outside the box).  Reads no memory.
__device__ __forceinline__ uint32_t knn_locate(const WarpDev& W, float3 p, int64_t& cell) {
  cell = 0;
  if (W.cand_head && fabsf(p.x) <= 1.001f && fabsf(p.y) <= 1.001f && fabsf(p.z) <= 1.001f) {
    cell = grid_cell(p.x, kKnnG) + kKnnG * (grid_cell(p.y, kKnnG) + kKnnG * grid_cell(p.z, kKnnG));
    return 0u;
  }
  return kKnnOverflow;
}

// Centre of candidate-grid cell `cell` (the builder's formula).
__device__ __forceinline__ float3 knn_cell_centre(int64_t cell) {
  constexpr float H = 2.0f / kKnnG;
  const int ix = (int)(cell % kKnnG), iy = (int)((cell / kKnnG) % kKnnG), iz = (int)(cell / (kKnnG * kKnnG));
  return make_float3(-1.0f + (ix + 0.5f) * H, -1.0f + (iy + 0.5f) * H, -1.0f + (iz + 0.5f) * H);
}

// Node i's live position, from global memory (read-only path) or from a copy in shared memory.
template <bool SMEM>
__device__ __forceinline__ float4 node_at(const float4* xs, int i) {
  if constexpr (SMEM) return xs[i];
  else return __ldg(xs + i);
}

// Four entries of a cell's list (one 16-byte load), their node loads issued together: each
// is inserted unless the list has ended or the distance bound rules it and every later entry
// out.  Returns false once the scan must stop.
template <int K, bool SMEM>
__device__ __forceinline__ bool knn_group(const float4* xs, float3 p, float pc, uint4 q, float (&keys)[K],
                                          int (&ids)[K]) {
  const uint32_t e[4] = {q.x, q.y, q.z, q.w};
  float4 x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t id = e[j] & 0xFFFFu;
    x[j] = node_at<SMEM>(xs, id == 0xFFFFu ? 0 : (int)id);  // end markers load node 0, never inserted
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if ((e[j] & 0xFFFFu) == 0xFFFFu) return false;
    // every later node is at least a = r_lo - |p - c| from p; its FP32 key is then at
    // least a^2 (1 - 2^-20), so a^2 (1 - 1e-5) > the K-th key rules all of them out
    const float a = (float)(e[j] >> 16) * kKnnRUnit - pc;
    if (a > 0.0f && a * a * 0.99999f > keys[K - 1]) return false;
    knn_insert_any<K>(knn_key(p, x[j]), (int)(e[j] & 0xFFFFu), keys, ids);
  }
  return true;
}

// The K nearest nodes of p from the located cell's list (or all nodes); xs is W.x_live or
// its copy in shared memory (SMEM).  The list's head first, then the rest of its row.
template <int K, bool SMEM = false>
__device__ __forceinline__ void knn_scan(const WarpDev& W, const float4* xs, float3 p, int64_t cell, uint32_t n,
                                         float (&keys)[K], int (&ids)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    keys[k] = INFINITY;
    ids[k] = -1;
  }
  uint4 h0 = make_uint4(kKnnHeadOverflow, 0u, 0u, 0u), h1 = h0;
  if (n != kKnnOverflow) {
    const uint4* head = reinterpret_cast<const uint4*>(W.cand_head + cell * kKnnHead);
    h0 = __ldg(head);
    h1 = __ldg(head + 1);
  }
  if (h0.x == kKnnHeadOverflow) {
    for (int i = 0; i < W.n_nodes; ++i) knn_insert<K>(knn_key(p, node_at<SMEM>(xs, i)), i, keys, ids);
    return;
  }
  // |p - c|, rounded up: the bound r_i - |p - c| must not exceed the true distance
  const float3 c = knn_cell_centre(cell);
  const float ex = p.x - c.x, ey = p.y - c.y, ez = p.z - c.z;
  const float pc = sqrtf(ex * ex + ey * ey + ez * ez) * 1.00001f + 1e-7f;
  if (!knn_group<K, SMEM>(xs, p, pc, h0, keys, ids) || !knn_group<K, SMEM>(xs, p, pc, h1, keys, ids)) return;
  const uint32_t* list = W.cand + cell * W.cap;  // entries from kKnnHead on (cap is a multiple of 8)
  for (int g = kKnnHead; g < W.cap; g += 4)
    if (!knn_group<K, SMEM>(xs, p, pc, __ldg(reinterpret_cast<const uint4*>(list + g)), keys, ids)) return;
}

template <int K>
__device__ __forceinline__ void knn_select(const WarpDev& W, float3 p, float (&keys)[K], int (&ids)[K]) {
  int64_t cell;
  const uint32_t n = knn_locate(W, p, cell);
  knn_scan<K>(W, W.x_live, p, cell, n, keys, ids);
}

}  // namespace invr
