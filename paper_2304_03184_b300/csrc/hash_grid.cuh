// Hash-grid corner geometry, the trilinear gather, and the gradient scatter (warp-aggregated
// runs per vertex-parity slot, x-adjacent pairs as one float4 atomic), used by the encoding
// kernels.
#pragma once

#include "invr_internal.cuh"

namespace invr {

struct Corners {
  uint32_t idx[8];
  float w[8];
  uint32_t par;  // parities of the cell's lower corner: slot k holds corner offset k ^ par
};

// The cell's 8 vertices (the trilinear interpolation of the hash grids, Sec. 4.2), stored by
// coordinate parity: slot k = px + 2 py + 4 pz holds the vertex whose x, y, z coordinates have
// parities px, py, pz.  Along each axis a cell's two vertices have opposite parity, so each
// slot is filled once, and two cells that share a vertex hold it in the same slot.  Slots k
// and k ^ 1 are the two x-adjacent vertices, the even-x one in the even slot.
//
// Per axis the even- and the odd-coordinate vertex (lower corner c, upper c + 1: the even one
// is (c + 1) & ~1, the odd one c | 1) and their interpolation weights are formed once; each
// slot then combines one term per axis: the dense row index x + y (N+1) + z (N+1)^2 or the hash
// (x ^ y pi2 ^ z pi3) mod T from the two y and two z terms, and the weight (w_x w_y) w_z from
// the four x-y products.  The same integers and the same FP32 products as slot-by-slot.
__device__ __forceinline__ void level_corners(const FieldDev& F, int l, float3 x, Corners& c) {
  const int res = F.res[l];
  const bool dense = (F.dense_mask >> l) & 1u;
  const uint32_t tmask = (1u << F.log2T) - 1u;
  float fx, fy, fz;
  const int cx = level_cell(x.x, res, fx), cy = level_cell(x.y, res, fy), cz = level_cell(x.z, res, fz);
  c.par = (uint32_t)((cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2));
  // [0]: the even-coordinate vertex, [1]: the odd one; its weight is f where it is the upper
  // corner (c + 1), 1 - f where it is the lower one
  const uint32_t vx[2] = {(uint32_t)(cx + 1) & ~1u, (uint32_t)cx | 1u};
  const uint32_t vy[2] = {(uint32_t)(cy + 1) & ~1u, (uint32_t)cy | 1u};
  const uint32_t vz[2] = {(uint32_t)(cz + 1) & ~1u, (uint32_t)cz | 1u};
  const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
  const float wx[2] = {(cx & 1) ? fx : gx, (cx & 1) ? gx : fx};
  const float wy[2] = {(cy & 1) ? fy : gy, (cy & 1) ? gy : fy};
  const float wz[2] = {(cz & 1) ? fz : gz, (cz & 1) ? gz : fz};
  uint32_t hy[2], hz[2];
  if (dense) {
    const uint32_t n = (uint32_t)res + 1u;
    hy[0] = vy[0] * n;
    hy[1] = vy[1] * n;
    hz[0] = vz[0] * n * n;
    hz[1] = vz[1] * n * n;
  } else {
    hy[0] = vy[0] * 2654435761u;
    hy[1] = vy[1] * 2654435761u;
    hz[0] = vz[0] * 805459861u;
    hz[1] = vz[1] * 805459861u;
  }
  float wxy[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) wxy[j] = wx[j & 1] * wy[j >> 1];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int px = k & 1, py = (k >> 1) & 1, pz = k >> 2;
    c.idx[k] = dense ? vx[px] + hy[py] + hz[pz] : (vx[px] ^ hy[py] ^ hz[pz]) & tmask;
    c.w[k] = wxy[k & 3] * wz[pz];
  }
}

__device__ __forceinline__ float2 level_feature(const FieldDev& F, int l, const Corners& c) {
  const float2* tab = reinterpret_cast<const float2*>(F.tables) + ((size_t)l << F.log2T);
  float2 e[8];
  // the two x-adjacent vertices share one 16-byte load when the even-x one's table slot is
  // even and the odd-x one's follows it
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    const uint32_t i0 = c.idx[k], i1 = c.idx[k + 1];
    if (i1 == i0 + 1u && !(i0 & 1u)) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(tab + i0));
      e[k] = make_float2(q.x, q.y);
      e[k + 1] = make_float2(q.z, q.w);
    } else {
      e[k] = __ldg(tab + i0);
      e[k + 1] = __ldg(tab + i1);
    }
  }
  float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f0 = fmaf(c.w[k], e[k].x, f0);
    f1 = fmaf(c.w[k], e[k].y, f1);
  }
  return make_float2(f0, f1);
}

// Segmented inclusive scan of val over runs of lanes with equal key: lanes hold consecutive
// samples, mostly of one ray, so consecutive lanes whose cells share a vertex hold it under
// the same key (same parity slot).  Lanes with nothing to add are run heads.  When no lane
// continues a run the scan is skipped, and so is every step longer than the warp's longest
// run needs.  Returns true on the lane that issues the run's sum (its last live lane).
__device__ __forceinline__ bool run_sum(uint32_t key, bool live, float2& val) {
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = !live || lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  if (heads != 0xffffffffu) {
    const int run_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    // need: bit i set when lanes i-o+1 .. i all continue their run, i.e. lane i takes the
    // step of stride o (warp-uniform)
    unsigned need = ~heads;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (need == 0u) break;
      const float x = __shfl_up_sync(0xffffffffu, val.x, o);
      const float y = __shfl_up_sync(0xffffffffu, val.y, o);
      if (lane - o >= run_start) {
        val.x += x;
        val.y += y;
      }
      need &= need << o;
    }
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  return live && tail;
}

// Warp-aggregated scatter of one sample-level: every slot's runs summed by run_sum, then the
// issuing lane sends slots k and k ^ 1 as one 16-byte atomic when it issues both and their
// table slots are the two halves of an aligned pair (i, i ^ 1), else one 8-byte atomic each.
// All lanes of the warp call it (dead lanes with live = false).
__device__ __forceinline__ void scatter_runs(float2* table, const Corners& c, bool live, float2 g) {
  float2 v[8];
  bool issue[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = make_float2(c.w[k] * g.x, c.w[k] * g.y);
    issue[k] = run_sum(c.idx[k], live, v[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    const uint32_t i0 = c.idx[k], i1 = c.idx[k + 1];
    if (issue[k] && issue[k + 1] && (i0 ^ i1) == 1u) {
      const float2 lo = (i0 & 1u) ? v[k + 1] : v[k], hi = (i0 & 1u) ? v[k] : v[k + 1];
      atomicAdd(reinterpret_cast<float4*>(table + (i0 & ~1u)), make_float4(lo.x, lo.y, hi.x, hi.y));
    } else {
      if (issue[k]) atomicAdd(table + i0, v[k]);
      if (issue[k + 1]) atomicAdd(table + i1, v[k + 1]);
    }
  }
}

// Scatter of one sample-level without run summation: the two corners of a cell that differ
// in x go out as one 16-byte atomic when their slots are the two halves of an aligned pair
// (i, i ^ 1: dense rows with an even first slot, hashed slots whenever x is even, in either
// order), else as two 8-byte atomics.
__device__ __forceinline__ void scatter_pairs(float2* table, const Corners& c, float2 g) {
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    const uint32_t i0 = c.idx[k], i1 = c.idx[k + 1];
    const float2 v0 = make_float2(c.w[k] * g.x, c.w[k] * g.y);
    const float2 v1 = make_float2(c.w[k + 1] * g.x, c.w[k + 1] * g.y);
    if ((i0 ^ i1) == 1u) {
      const float2 lo = (i0 & 1u) ? v1 : v0, hi = (i0 & 1u) ? v0 : v1;
      atomicAdd(reinterpret_cast<float4*>(table + (i0 & ~1u)), make_float4(lo.x, lo.y, hi.x, hi.y));
    } else {
      atomicAdd(table + i0, v0);
      atomicAdd(table + i1, v1);
    }
  }
}

}  // namespace invr
