// Multiresolution hash encoding (the canonical hash grids H^h, H^o of Sec. 4.2, built as
// in Instant-NGP): per level l, the cell of the canonical point on a grid of resolution
// N_l, the table slots of its 8 corners (dense row-major when (N_l+1)^3 <= T, else the
// XOR-of-primes spatial hash mod T) and the trilinear blend of their F = 2 features.
//
// Forward: one thread per sample, all its levels; a block takes a chunk of 256 consecutive
// samples, so a warp reads a level's table for 32 consecutive samples of one ray (spatially
// coherent).  Backward: one thread per (sample, level); a block takes one level of a chunk,
// and the blocks of a chunk's levels run together (its positions are read from DRAM once,
// then from L2).  Tables are level-major [L][T][2] FP32: each corner is one 8-byte load, and
// the +x corner pair shares a 32-byte sector.  Features are written feature-major [L*2][S]
// (coalesced) for FP32 fields, and as the 16-bit MMA operand tiles of the tensor-core MLPs
// for FP16/BF16 fields.
//
// Backward: the same corners receive w_corner * dL/dfeat through atomics into the gradient
// table (same layout).  Corners are held by vertex parity, so consecutive lanes whose cells
// share a vertex hold it in the same slot; on coarse levels each slot's runs are summed
// first (segmented warp scan) and one atomic carries a run's sum.
//
// Bound: the tables (up to 64 MiB per field) stay L2-resident; the forward is bound by the
// L1 wavefronts of its 8 x 8 B gathers per sample-level, the backward by instruction issue
// together with the L2's atomic rate (8 x 8 B of corner updates per sample-level).
#include "hash_grid.cuh"
#include "tc_ptx.cuh"
#include "warp.cuh"

namespace invr {

// The features of sample slot s at canonical position x (zero where !live), written as the
// field's layout: FP32 feature-major, or the 16-bit operand tiles (and, for training, the
// remainder tiles).
__device__ __forceinline__ void encode_sample(const Plan& P, const FieldDev& F, int64_t s, float3 x, bool live) {
  const int64_t S_cap = P.ws.S_cap;
  float* feat = static_cast<float*>(P.ws.feat);
  // F.L is a multiple of 4 (mlp_in = 2 L is 16 or 32; the deformation net's 2 L a multiple of 8)
  for (int l0 = 0; l0 < F.L; l0 += 4) {
    uint32_t packed[4], rest[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + j;
      float2 f = make_float2(0.0f, 0.0f);
      if (live) {
        Corners c;
        level_corners(F, l, x, c);
        f = level_feature(F, l, c);
      }
      if (F.mlp_kind == kMlpF32) {
        feat[(int64_t)(2 * l) * S_cap + s] = f.x;
        feat[(int64_t)(2 * l + 1) * S_cap + s] = f.y;
      } else {
        // tensor-core field: the pair as 16-bit operand row s of its tile (rounded to nearest)
        // and, for training, the remainder of that rounding
        if (F.mlp_kind == kMlpBF16)
          tc::split2<true>(f.x, f.y, packed[j], rest[j]);
        else
          tc::split2<false>(f.x, f.y, packed[j], rest[j]);
      }
    }
    if (F.mlp_kind != kMlpF32) {
      uint8_t* dst = reinterpret_cast<uint8_t*>(feat) + feat16_offset(S_cap, s, 2 * l0);
      *reinterpret_cast<uint4*>(dst) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
      if (P.feat_split)
        *reinterpret_cast<uint4*>(dst + feat16_lo_offset(S_cap)) = make_uint4(rest[0], rest[1], rest[2], rest[3]);
    }
  }
}

// Work items: chunks of 256 consecutive samples.  A thread evaluates every level of its
// sample, level by level in step with the other warps of its block, so the block's warps
// share each level's table lines in L1 (4 levels per item ran 6% slower, 8 levels 15%: the
// blocks of an SM then interleave more tables).  For a tensor-core field each group of 4
// levels -- 8 16-bit features, one 16-byte row of an operand core matrix -- is written by
// one store.
__global__ void __launch_bounds__(256) k_encode(const __grid_constant__ Plan P) {
  __shared__ int32_t vb[kMaxViews + 1];  // view sample bases
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  if (threadIdx.x <= P.n_views) vb[threadIdx.x] = P.ws.view_base[threadIdx.x];
  __syncthreads();
  const int64_t S0 = vb[P.view_lo], S = vb[P.view_hi];
  const int64_t n_chunks = (S - S0 + 255) / 256;
  int v = P.view_lo;  // cursor: this thread's samples only increase over its chunks
  for (int64_t chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    const int64_t s = S0 + chunk * 256 + threadIdx.x;
    if (s >= S) continue;
    v = advance_view(vb, P.view_hi, s, v);
    const bool live = P.ws.s_ray[s] >= 0;
    const float3 x = live ? make_float3(P.ws.s_vc[s], P.ws.s_vc[S_cap + s], P.ws.s_vc[2 * S_cap + s])
                          : make_float3(0.0f, 0.0f, 0.0f);
    encode_sample(P, P.v[v].field, s, x, live);
  }
}

// The forward chain's first two steps fused per work item of CHUNK consecutive samples: each
// thread warps its sample (the K nearest nodes and the dual-quaternion blend, or the rigid
// pose), writes v_c (the backward's scatter reads it), and -- after a block barrier, so that
// the block's warps walk the levels together and share each level's table lines in L1 --
// encodes it from registers.  One launch per field (the field's tables stay in L2); the
// canonical positions never go through DRAM between the two steps, and the warp's latency
// overlaps the other blocks' gathers.  CHUNK (128 or 256) is chosen by the autotuner.
template <int KMAX, int CHUNK>
__global__ void __launch_bounds__(CHUNK) k_warp_encode(const __grid_constant__ Plan P) {
  __shared__ int32_t vb[kMaxViews + 1];  // view sample bases
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  if (threadIdx.x <= P.n_views) vb[threadIdx.x] = P.ws.view_base[threadIdx.x];
  __syncthreads();
  const int64_t S0 = vb[P.view_lo], S = vb[P.view_hi];
  const int64_t n_chunks = (S - S0 + CHUNK - 1) / CHUNK;
  int v = P.view_lo;  // cursor: this thread's samples only increase over its chunks
  for (int64_t chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    const int64_t s = S0 + chunk * CHUNK + threadIdx.x;
    bool live = false;
    float3 x = make_float3(0.0f, 0.0f, 0.0f);
    if (s < S) {
      v = advance_view(vb, P.view_hi, s, v);
      if (P.ws.s_ray[s] >= 0) {
        live = true;
        const WarpDev& W = P.v[v].warp;
        const float3 p = make_float3(P.ws.s_pos[s], P.ws.s_pos[S_cap + s], P.ws.s_pos[2 * S_cap + s]);
        int64_t cell = 0;
        const uint32_t n = (W.mode == 0 || W.lut_live) ? 0u : knn_locate(W, p, cell);
        x = warp_point_upto<KMAX>(W, W.x_live, p, cell, n);
      }
      P.ws.s_vc[s] = x.x;
      P.ws.s_vc[S_cap + s] = x.y;
      P.ws.s_vc[2 * S_cap + s] = x.z;
    }
    __syncthreads();
    if (s < S) encode_sample(P, P.v[v].field, s, x, live);
  }
}

// Work items: (chunk of 256 samples, group of kBwdLevels levels), group fastest; a thread
// takes its sample's levels of the group in turn (each level uniform across the warp, as
// the run scan needs).  One level per item: with 2 or 4 the scatter ran 3% and 24% slower
// (fewer items in flight per level, so the atomics of concurrent warps spread over more of
// the gradient tables).
constexpr int kBwdLevels = 1;

__global__ void __launch_bounds__(256) k_encode_bwd(const __grid_constant__ Plan P, int L) {
  __shared__ int32_t vb[kMaxViews + 1];  // view sample bases
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  if (threadIdx.x <= P.n_views) vb[threadIdx.x] = P.ws.view_base[threadIdx.x];
  __syncthreads();
  const int64_t S0 = vb[P.view_lo], S = vb[P.view_hi];
  const float scale = P.grad_scale;
  const int64_t n_chunks = (S - S0 + 255) / 256;
  int v = P.view_lo;  // cursor: this warp's samples only increase over its work items
  // warps never straddle two views: view ranges are kTile-aligned (S0 too) and a warp is 32
  for (ItemWalk w((L + kBwdLevels - 1) / kBwdLevels); w.chunk < n_chunks; w.next()) {
    const int l0 = kBwdLevels * w.l;
    const int64_t s0 = S0 + w.chunk * 256;
    const int64_t s = s0 + threadIdx.x;
    const int64_t sw = s0 + (threadIdx.x & ~31);
    v = advance_view(vb, P.view_hi, sw, v);
    const FieldDev& F = P.v[v].field;
    if (l0 >= F.L || sw >= S) continue;  // warp-uniform
    const bool in = s < S && P.ws.s_ray[s] >= 0;
    const float3 x = in ? make_float3(P.ws.s_vc[s], P.ws.s_vc[S_cap + s], P.ws.s_vc[2 * S_cap + s])
                        : make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < kBwdLevels; ++j) {
      const int l = l0 + j;
      if (l >= F.L) break;  // warp-uniform
      bool live = in;
      float2 g = make_float2(0.0f, 0.0f);
      if (live) {
        g.x = P.ws.dfeat[(int64_t)(2 * l) * S_cap + s] * scale;
        g.y = P.ws.dfeat[(int64_t)(2 * l + 1) * S_cap + s] * scale;
        live = (g.x != 0.0f) || (g.y != 0.0f);
      }
      Corners c;
      if (live) {
        level_corners(F, l, x, c);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          c.idx[k] = 0;
          c.w[k] = 0.0f;
        }
      }
      float2* gt = reinterpret_cast<float2*>(F.grad_tables) + ((size_t)l << F.log2T);
      if (F.res[l] <= P.agg_res) {
        scatter_runs(gt, c, live, g);
      } else if (live) {
        scatter_pairs(gt, c, g);
      }
    }
  }
}

cudaError_t launch_encode(const Plan& P, int num_sms, cudaStream_t s) {
  k_encode<<<num_sms * P.tune.encode_ctas_per_sm, 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_encode_bwd(const Plan& P, int num_sms, cudaStream_t s) {
  int L = 0;
  for (int v = 0; v < P.n_views; ++v) L = P.v[v].field.L > L ? P.v[v].field.L : L;
  k_encode_bwd<<<num_sms * P.tune.encode_bwd_ctas_per_sm * ((L + kBwdLevels - 1) / kBwdLevels), 256, 0, s>>>(P, L);
  return cudaGetLastError();
}

// One launch per group of consecutive views that share a field.
template <class Launch>
cudaError_t per_field(const Plan& P, Launch launch) {
  Plan Q = P;
  int lo = P.view_lo;
  while (lo < P.view_hi) {
    int hi = lo + 1;
    while (hi < P.view_hi && P.v[hi].field.tables == P.v[lo].field.tables) ++hi;
    Q.view_lo = lo;
    Q.view_hi = hi;
    const cudaError_t e = launch(Q);
    if (e != cudaSuccess) return e;
    lo = hi;
  }
  return cudaSuccess;
}

cudaError_t launch_encode_by_field(const Plan& P, int num_sms, cudaStream_t s) {
  return per_field(P, [&](const Plan& Q) { return launch_encode(Q, num_sms, s); });
}

cudaError_t launch_encode_bwd_by_field(const Plan& P, int num_sms, cudaStream_t s) {
  return per_field(P, [&](const Plan& Q) { return launch_encode_bwd(Q, num_sms, s); });
}

template <int KMAX>
cudaError_t launch_warp_encode_k(const Plan& Q, int num_sms, cudaStream_t s) {
  const int grid = num_sms * Q.tune.encode_ctas_per_sm;
  if (Q.tune.chunk == 128)
    k_warp_encode<KMAX, 128><<<grid, 128, 0, s>>>(Q);
  else
    k_warp_encode<KMAX, 256><<<grid, 256, 0, s>>>(Q);
  return cudaGetLastError();
}

cudaError_t launch_warp_encode_by_field(const Plan& P, int num_sms, cudaStream_t s) {
  int kmax = 0;
  for (int v = 0; v < P.n_views; ++v)
    if (P.v[v].warp.mode == 1 && P.v[v].warp.K > kmax) kmax = P.v[v].warp.K;
  return per_field(P, [&](const Plan& Q) {
    return kmax <= 4 ? launch_warp_encode_k<4>(Q, num_sms, s) : launch_warp_encode_k<8>(Q, num_sms, s);
  });
}

// ------------------------------------------------------------------ single step
// One thread per point over all its levels, in step with its block (as k_encode); FP32
// features [L*2][n].  Held to 48 registers (5 blocks per SM): with the per-axis corners it
// took 56 (4 blocks), and the occupancy update's queries ran 5% slower.
__global__ void __launch_bounds__(256, 5) k_encode_points(const __grid_constant__ FieldDev F, int64_t n,
                                                       const float* __restrict__ x, float* feat, uint32_t* idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float3 p = make_float3(x[i], x[n + i], x[2 * n + i]);
    for (int l = 0; l < F.L; ++l) {
      Corners c;
      level_corners(F, l, p, c);
      const float2 f = level_feature(F, l, c);
      feat[(int64_t)(2 * l) * n + i] = f.x;
      feat[(int64_t)(2 * l + 1) * n + i] = f.y;
      if (idx) {
        // rows by corner offset bx + 2 by + 4 bz from the cell's lower corner
#pragma unroll
        for (int k = 0; k < 8; ++k) idx[(int64_t)(l * 8 + (int)(k ^ c.par)) * n + i] = c.idx[k];
      }
    }
  }
}

cudaError_t launch_encode_points(const FieldDev& f, int64_t n, const float* x, float* feat, uint32_t* idx,
                                 cudaStream_t s) {
  if (n > 0) k_encode_points<<<min(ceil_div(n, 256), 65535), 256, 0, s>>>(f, n, x, feat, idx);
  return cudaGetLastError();
}

cudaError_t preload_encode_points() {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, k_encode_points);
}

}  // namespace invr
