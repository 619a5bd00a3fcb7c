// Multiresolution hash encoding (the canonical hash grids H^h, H^o of Sec. 4.2, built as
// in Instant-NGP): per level l, the cell of the canonical point on a grid of resolution
// N_l, the table slots of its 8 corners (dense row-major when (N_l+1)^3 <= T, else the
// XOR-of-primes spatial hash mod T) and the trilinear blend of their F = 2 features.
//
// One thread per (sample, level); blockIdx.y is the level, so a warp reads one level's
// table for 32 consecutive samples of one ray (spatially coherent).  Tables are level-major
// [L][T][2] FP32: each corner is one 8-byte load, and the +x corner pair shares a 32-byte
// sector.  Features are written feature-major [L*2][S] (coalesced).
//
// Backward: the same corners receive w_corner * dL/dfeat through float2 atomics into the
// gradient table (same layout).  On coarse levels, lanes of a warp that hit the same slot
// are summed first (segmented run reduction) so that one atomic carries the run's sum.
//
// Bound: L2 (tables up to 64 MiB per field stay L2-resident) -- 8 x 8 B gathers per
// sample-level forward, 8 x 8 B atomics backward.
#include "invr_internal.cuh"

namespace invr {

struct Corners {
  uint32_t idx[8];
  float w[8];
};

__device__ __forceinline__ void level_corners(const FieldDev& F, int l, float3 x, Corners& c) {
  const int res = F.res[l];
  const bool dense = (F.dense_mask >> l) & 1u;
  const uint32_t tmask = (1u << F.log2T) - 1u;
  float fx, fy, fz;
  const int cx = level_cell(x.x, res, fx), cy = level_cell(x.y, res, fy), cz = level_cell(x.z, res, fz);
  const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
    c.idx[k] = vertex_index((uint32_t)(cx + bx), (uint32_t)(cy + by), (uint32_t)(cz + bz), res, dense, tmask);
    c.w[k] = (wx[bx] * wy[by]) * wz[bz];
  }
}

__device__ __forceinline__ float2 level_feature(const FieldDev& F, int l, const Corners& c) {
  const float2* tab = reinterpret_cast<const float2*>(F.tables) + ((size_t)l << F.log2T);
  float2 e[8];
  // the two corners that differ in x share one 16-byte load when their slots are an
  // aligned adjacent pair
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

__global__ void __launch_bounds__(256) k_encode(const __grid_constant__ Plan P) {
  const int l = blockIdx.y;
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  const int64_t S0 = P.ws.view_base[P.view_lo], S = P.ws.view_base[P.view_hi];
  float* feat = static_cast<float*>(P.ws.feat);
  int v = P.view_lo;
  for (int64_t s = S0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    while (v + 1 < P.view_hi && s >= P.ws.view_base[v + 1]) ++v;
    const FieldDev& F = P.v[v].field;
    if (l >= F.L) continue;
    float2 f = make_float2(0.0f, 0.0f);
    if (P.ws.s_ray[s] >= 0) {
      Corners c;
      level_corners(F, l, make_float3(P.ws.s_vc[s], P.ws.s_vc[S_cap + s], P.ws.s_vc[2 * S_cap + s]), c);
      f = level_feature(F, l, c);
    }
    feat[(int64_t)(2 * l) * S_cap + s] = f.x;
    feat[(int64_t)(2 * l + 1) * S_cap + s] = f.y;
  }
}

// Warp-aggregated scatter: lanes hold consecutive samples, mostly of one ray, so lanes
// hitting the same slot form contiguous runs on coarse levels.  A segmented inclusive
// scan sums each run; the run's last lane issues one atomic for the whole run.  Lanes
// with nothing to add are run heads that issue nothing.  When no lane continues a run the
// scan is skipped.
__device__ __forceinline__ void scatter_runs(float2* table, uint32_t key, bool live, float2 val) {
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = !live || lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  if (heads != 0xffffffffu) {
    const int run_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float x = __shfl_up_sync(0xffffffffu, val.x, o);
      const float y = __shfl_up_sync(0xffffffffu, val.y, o);
      if (lane - o >= run_start) {
        val.x += x;
        val.y += y;
      }
    }
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  if (live && tail) atomicAdd(table + key, val);
}

// Scatter of one sample-level without run summation: the two corners of a cell that differ
// in x go out as one 16-byte atomic when their slots are an aligned adjacent pair (dense
// rows, or a hashed slot with x even), else as two 8-byte atomics.
__device__ __forceinline__ void scatter_pairs(float2* table, const Corners& c, float2 g) {
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    const uint32_t i0 = c.idx[k], i1 = c.idx[k + 1];
    const float2 v0 = make_float2(c.w[k] * g.x, c.w[k] * g.y);
    const float2 v1 = make_float2(c.w[k + 1] * g.x, c.w[k + 1] * g.y);
    if (i1 == i0 + 1u && !(i0 & 1u)) {
      atomicAdd(reinterpret_cast<float4*>(table + i0), make_float4(v0.x, v0.y, v1.x, v1.y));
    } else {
      atomicAdd(table + i0, v0);
      atomicAdd(table + i1, v1);
    }
  }
}

__global__ void __launch_bounds__(256) k_encode_bwd(const __grid_constant__ Plan P) {
  const int l = blockIdx.y;
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  const int64_t S0 = P.ws.view_base[P.view_lo], S = P.ws.view_base[P.view_hi];
  const float scale = P.grad_scale;
  int v = P.view_lo;
  // warps never straddle two views: view ranges are kTile-aligned (S0 too) and a warp is 32
  for (int64_t s0 = S0 + (int64_t)blockIdx.x * blockDim.x; s0 < S; s0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = s0 + threadIdx.x;
    const int64_t sw = s0 + (threadIdx.x & ~31);
    while (v + 1 < P.view_hi && sw >= P.ws.view_base[v + 1]) ++v;
    const FieldDev& F = P.v[v].field;
    if (l >= F.L || sw >= S) continue;  // warp-uniform
    bool live = s < S && P.ws.s_ray[s] >= 0;
    float2 g = make_float2(0.0f, 0.0f);
    if (live) {
      g.x = P.ws.dfeat[(int64_t)(2 * l) * S_cap + s] * scale;
      g.y = P.ws.dfeat[(int64_t)(2 * l + 1) * S_cap + s] * scale;
      live = (g.x != 0.0f) || (g.y != 0.0f);
    }
    Corners c;
    if (live) {
      level_corners(F, l, make_float3(P.ws.s_vc[s], P.ws.s_vc[S_cap + s], P.ws.s_vc[2 * S_cap + s]), c);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c.idx[k] = 0;
        c.w[k] = 0.0f;
      }
    }
    float2* gt = reinterpret_cast<float2*>(F.grad_tables) + ((size_t)l << F.log2T);
    if (F.res[l] <= P.agg_res) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        scatter_runs(gt, c.idx[k], live, make_float2(c.w[k] * g.x, c.w[k] * g.y));
    } else if (live) {
      scatter_pairs(gt, c, g);
    }
  }
}

cudaError_t launch_encode(const Plan& P, int num_sms, cudaStream_t s) {
  int L = 0;
  for (int v = 0; v < P.n_views; ++v) L = P.v[v].field.L > L ? P.v[v].field.L : L;
  dim3 grid(num_sms * P.tune.encode_ctas_per_sm, L);
  k_encode<<<grid, 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_encode_bwd(const Plan& P, int num_sms, cudaStream_t s) {
  int L = 0;
  for (int v = 0; v < P.n_views; ++v) L = P.v[v].field.L > L ? P.v[v].field.L : L;
  dim3 grid(num_sms * P.tune.encode_bwd_ctas_per_sm, L);
  k_encode_bwd<<<grid, 256, 0, s>>>(P);
  return cudaGetLastError();
}

// One launch per group of consecutive views that share a field.
template <class Launch>
cudaError_t per_field(const Plan& P, Launch launch) {
  Plan Q = P;
  int lo = 0;
  while (lo < P.n_views) {
    int hi = lo + 1;
    while (hi < P.n_views && P.v[hi].field.tables == P.v[lo].field.tables) ++hi;
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

// ------------------------------------------------------------------ single step
__global__ void __launch_bounds__(256) k_encode_points(const __grid_constant__ FieldDev F, int64_t n,
                                                       const float* __restrict__ x, float* feat, uint32_t* idx) {
  const int l = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Corners c;
    level_corners(F, l, make_float3(x[i], x[n + i], x[2 * n + i]), c);
    const float2 f = level_feature(F, l, c);
    feat[(int64_t)(2 * l) * n + i] = f.x;
    feat[(int64_t)(2 * l + 1) * n + i] = f.y;
    if (idx) {
#pragma unroll
      for (int k = 0; k < 8; ++k) idx[(int64_t)(l * 8 + k) * n + i] = c.idx[k];
    }
  }
}

cudaError_t launch_encode_points(const FieldDev& f, int64_t n, const float* x, float* feat, uint32_t* idx,
                                 cudaStream_t s) {
  if (n > 0) {
    dim3 grid(min(ceil_div(n, 256), 4096), f.L);
    k_encode_points<<<grid, 256, 0, s>>>(f, n, x, feat, idx);
  }
  return cudaGetLastError();
}

}  // namespace invr
