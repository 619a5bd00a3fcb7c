// Ray setup, sampling and occupancy skipping, and the compaction of occupied samples.
//
// Per ray: slab intersection with [-1,1]^3, n_samples uniform midpoint samples, and a
// lookup in the view's 128^3 live-space occupancy bitfield (empty cells carry zero
// density, so their samples are never evaluated).  The occupied samples of all rays of a
// call are compacted into one sample list: per view, rays in order, each ray's samples
// in order; every view's range starts on a kTile boundary so that an MLP tile never
// mixes two fields.  Padding slots carry s_ray = -1.
//
// The count pass records each ray's occupancy bits (word-major, coalesced), so the emit
// pass visits only the occupied samples instead of re-marching the ray.
//
// Bound: HBM reads of the rays (24 B/ray) and bitfield lookups that hit L1/L2 (256 KiB
// per view); writes 4 B per 32 samples of each ray and 24 B per occupied sample.
#include "invr_internal.cuh"

namespace invr {

constexpr int kScanB = 1024;  // rays per scan block

__device__ __forceinline__ void load_ray(const ViewDev& V, int64_t r, float3& o, float3& d) {
  const int64_t n = V.n_rays;
  o = make_float3(__ldg(V.o + r), __ldg(V.o + n + r), __ldg(V.o + 2 * n + r));
  d = make_float3(__ldg(V.d + r), __ldg(V.d + n + r), __ldg(V.d + 2 * n + r));
}

__global__ void __launch_bounds__(256) k_march_count(const __grid_constant__ Plan P) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.total_rays) return;
  const ViewDev& V = P.v[view_of_ray(P, g)];
  float3 o, d;
  load_ray(V, g - V.ray_begin, o, d);
  float tn, dt;
  int cnt = 0;
  uint32_t* bits = P.ws.ray_bits + g;
  const int64_t R_cap = P.ws.R_cap;
  const int words = (P.n_samples + 31) / 32;
  const bool hit = ray_box(o, d, P.n_samples, tn, dt);
  for (int w = 0; w < words; ++w) {
    uint32_t m = 0;
    if (hit) {
      const int j1 = min(32, P.n_samples - 32 * w);
      for (int i = 0; i < j1; ++i) {
        const int j = 32 * w + i;
        if (!V.occ || occupied(V.occ, sample_p(o, d, sample_t(tn, dt, j)))) m |= 1u << i;
      }
    }
    bits[w * R_cap] = m;
    cnt += __popc(m);
  }
  P.ws.ray_count[g] = cnt;
}

// ------------------------------------------------------------------ block scan
__device__ __forceinline__ int block_exclusive_scan(int x, int* warp_tot, int& block_total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == nw - 1) warp_tot[32] = ti;
  }
  __syncthreads();
  int res = warp_tot[wid] + incl - x;
  block_total = warp_tot[32];
  __syncthreads();
  return res;
}

__device__ __forceinline__ void scan_block_range(const Plan& P, int b, int& v, int64_t& g0, int64_t& g1) {
  v = 0;
  while (v + 1 < P.n_views && b >= P.v[v + 1].scan_block_begin) ++v;
  const ViewDev& V = P.v[v];
  g0 = V.ray_begin + (int64_t)(b - V.scan_block_begin) * kScanB;
  g1 = min(g0 + kScanB, V.ray_begin + V.n_rays);
}

__global__ void __launch_bounds__(kScanB) k_scan_blocks(const __grid_constant__ Plan P) {
  __shared__ int warp_tot[33];
  int v;
  int64_t g0, g1;
  scan_block_range(P, blockIdx.x, v, g0, g1);
  const int64_t g = g0 + threadIdx.x;
  int x = g < g1 ? P.ws.ray_count[g] : 0;
  int total;
  block_exclusive_scan(x, warp_tot, total);
  if (threadIdx.x == 0) P.ws.block_sums[blockIdx.x] = total;
}

// One block: per view, turn block sums into global block offsets and lay the views out
// back to back, each padded to a multiple of kTile.
__global__ void __launch_bounds__(kScanB) k_scan_top(const __grid_constant__ Plan P) {
  __shared__ int warp_tot[33];
  int base = 0;
  for (int v = 0; v < P.n_views; ++v) {
    const int b0 = P.v[v].scan_block_begin;
    const int b1 = (v + 1 < P.n_views) ? P.v[v + 1].scan_block_begin : P.n_scan_blocks;
    int carry = 0;
    for (int c = b0; c < b1; c += kScanB) {
      const int b = c + threadIdx.x;
      int x = b < b1 ? P.ws.block_sums[b] : 0;
      int total;
      int ex = block_exclusive_scan(x, warp_tot, total);
      if (b < b1) P.ws.block_sums[b] = base + carry + ex;
      carry += total;
    }
    if (threadIdx.x == 0) {
      P.ws.view_base[v] = base;
      P.ws.view_count[v] = carry;
    }
    base += (carry + kTile - 1) / kTile * kTile;
  }
  if (threadIdx.x == 0) {
    P.ws.view_base[P.n_views] = base;
    if ((int64_t)base > P.ws.S_cap) flag_status(P.status, kStatusOverflow);
  }
}

__global__ void __launch_bounds__(kScanB) k_scan_final(const __grid_constant__ Plan P) {
  __shared__ int warp_tot[33];
  int v;
  int64_t g0, g1;
  scan_block_range(P, blockIdx.x, v, g0, g1);
  const int64_t g = g0 + threadIdx.x;
  int x = g < g1 ? P.ws.ray_count[g] : 0;
  int total;
  int ex = block_exclusive_scan(x, warp_tot, total);
  if (g < g1) P.ws.ray_first[g] = P.ws.block_sums[blockIdx.x] + ex;
}

__global__ void __launch_bounds__(256) k_march_emit(const __grid_constant__ Plan P) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;  // overflow flagged by the scan
  // padding slots at the end of each view's range
  if (g < (int64_t)P.n_views * kTile) {
    const int v = (int)(g / kTile);
    const int64_t slot = (int64_t)P.ws.view_base[v] + P.ws.view_count[v] + (g % kTile);
    if (slot < P.ws.view_base[v + 1]) {
      P.ws.s_ray[slot] = -1;
      P.ws.s_t[slot] = 0.0f;
      P.ws.s_pos[slot] = 0.0f;
      P.ws.s_pos[S_cap + slot] = 0.0f;
      P.ws.s_pos[2 * S_cap + slot] = 0.0f;
    }
  }
  if (g >= P.total_rays) return;
  const int cnt = P.ws.ray_count[g];
  if (cnt == 0) return;
  const ViewDev& V = P.v[view_of_ray(P, g)];
  float3 o, d;
  load_ray(V, g - V.ray_begin, o, d);
  float tn, dt;
  ray_box(o, d, P.n_samples, tn, dt);
  int64_t s = P.ws.ray_first[g];
  const uint32_t* bits = P.ws.ray_bits + g;
  const int words = (P.n_samples + 31) / 32;
  for (int w = 0; w < words; ++w) {
    // the occupied samples recorded by the count pass, in order
    for (uint32_t m = bits[w * P.ws.R_cap]; m; m &= m - 1) {
      const int j = 32 * w + __ffs(m) - 1;
      const float t = sample_t(tn, dt, j);
      const float3 p = sample_p(o, d, t);
      P.ws.s_ray[s] = (int32_t)g;
      P.ws.s_t[s] = t;
      P.ws.s_pos[s] = p.x;
      P.ws.s_pos[S_cap + s] = p.y;
      P.ws.s_pos[2 * S_cap + s] = p.z;
      ++s;
    }
  }
}

cudaError_t launch_march_count(const Plan& P, cudaStream_t s) {
  k_march_count<<<ceil_div(P.total_rays, 256), 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_scan(const Plan& P, cudaStream_t s) {
  k_scan_blocks<<<P.n_scan_blocks, kScanB, 0, s>>>(P);
  k_scan_top<<<1, kScanB, 0, s>>>(P);
  k_scan_final<<<P.n_scan_blocks, kScanB, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_march_emit(const Plan& P, cudaStream_t s) {
  const int64_t n = P.total_rays > (int64_t)P.n_views * kTile ? P.total_rays : (int64_t)P.n_views * kTile;
  k_march_emit<<<ceil_div(n, 256), 256, 0, s>>>(P);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ single step
__global__ void __launch_bounds__(256) k_ray_samples(int64_t n_rays, const float* __restrict__ o_,
                                                     const float* __restrict__ d_, int n_samples,
                                                     const uint32_t* __restrict__ occ, int32_t* count,
                                                     float* t_out, float* p_out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  const float3 o = make_float3(o_[r], o_[n_rays + r], o_[2 * n_rays + r]);
  const float3 d = make_float3(d_[r], d_[n_rays + r], d_[2 * n_rays + r]);
  const int64_t RS = n_rays * n_samples;
  float tn, dt;
  int k = 0;
  if (ray_box(o, d, n_samples, tn, dt)) {
    for (int j = 0; j < n_samples; ++j) {
      const float t = sample_t(tn, dt, j);
      const float3 p = sample_p(o, d, t);
      if (occ && !occupied(occ, p)) continue;
      const int64_t i = r * n_samples + k;
      t_out[i] = t;
      p_out[i] = p.x;
      p_out[RS + i] = p.y;
      p_out[2 * RS + i] = p.z;
      ++k;
    }
  }
  count[r] = k;
}

cudaError_t launch_ray_samples(int64_t n_rays, const float* o, const float* d, int n_samples, const uint32_t* occ,
                               int32_t* count, float* t, float* p, cudaStream_t s) {
  if (n_rays > 0) k_ray_samples<<<ceil_div(n_rays, 256), 256, 0, s>>>(n_rays, o, d, n_samples, occ, count, t, p);
  return cudaGetLastError();
}

}  // namespace invr
