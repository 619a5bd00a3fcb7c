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
// pass visits only the occupied samples instead of re-marching the ray; it tests only the
// samples inside the box of the view's occupied cells (k_occ_box, once per call).
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

// Index bounds of each view's occupied cells, as six minima per view: lo x, y, z and -hi x,
// y, z (the workspace is preset to a large value; lo > hi: no occupied cell; a view without
// occupancy gets the whole grid).  Grid (64, n_views): each block reduces 1,024 words of the
// view's bitfield and folds its bounds in with atomicMin.  Bit c of the field is cell (c % 128,
// c / 128 % 128, c / 128^2), so a 32-bit word covers 32 consecutive x cells of one (y, z) row.
constexpr int kOccBoxBlocks = 64;

__global__ void __launch_bounds__(256) k_occ_box(const __grid_constant__ Plan P) {
  __shared__ int part[8][6];
  const int v = blockIdx.y;
  const uint32_t* occ = P.v[v].occ;
  int b[6] = {kOccRes, kOccRes, kOccRes, 1, 1, 1};
  if (!occ) {
    if (blockIdx.x == 0) {
      b[0] = b[1] = b[2] = 0;
      b[3] = b[4] = b[5] = -(kOccRes - 1);
    }
  } else {
    constexpr int kWords = kOccRes * kOccRes * kOccRes / 32;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < kWords; w += gridDim.x * blockDim.x) {
      const uint32_t m = __ldg(occ + w);
      if (!m) continue;
      const int x0 = 32 * (w % (kOccRes / 32)), y = (w / (kOccRes / 32)) % kOccRes, z = w / (kOccRes * kOccRes / 32);
      b[0] = min(b[0], x0 + __ffs(m) - 1);
      b[3] = min(b[3], -(x0 + 31 - __clz(m)));
      b[1] = min(b[1], y);
      b[4] = min(b[4], -y);
      b[2] = min(b[2], z);
      b[5] = min(b[5], -z);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const int r = __reduce_min_sync(0xffffffffu, b[a]);
    if (lane == 0) part[wid][a] = r;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    int r = part[0][a];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = min(r, part[w][a]);
    atomicMin(P.ws.occ_box + 6 * v + a, r);
  }
}

// The samples j0 .. j1 of a ray (tn, dt) that can lie in the box of occupied cells `b` (lo
// x, y, z, -hi x, y, z): the ray's interval inside the box widened by 1e-4 (covering every
// FP32 rounding of a sample position and its cell) plus one sample on each side.  Outside
// it no sample is occupied, so skipping those samples changes no result.  Returns false
// when the ray misses the box.
__device__ __forceinline__ bool occupied_range(const int32_t* b, float3 o, float3 d, float tn, float dt,
                                               int n_samples, int& j0, int& j1) {
  const int lo_i[3] = {b[0], b[1], b[2]}, hi_i[3] = {-b[3], -b[4], -b[5]};
  if (lo_i[0] > hi_i[0]) return false;
  constexpr float kCell = 2.0f / kOccRes, kMargin = 1e-4f;
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  float t0 = -INFINITY, t1 = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = -1.0f + kCell * (float)lo_i[a] - kMargin, hi = -1.0f + kCell * (float)(hi_i[a] + 1) + kMargin;
    if (dd[a] == 0.0f) {
      if (oo[a] < lo || oo[a] > hi) return false;
      continue;
    }
    const float ta = (lo - oo[a]) / dd[a], tb = (hi - oo[a]) / dd[a];
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  }
  if (!(t0 <= t1)) return false;
  const float f0 = floorf((t0 - tn) / dt - 0.5f) - 1.0f, f1 = ceilf((t1 - tn) / dt - 0.5f) + 1.0f;
  j0 = f0 > 0.0f ? (f0 < (float)n_samples ? (int)f0 : n_samples) : 0;
  j1 = f1 < (float)(n_samples - 1) ? (f1 > -1.0f ? (int)f1 : -1) : n_samples - 1;
  return j0 <= j1;
}

// One thread per ray sets up its ray (slab entry, sample spacing, the range of samples that
// can lie in the occupied box).  The warp then tests its 32 rays' samples in one of two ways
// (identical bits: the same per-sample recipe).  Renders: each lane walks its own ray's
// samples -- a warp takes as long as its longest ray, which costs little for image-ordered
// rays of alike lengths.  Training (P.march_coop): the warp takes its rays in turn, one lane
// per sample of a 32-sample word, and a ballot gives the word, so a warp's cost is the sum of
// its rays' words -- training batches draw rays in random order, whose lengths in the box
// differ widely (0.240 -> 0.203 ms on the key-frame batch; the same on the 512x512 render
// cost 0.02 ms).  Rays of more than kCoopWords words (over 256 samples) always walk per thread.
constexpr int kCoopWords = 8;

__global__ void __launch_bounds__(256) k_march_count(const __grid_constant__ Plan P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool real = g < P.total_rays;
  const int64_t R_cap = P.ws.R_cap;
  const int words = (P.n_samples + 31) / 32;
  float3 o = make_float3(0.f, 0.f, 0.f), d = o;
  float tn = 0.0f, dt = 0.0f;
  int j0 = 0, j1 = -1;
  const uint32_t* occ = nullptr;
  if (real) {
    const int v = view_of_ray(P, g);
    const ViewDev& V = P.v[v];
    occ = V.occ;
    load_ray(V, g - V.ray_begin, o, d);
    if (ray_box(o, d, P.n_samples, tn, dt)) {
      if (V.occ)
        occupied_range(P.ws.occ_box + 6 * v, o, d, tn, dt, P.n_samples, j0, j1);
      else
        j1 = P.n_samples - 1;
    }
  }
  uint32_t* bits = P.ws.ray_bits + g;
  if (words > kCoopWords || !P.march_coop) {  // per thread
    if (!real) return;
    int cnt = 0;
    for (int w = 0; w < words; ++w) {
      uint32_t m = 0;
      const int lo = max(j0, 32 * w), hi = min(j1, 32 * w + 31);
      for (int j = lo; j <= hi; ++j)
        if (!occ || occupied(occ, sample_p(o, d, sample_t(tn, dt, j)))) m |= 1u << (j - 32 * w);
      bits[w * R_cap] = m;
      cnt += __popc(m);
    }
    P.ws.ray_count[g] = cnt;
    return;
  }
  uint32_t mine[kCoopWords];  // this lane's ray's words
#pragma unroll
  for (int w = 0; w < kCoopWords; ++w) mine[w] = 0u;
  for (int i = 0; i < 32; ++i) {
    const int a = __shfl_sync(FULL, j0, i), b = __shfl_sync(FULL, j1, i);
    if (a > b) continue;  // warp-uniform: ray i has no sample in the box
    const float3 oi = make_float3(__shfl_sync(FULL, o.x, i), __shfl_sync(FULL, o.y, i), __shfl_sync(FULL, o.z, i));
    const float3 di = make_float3(__shfl_sync(FULL, d.x, i), __shfl_sync(FULL, d.y, i), __shfl_sync(FULL, d.z, i));
    const float tni = __shfl_sync(FULL, tn, i), dti = __shfl_sync(FULL, dt, i);
    const uint32_t* occi = reinterpret_cast<const uint32_t*>(
        __shfl_sync(FULL, reinterpret_cast<unsigned long long>(occ), i));
#pragma unroll
    for (int w = 0; w < kCoopWords; ++w) {
      if (w >= words || 32 * w > b || 32 * w + 31 < a) continue;  // warp-uniform
      const int j = 32 * w + lane;
      const bool in = j >= a && j <= b && (!occi || occupied(occi, sample_p(oi, di, sample_t(tni, dti, j))));
      const uint32_t m = __ballot_sync(FULL, in);
      if (lane == i) mine[w] = m;
    }
  }
  if (!real) return;
  int cnt = 0;
#pragma unroll
  for (int w = 0; w < kCoopWords; ++w)
    if (w < words) {
      bits[w * R_cap] = mine[w];
      cnt += __popc(mine[w]);
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

// One warp per 32 consecutive rays: their occupied samples fill one contiguous range of
// slots per view, which the warp writes 32 slots at a time (coalesced).  For the slot of
// ordinal q within the warp's samples, a binary search over the warp's inclusive prefix
// counts (shuffles) finds its ray r, the (q - first of r)-th set bit of r's occupancy words
// gives the sample index j, and r's ray parameters come from lane r.
__global__ void __launch_bounds__(256) k_march_emit(const __grid_constant__ Plan P) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
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
  const int lane = threadIdx.x & 31;
  const int64_t g0 = g - lane;                       // first ray of this warp
  if (g0 >= P.total_rays) return;                    // warp-uniform
  const bool mine = g < P.total_rays;
  const int cnt = mine ? P.ws.ray_count[g] : 0;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;                            // warp-uniform
  // this lane's ray parameters, for the lanes that emit its samples
  float3 o = make_float3(0.f, 0.f, 0.f), d = o;
  float tn = 0.0f, dt = 0.0f;
  int64_t first = 0;
  if (cnt > 0) {
    const ViewDev& V = P.v[view_of_ray(P, g)];
    load_ray(V, g - V.ray_begin, o, d);
    ray_box(o, d, P.n_samples, tn, dt);
    first = P.ws.ray_first[g];
  }
  const int64_t R_cap = P.ws.R_cap;
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int q = q0 + lane;
    const bool act = q < total;
    // ray r of ordinal q: the first lane whose inclusive count exceeds q
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (lo + hi) >> 1;
      const int c = __shfl_sync(0xffffffffu, incl, mid);
      if (q < c) hi = mid; else lo = mid + 1;
    }
    const int r = lo;
    const int ex = __shfl_sync(0xffffffffu, incl, r) - __shfl_sync(0xffffffffu, cnt, r);
    const float ox = __shfl_sync(0xffffffffu, o.x, r), oy = __shfl_sync(0xffffffffu, o.y, r),
                oz = __shfl_sync(0xffffffffu, o.z, r);
    const float dx = __shfl_sync(0xffffffffu, d.x, r), dy = __shfl_sync(0xffffffffu, d.y, r),
                dz = __shfl_sync(0xffffffffu, d.z, r);
    const float rtn = __shfl_sync(0xffffffffu, tn, r), rdt = __shfl_sync(0xffffffffu, dt, r);
    const int64_t rfirst = __shfl_sync(0xffffffffu, first, r);
    if (!act) continue;
    // the k-th occupied sample of ray g0 + r
    int k = q - ex, j = 0;
    const uint32_t* bits = P.ws.ray_bits + g0 + r;
    for (int w = 0;; ++w) {
      const uint32_t m = bits[w * R_cap];
      const int pc = __popc(m);
      if (k < pc) {
        j = 32 * w + (int)__fns(m, 0, k + 1);
        break;
      }
      k -= pc;
    }
    const float t = sample_t(rtn, rdt, j);
    const float3 p = sample_p(make_float3(ox, oy, oz), make_float3(dx, dy, dz), t);
    const int64_t slot = rfirst + (q - ex);
    P.ws.s_ray[slot] = (int32_t)(g0 + r);
    P.ws.s_t[slot] = t;
    P.ws.s_pos[slot] = p.x;
    P.ws.s_pos[S_cap + slot] = p.y;
    P.ws.s_pos[2 * S_cap + slot] = p.z;
  }
}

// Blocks of two warps for the count and, in training calls, the emit: a warp's cost follows
// its rays' lengths, and a block holds its slot until its slowest warp ends (training rays in
// random order: count 0.203 -> 0.189 ms, emit 0.130 -> 0.124 ms per batched step against
// blocks of 8 warps).  A render's image-ordered rays are alike, and its emit keeps blocks of 8
// warps (43 against 55 us per 512x512 frame in the ncu launch list).
constexpr int kMarchB = 64;

cudaError_t launch_march_count(const Plan& P, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(P.ws.occ_box, 0x7F, 6 * sizeof(int32_t) * P.n_views, s);  // 0x7F7F7F7F
  if (e != cudaSuccess) return e;
  k_occ_box<<<dim3(kOccBoxBlocks, P.n_views), 256, 0, s>>>(P);
  k_march_count<<<ceil_div(P.total_rays, kMarchB), kMarchB, 0, s>>>(P);
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
  const int block = P.march_coop ? kMarchB : 256;
  k_march_emit<<<ceil_div(n, block), block, 0, s>>>(P);
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
