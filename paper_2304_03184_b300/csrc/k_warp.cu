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
// single-precision rounding of the keys and of the cell assignment), so scanning the list
// with the same keys and tie rule (key, then node index) as a scan of all nodes selects the
// same K nodes.  The list is sorted by distance from the cell centre, and the scan stops at
// the first entry whose distance bound rules out it and every later one (knn.cuh): about 6
// of a list's 11 entries are visited on the human workloads.  Cells whose list exceeds the
// capacity, and points outside the box, fall back to scanning all nodes.  This is the
// default; the approximate look-up tables of Sec. 4.2 ("On-the-fly Radiance Fields", built
// in k_lut.cu) replace the search when a graph has them.
//
// Bound: FP32 ALU and issue (about 10 operations per candidate key, the blend's ~150 per
// sample) plus node reads from shared memory.
#include "tc_ptx.cuh"
#include "warp.cuh"

namespace invr {

// Work items are chunks of kWarpChunk consecutive sample slots, taken from a per-launch counter
// by the CTAs resident on the SMs.  Within a chunk, the samples of each view in turn; a human
// view searched without look-up tables reads its nodes' live positions from a copy in shared
// memory (one bulk copy of the packed float4 records when the CTA's view changes), when it
// has at most smem_nodes nodes.  The copy's wait is bounded: on a time-out the CTA flags the
// status word, waits (bounded) for the copy to land and returns.
constexpr int kWarpChunk = 4096;
constexpr uint32_t kWarpDrainLimit = 1u << 22;

template <int KMAX>
__global__ void __launch_bounds__(256, KMAX <= 4 ? 4 : 1) k_warp(const __grid_constant__ Plan P, int smem_nodes) {
  extern __shared__ __align__(16) float4 s_nodes[];
  __shared__ int32_t vb[kMaxViews + 1];
  __shared__ int64_t s_item;
  __shared__ __align__(8) uint64_t s_nbar;  // node copy landed
  const int64_t S_cap = P.ws.S_cap;
  if (P.ws.view_base[P.n_views] > S_cap) return;
  if (threadIdx.x <= P.n_views) vb[threadIdx.x] = P.ws.view_base[threadIdx.x];
  const uint32_t nbar = tc::smem_u32(&s_nbar);
  if (threadIdx.x == 0) tc::mbar_init(nbar, 1);
  uint32_t nphase = 0;
  const int64_t S = P.ws.view_base[P.n_views];
  const int64_t n_items = (S + kWarpChunk - 1) / kWarpChunk;
  int staged = -1;
  for (;;) {
    __syncthreads();  // s_item consumed, shared node reads of the last item done
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(P.ws.tickets + kTicketWarp, 1u);
    __syncthreads();
    const int64_t c0 = s_item * kWarpChunk;
    if (c0 >= S) break;
    const int64_t c1 = min(S, c0 + kWarpChunk);
    for (int v = 0; v < P.n_views; ++v) {
      const int64_t lo = max(c0, (int64_t)vb[v]), hi = min(c1, (int64_t)vb[v + 1]);
      if (lo >= hi) continue;  // block-uniform
      const WarpDev& W = P.v[v].warp;
      const bool in_smem = W.mode == 1 && !W.lut_live && W.n_nodes <= smem_nodes;
      if (in_smem && staged != v) {
        __syncthreads();  // the block's reads of the previous copy are done
        const uint32_t bytes = (uint32_t)W.n_nodes * (uint32_t)sizeof(float4);  // 16-byte records
        if (threadIdx.x == 0) {
          tc::fence_smem_to_async();
          tc::mbar_expect_tx(nbar, bytes);
          tc::bulk_g2s(tc::smem_u32(s_nodes), W.x_live, bytes, nbar);
        }
        const bool got = tc::mbar_wait(nbar, nphase, P.wait_limit);
        if (!__syncthreads_and(got)) {
          if (threadIdx.x == 0) {
            flag_status(P.status, kStatusTimeout);
            if (!tc::mbar_wait(nbar, nphase, kWarpDrainLimit)) flag_status(P.status, kStatusDrainTimeout);
          }
          __syncthreads();
          return;
        }
        nphase ^= 1u;
        staged = v;
      }
      for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        const int g = P.ws.s_ray[s];
        float3 vc = make_float3(0.f, 0.f, 0.f);
        if (g >= 0) {
          const float3 p = make_float3(P.ws.s_pos[s], P.ws.s_pos[S_cap + s], P.ws.s_pos[2 * S_cap + s]);
          int64_t cell = 0;
          const uint32_t n = (W.mode == 0 || W.lut_live) ? 0u : knn_locate(W, p, cell);
          vc = in_smem ? warp_point_upto<KMAX, true>(W, s_nodes, p, cell, n)
                       : warp_point_upto<KMAX>(W, W.x_live, p, cell, n);
        }
        P.ws.s_vc[s] = vc.x;
        P.ws.s_vc[S_cap + s] = vc.y;
        P.ws.s_vc[2 * S_cap + s] = vc.z;
      }
    }
  }
  (void)n_items;
}

// Shared memory for the node copies: the largest human view's nodes, up to kWarpSmemBytes.
constexpr int kWarpSmemBytes = 48 * 1024;

cudaError_t launch_warp(const Plan& P, int num_sms, cudaStream_t s) {
  int kmax = 0, nmax = 0;
  for (int v = 0; v < P.n_views; ++v)
    if (P.v[v].warp.mode == 1) {
      kmax = max(kmax, P.v[v].warp.K);
      if (!P.v[v].warp.lut_live && P.v[v].warp.n_nodes * 16 <= kWarpSmemBytes) nmax = max(nmax, P.v[v].warp.n_nodes);
    }
  cudaError_t e = cudaMemsetAsync(P.ws.tickets + kTicketWarp, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)nmax * sizeof(float4);
  if (kmax <= 4)
    k_warp<4><<<num_sms * P.tune.warp_ctas_per_sm, 256, smem, s>>>(P, nmax);
  else
    k_warp<8><<<num_sms * P.tune.warp_ctas_per_sm, 256, smem, s>>>(P, nmax);
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

cudaError_t preload_warp_points() {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, k_warp_points);
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

// One warp per grid cell of resolution G: K-th nearest distance from the cell centre, then
// every node within d_K + 2 rho (with margin).  Built in two levels: a G/2 grid scans all
// nodes; a G cell scans only its parent's list, which holds every node it needs -- the
// child's K nearest are among the parent's (the child centre is a point of the parent cell),
// and a node within d_K(c') + 2 rho' of the child centre c' lies within d_K(c) + 2 rho of the
// parent centre c, because d_K is 1-Lipschitz, |c - c'| = rho / 2 and rho' = rho / 2.  The
// coarse lists (build scratch only: node ids in index order) hold 4x the fine capacity, so
// few parents overflow; a child of an overflowed parent scans all nodes.  A fine list
// (REFINE) is sorted by the entries (r_lo << 16) | id, r_lo a lower bound of the node's
// distance from the cell centre in units of kKnnRUnit (the scan's early stop), and ends with
// kKnnEnd when shorter than cap; its first kKnnHead entries are copied into the cell's head
// (kKnnEnd-padded), whose first entry is kKnnHeadOverflow when the list overflowed.  The
// coarse level (!REFINE) writes ids in index order and a count per cell.
template <int K, int G, bool REFINE>
__global__ void __launch_bounds__(256) k_knn_grid_build(const float4* __restrict__ x, int n, int cap, int pcap,
                                                        const uint16_t* __restrict__ pcand,
                                                        const uint16_t* __restrict__ pcand_n, void* cand_out,
                                                        uint16_t* cand_n, uint32_t* cand_head) {
  constexpr float H = 2.0f / G;
  constexpr float Rho = 0.8660254037844386f * H;
  __shared__ uint32_t srt[8][kKnnMaxCap];  // a fine cell's entries before sorting (one row per warp)
  const int lane = threadIdx.x & 31;
  uint32_t* mine_row = srt[threadIdx.x >> 5];
  const int64_t n_cells = (int64_t)G * G * G;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = warp0; cell < n_cells; cell += n_warps) {
    const int ix = (int)(cell % G), iy = (int)((cell / G) % G), iz = (int)(cell / (G * G));
    const float cx = -1.0f + (ix + 0.5f) * H, cy = -1.0f + (iy + 0.5f) * H, cz = -1.0f + (iz + 0.5f) * H;
    // source of candidates: all nodes, or the parent cell's list
    const uint16_t* src = nullptr;
    int m = n;
    if (REFINE) {
      const int64_t pc = (ix >> 1) + (int64_t)(G / 2) * ((iy >> 1) + (int64_t)(G / 2) * (iz >> 1));
      const uint16_t pn = __ldg(pcand_n + pc);
      if (pn != kKnnOverflow) {
        src = pcand + pc * pcap;
        m = pn;
      }
    }
    float best[K];
#pragma unroll
    for (int k = 0; k < K; ++k) best[k] = INFINITY;
    for (int j = lane; j < m; j += 32) {
      const int i = src ? (int)__ldg(src + j) : j;
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
      float mn = best[0];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      const unsigned who = __ballot_sync(0xffffffffu, best[0] == mn);
      if (lane == __ffs(who) - 1) {
#pragma unroll
        for (int j = 0; j + 1 < K; ++j) best[j] = best[j + 1];
        best[K - 1] = INFINITY;
      }
      kth = mn;
    }
    const float rad = (sqrtf(kth) + 2.0f * Rho) * 1.001f + 1e-4f;
    const float rad2 = rad * rad;
    int count = 0;
    for (int base = 0; base < m; base += 32) {
      const int j = base + lane;
      bool in = false;
      int i = 0;
      float d2 = 0.0f;
      if (j < m) {
        i = src ? (int)__ldg(src + j) : j;
        const float4 p = __ldg(x + i);
        const float dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
        d2 = dx * dx + dy * dy + dz * dz;
        in = d2 <= rad2;
      }
      const unsigned mk = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = count + __popc(mk & ((1u << lane) - 1u));
        if (pos < cap) {
          if (REFINE) {
            // r rounded down by a margin covering the FP32 evaluation of the distance
            const float r = fmaxf(sqrtf(d2) * (1.0f - 1e-6f) - 1e-6f, 0.0f);
            const uint32_t rq = (uint32_t)fminf(floorf(r * (1.0f / kKnnRUnit)), 65535.0f);
            mine_row[pos] = (rq << 16) | (uint32_t)i;
          } else {
            static_cast<uint16_t*>(cand_out)[cell * cap + pos] = (uint16_t)i;
          }
        }
      }
      count += __popc(mk);
    }
    if (REFINE && count <= cap) {
      // rank sort of the (unique) entries, then the list in ascending order
      __syncwarp();
      uint32_t e[kKnnMaxCap / 32];
      int rank[kKnnMaxCap / 32];
#pragma unroll
      for (int t = 0; t < kKnnMaxCap / 32; ++t) {
        const int j = lane + 32 * t;
        e[t] = j < count ? mine_row[j] : 0u;
        rank[t] = 0;
      }
      for (int k = 0; k < count; ++k) {
        const uint32_t o = mine_row[k];
#pragma unroll
        for (int t = 0; t < kKnnMaxCap / 32; ++t) rank[t] += o < e[t];
      }
      uint32_t* row = static_cast<uint32_t*>(cand_out) + cell * cap;
      uint32_t* head = cand_head + cell * kKnnHead;
#pragma unroll
      for (int t = 0; t < kKnnMaxCap / 32; ++t)
        if (lane + 32 * t < count) {
          row[rank[t]] = e[t];
          if (rank[t] < kKnnHead) head[rank[t]] = e[t];
        }
      if (lane < kKnnHead && lane >= count) head[lane] = kKnnEnd;
      if (lane == 0 && count < cap) row[count] = kKnnEnd;
      __syncwarp();
    } else if (REFINE && lane == 0) {
      cand_head[cell * kKnnHead] = kKnnHeadOverflow;
    }
    if (!REFINE && lane == 0) cand_n[cell] = count <= cap ? (uint16_t)count : kKnnOverflow;
  }
}

template <int K>
static void grid_build_k(const float4* x, int n, int cap, uint16_t* coarse, uint16_t* coarse_n, uint32_t* cand,
                         uint32_t* cand_head, int grid, cudaStream_t s) {
  const int pcap = kKnnCoarseCapFactor * cap;
  k_knn_grid_build<K, kKnnG / 2, false>
      <<<grid, 256, 0, s>>>(x, n, pcap, 0, nullptr, nullptr, coarse, coarse_n, nullptr);
  k_knn_grid_build<K, kKnnG, true><<<grid, 256, 0, s>>>(x, n, cap, pcap, coarse, coarse_n, cand, nullptr, cand_head);
}

cudaError_t launch_knn_grid_build(const float4* x_live, int n, int K, int cap, uint16_t* coarse, uint16_t* coarse_n,
                                  uint32_t* cand, uint32_t* cand_head, int num_sms, cudaStream_t s) {
  if (cap > kKnnMaxCap || cap % 8 != 0) return cudaErrorInvalidValue;
  const int grid = num_sms * 8;
  switch (K) {
    case 1: grid_build_k<1>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 2: grid_build_k<2>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 3: grid_build_k<3>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 4: grid_build_k<4>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 5: grid_build_k<5>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 6: grid_build_k<6>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    case 7: grid_build_k<7>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
    default: grid_build_k<8>(x_live, n, cap, coarse, coarse_n, cand, cand_head, grid, s); break;
  }
  return cudaGetLastError();
}

}  // namespace invr
