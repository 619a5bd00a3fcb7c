// Pose-conditioned deformation net (Sec. 4.2) forward on the 5th-generation tensor cores:
// BF16 operands, FP32 accumulation in tensor memory.
//
//   X [128 x Kf] (the net's hash features of v_t, Kf = n_feat padded to 16)
//     -> D = X W_1f^T (N = H) -> + pose bias, ReLU -> H (smem, BF16)
//     -> D = H W_k^T (N = H) -> ReLU -> H        (k = 2..n_hidden)
//     -> D = H W_out^T (N = 16, rows 3..15 zero) -> delta v; v_c = v_t + delta v.
//
// One CTA = 128 threads (one warpgroup) per SM; thread t owns sample t of a tile (row t of
// every MMA, lane t of tensor memory).  Every layer's weights are staged once per net as
// BF16 K-major operands (108 KB at 32 / 4 x 128).  Two tiles are in flight: while the
// tensor core runs one tile's layer, the threads run the other tile's epilogue (tensor
// memory -> bias, ReLU -> next operand row).  Waits are bounded; a timeout sets the status
// word, drains this CTA's MMAs (bounded) and frees its tensor memory.
#include "invr_internal.cuh"
#include "tc_ptx.cuh"

namespace invr {

namespace {

constexpr int kTM = 128;
constexpr int kThreads = 128;
constexpr int kH = kDeformMaxHidden;        // 128
constexpr int kKf = kDeformMaxFeat;         // 32
constexpr uint32_t kTmemCols = 512;         // per slot: D at 256 s + 0 (H cols), out at 256 s + 128 (16)
constexpr uint32_t kDrainLimit = 1u << 22;

// shared-memory plan (bytes)
constexpr uint32_t OFF_W1 = 0;                                   // [H][Kf]
constexpr uint32_t OFF_WH = OFF_W1 + kH * kKf * 2;               // 3 x [H][H]
constexpr uint32_t OFF_WO = OFF_WH + 3 * kH * kH * 2;            // [16][H]
constexpr uint32_t OFF_X = OFF_WO + 16 * kH * 2;                 // 2 x [128][Kf]
constexpr uint32_t OFF_HB = OFF_X + 2 * kTM * kKf * 2;           // 2 x [128][H]
constexpr uint32_t OFF_BIAS = OFF_HB + 2 * kTM * kH * 2;         // 2 x [H] floats
constexpr uint32_t OFF_MISC = OFF_BIAS + 2 * kH * 4;             // 2 mbarriers + TMEM base
constexpr uint32_t kSmem = OFF_MISC + 64 + 1024;

__device__ __forceinline__ int view_of_slot(const Plan& P, int64_t s) {
  int v = 0;
  while (v + 1 < P.n_views && s >= P.ws.view_base[v + 1]) ++v;
  return v;
}

__device__ __forceinline__ int64_t layer_offset(const DeformDev& D, int layer) {
  const int64_t n_in = D.n_feat + D.pose_dim;
  if (layer == 0) return 0;
  return (int64_t)D.hidden * n_in + (int64_t)(layer - 1) * D.hidden * D.hidden;
}

// dst = W (rows [0, N), columns [k0, k0 + K) of a row-major [.][ldw] matrix; zero rows
// from n_valid on and zero columns from k_valid on) as a K-major BF16 operand.
__device__ void stage(uint8_t* dst, const float* __restrict__ W, int N, int K, int ldw, int n_valid, int k_valid) {
  for (int e = threadIdx.x; e < N * K / 2; e += kThreads) {
    const int n = (2 * e) / K, k = (2 * e) % K;
    const float a = (n < n_valid && k < k_valid) ? __ldg(W + (int64_t)n * ldw + k) : 0.0f;
    const float b = (n < n_valid && k + 1 < k_valid) ? __ldg(W + (int64_t)n * ldw + k + 1) : 0.0f;
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_offset(n, k, K)) = tc::pack2<true>(a, b);
  }
}

__device__ __forceinline__ void issue(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, true);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

__device__ __forceinline__ void operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
}

struct Slot {
  int64_t s0 = -1;      // first sample of the tile, -1 = no tile
  int view = 0;
};

__global__ void __launch_bounds__(kThreads, 1) k_deform_fwd_tc(const __grid_constant__ Plan P) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  const int t = threadIdx.x, warp = t >> 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 16);
  const uint32_t mbar0 = tc::smem_u32(sm + OFF_MISC);
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) {
    tc::mbar_init(mbar0, 1);
    tc::mbar_init(mbar0 + 8, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

  // tiles of views with a net, in order; this CTA takes every gridDim.x-th one, two at a time
  const int64_t n_tiles = S / kTM;
  const float* loaded = nullptr;
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};  // an MMA commit of the slot not yet waited for
  bool ok = true;
  int64_t next = blockIdx.x;
  auto next_tile = [&](Slot& sl) {
    sl.s0 = -1;
    while (next < n_tiles) {
      const int64_t s0 = next * kTM;
      next += gridDim.x;
      const int v = view_of_slot(P, s0);
      if (P.v[v].has_deform && P.v[v].deform.tc) {
        sl.s0 = s0;
        sl.view = v;
        return;
      }
    }
  };
  Slot slot[2];
  while (ok) {
    next_tile(slot[0]);
    next_tile(slot[1]);
    if (slot[0].s0 < 0) break;
    // both tiles of a pair use the net of the first (a second tile of another net waits)
    const DeformDev& D = P.v[slot[0].view].deform;
    if (slot[1].s0 >= 0 && P.v[slot[1].view].deform.weights != D.weights) {
      next -= gridDim.x;  // hand the tile back: it starts the next pair
      slot[1].s0 = -1;
    }
    const int H = D.hidden, n = D.n_hidden;
    const int Kf = (D.n_feat + 15) / 16 * 16;
    if (D.weights != loaded) {
      __syncthreads();
      const int n_in = D.n_feat + D.pose_dim;
      stage(sm + OFF_W1, D.weights, H, Kf, n_in, H, D.n_feat);
      for (int l = 1; l < n; ++l) stage(sm + OFF_WH + (l - 1) * kH * kH * 2, D.weights + layer_offset(D, l), H, H, H, H, H);
      stage(sm + OFF_WO, D.weights + layer_offset(D, n), 16, H, H, 3, H);
      loaded = D.weights;
    }
    // operands of both tiles: features (FP32 feature-major) -> BF16 rows, pose bias
    for (int j = 0; j < 2; ++j) {
      if (slot[j].s0 < 0) continue;
      const int64_t s0 = slot[j].s0;
      uint8_t* X = sm + OFF_X + j * kTM * kKf * 2;
      for (int k = 0; k < Kf; k += 8) {
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          x[i] = k + i < D.n_feat ? P.ws.feat_d[(int64_t)(k + i) * S_cap + s0 + t] : 0.0f;
        uint4 q;
        q.x = tc::pack2<true>(x[0], x[1]);
        q.y = tc::pack2<true>(x[2], x[3]);
        q.z = tc::pack2<true>(x[4], x[5]);
        q.w = tc::pack2<true>(x[6], x[7]);
        *reinterpret_cast<uint4*>(X + tc::kmajor_offset(t, k, Kf)) = q;
      }
      float* bias = reinterpret_cast<float*>(sm + OFF_BIAS) + j * kH;
      for (int o = t; o < H; o += kThreads) bias[o] = P.v[slot[j].view].deform.pose_bias[o];
    }
    operands_ready();
    if (t == 0) {
      tc::fence_after_sync();
      for (int j = 0; j < 2; ++j) {
        if (slot[j].s0 < 0) continue;
        issue(tmem + 256 * j, sbase + OFF_X + j * kTM * kKf * 2, sbase + OFF_W1, Kf, H);
        tc::commit_to(mbar0 + 8 * j);
      }
    }
    for (int j = 0; j < 2; ++j) pending[j] = slot[j].s0 >= 0;
    // layers 1..n: epilogue of layer l of tile j, then issue layer l+1 of tile j
    for (int l = 0; l <= n && ok; ++l) {
      for (int j = 0; j < 2; ++j) {
        if (slot[j].s0 < 0) continue;
        ok = tc::mbar_wait(mbar0 + 8 * j, phase[j], P.wait_limit);
        if (!__syncthreads_and(ok)) {
          ok = false;
          break;
        }
        phase[j] ^= 1u;
        pending[j] = false;
        tc::fence_after_sync();
        const uint32_t row = tmem + 256 * j + lane_off;
        uint8_t* Hb = sm + OFF_HB + j * kTM * kH * 2;
        if (l < n) {
          const float* bias = reinterpret_cast<const float*>(sm + OFF_BIAS) + j * kH;
          for (int c = 0; c < H; c += 16) {
            float v[16];
            tc::tmem_ld16(row + c, v);
            if (l == 0) {
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] += bias[c + i];
            }
            uint4 lo, hi;
            lo.x = tc::pack2<true>(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f));
            lo.y = tc::pack2<true>(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f));
            lo.z = tc::pack2<true>(fmaxf(v[4], 0.f), fmaxf(v[5], 0.f));
            lo.w = tc::pack2<true>(fmaxf(v[6], 0.f), fmaxf(v[7], 0.f));
            hi.x = tc::pack2<true>(fmaxf(v[8], 0.f), fmaxf(v[9], 0.f));
            hi.y = tc::pack2<true>(fmaxf(v[10], 0.f), fmaxf(v[11], 0.f));
            hi.z = tc::pack2<true>(fmaxf(v[12], 0.f), fmaxf(v[13], 0.f));
            hi.w = tc::pack2<true>(fmaxf(v[14], 0.f), fmaxf(v[15], 0.f));
            *reinterpret_cast<uint4*>(Hb + tc::kmajor_offset(t, c, H)) = lo;
            *reinterpret_cast<uint4*>(Hb + tc::kmajor_offset(t, c + 8, H)) = hi;
          }
          operands_ready();
          if (t == 0) {
            tc::fence_after_sync();
            if (l + 1 < n)
              issue(tmem + 256 * j, sbase + OFF_HB + j * kTM * kH * 2, sbase + OFF_WH + l * kH * kH * 2, H, H);
            else
              issue(tmem + 256 * j + 128, sbase + OFF_HB + j * kTM * kH * 2, sbase + OFF_WO, H, 16);
            tc::commit_to(mbar0 + 8 * j);
          }
          pending[j] = true;
        } else {
          float v[16];
          tc::tmem_ld16(row + 128, v);
          const int64_t g = slot[j].s0 + t;
          if (P.ws.s_ray[g] >= 0) {
            P.ws.s_vc[g] = P.ws.s_vt[g] + v[0];
            P.ws.s_vc[S_cap + g] = P.ws.s_vt[S_cap + g] + v[1];
            P.ws.s_vc[2 * S_cap + g] = P.ws.s_vt[2 * S_cap + g] + v[2];
          }
          tc::fence_before_sync();
        }
      }
    }
    __syncthreads();
  }
  if (!ok) {
    if (t == 0) atomicOr(P.status, kStatusTimeout);
    // let this CTA's outstanding MMAs finish (bounded) before their tensor memory is freed
    for (int j = 0; j < 2; ++j)
      if (pending[j]) tc::mbar_wait(mbar0 + 8 * j, phase[j], kDrainLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

cudaError_t launch_deform_forward_tc(const Plan& P, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_deform_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  k_deform_fwd_tc<<<num_sms, kThreads, kSmem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace invr
