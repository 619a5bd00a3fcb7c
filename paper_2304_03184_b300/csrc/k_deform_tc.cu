// Pose-conditioned deformation net (Sec. 4.2) forward on the 5th-generation tensor cores:
// BF16 operands, FP32 accumulation in tensor memory.
//
//   X [128 x Kf] (the net's hash features of v_t, Kf = n_feat padded to 16)
//     -> D = X W_1f^T (N = H) -> + pose bias, ReLU -> H (smem, BF16)
//     -> D = H W_k^T (N = H) -> ReLU -> H        (k = 2..n_hidden)
//     -> D = H W_out^T (N = 16, rows 3..15 zero) -> delta v; v_c = v_t + delta v.
//
// One CTA per SM; thread t of a warpgroup owns sample t of a tile (row t of every MMA, lane
// t of tensor memory).  Every layer's weights are staged once per net as BF16 K-major
// operands (108 KB at 32 / 4 x 128).  Two tiles are in flight, each owned by its own
// warpgroup, which runs its tile's epilogues while the tensor core runs the other tile's
// layer (in the forward and in the adjoint chain).  Waits
// are bounded; a timeout sets the status word, drains the outstanding MMAs (bounded) and
// frees the tensor memory.
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
constexpr int64_t kHTile = (int64_t)kTM * kH * 2;    // bytes of a stored [128 x 128] operand tile
constexpr int64_t kXTile = (int64_t)kTM * kKf * 2;   // [128 x 32]
constexpr int64_t kGoTile = (int64_t)kTM * 16 * 2;   // [128 x 16]

// shared-memory plan (bytes)
constexpr uint32_t OFF_W1 = 0;                                   // [H][Kf]
constexpr uint32_t OFF_WH = OFF_W1 + kH * kKf * 2;               // 3 x [H][H]
constexpr uint32_t OFF_WO = OFF_WH + 3 * kH * kH * 2;            // [16][H]
constexpr uint32_t OFF_X = OFF_WO + 16 * kH * 2;                 // 2 x [128][Kf]
constexpr uint32_t OFF_HB = OFF_X + 2 * kTM * kKf * 2;           // 2 x [128][H]
constexpr uint32_t OFF_BIAS = OFF_HB + 2 * kTM * kH * 2;         // 2 x [H] floats
constexpr uint32_t OFF_MISC = OFF_BIAS + 2 * kH * 4;             // 2 mbarriers + TMEM base
constexpr uint32_t kSmem = OFF_MISC + 64 + 1024;
// the forward's plan: every weight as 16-bit values directly followed by their rounding
// remainders (the activations live in tensor memory)
constexpr uint32_t F_W1 = 0;                                     // 2 x [H][Kf]
constexpr uint32_t F_WH = F_W1 + 2 * kH * kKf * 2;               // 3 x 2 x [H][H]
constexpr uint32_t F_WO = F_WH + 3 * 2 * kH * kH * 2;            // 2 x [16][H]
constexpr uint32_t F_BIAS = F_WO + 2 * 16 * kH * 2;              // 2 x [H] floats
constexpr uint32_t F_MISC = F_BIAS + 2 * kH * 4;                 // 2 mbarriers + TMEM base
constexpr uint32_t kSmemF = F_MISC + 64 + 1024;
static_assert(kSmemF <= 227 * 1024, "the forward's weights fit one CTA");

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
template <bool BF16, int NT = kThreads>
__device__ void stage(uint8_t* dst, const float* __restrict__ W, int N, int K, int ldw, int n_valid, int k_valid) {
  for (int e = threadIdx.x; e < N * K / 2; e += NT) {
    const int n = (2 * e) / K, k = (2 * e) % K;
    const float a = (n < n_valid && k < k_valid) ? __ldg(W + (int64_t)n * ldw + k) : 0.0f;
    const float b = (n < n_valid && k + 1 < k_valid) ? __ldg(W + (int64_t)n * ldw + k + 1) : 0.0f;
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_offset(n, k, K)) = tc::pack2<BF16>(a, b);
  }
}

// The same as 16-bit values at dst and their rounding remainders at dst + N K 2 bytes (by
// the NT threads of the block).
template <bool BF16, int NT = kThreads>
__device__ void stage_split(uint8_t* dst, const float* __restrict__ W, int N, int K, int ldw, int n_valid,
                            int k_valid) {
  uint8_t* lo = dst + N * K * 2;
  for (int e = threadIdx.x; e < N * K / 2; e += NT) {
    const int n = (2 * e) / K, k = (2 * e) % K;
    const float a = (n < n_valid && k < k_valid) ? __ldg(W + (int64_t)n * ldw + k) : 0.0f;
    const float b = (n < n_valid && k + 1 < k_valid) ? __ldg(W + (int64_t)n * ldw + k + 1) : 0.0f;
    uint32_t h, l;
    tc::split2<BF16>(a, b, h, l);
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_offset(n, k, K)) = h;
    *reinterpret_cast<uint32_t*>(lo + tc::kmajor_offset(n, k, K)) = l;
  }
}

template <bool BF16>
__device__ __forceinline__ void issue(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, BF16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

// Slot tensor memory: accumulator [0, 128) (the output layer's in [0, 16)), the current
// layer's A operand as 16-bit values [128, 192) and rounding remainders [192, 256).
constexpr uint32_t T_HI = 128, T_LO = 192;

// One thread: D = A W^T with A in tensor memory as values and remainders (8 columns per K
// step of 16) and W in shared memory as values and remainders (N K 2 bytes apart):
// hi*hi + lo*hi + hi*lo, both operands to about twice the 16-bit precision.
template <bool BF16>
__device__ __forceinline__ void issue_split(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_saddr, int K,
                                            int N) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, BF16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    const uint64_t bl = tc::smem_desc(b_saddr + N * K * 2 + kk * 256, 128, K * 16);
    tc::mma_f16_ts(d_tmem, a_hi + kk * 8, bd, idesc, kk > 0 ? 1u : 0u);
    tc::mma_f16_ts(d_tmem, a_lo + kk * 8, bd, idesc, 1u);
    tc::mma_f16_ts(d_tmem, a_hi + kk * 8, bl, idesc, 1u);
  }
}

struct Slot {
  int64_t s0 = -1;      // first sample of the tile, -1 = no tile
  int view = 0;
};

// The forward's two tile slots belong to two warpgroups (256 threads): warpgroup g runs slot
// g's whole layer chain -- its epilogues and, from its first thread, its MMAs -- with its own
// named barrier (id 1 + g), so one slot's epilogue overlaps the other's MMAs on separate warps.
constexpr int kThreadsF = 256;

__device__ __forceinline__ void wg_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Named-barrier AND over the 128 threads of a warpgroup.
__device__ __forceinline__ bool wg_and(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsF, 1) k_deform_fwd_tc(const __grid_constant__ Plan P) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  const int t = threadIdx.x, warp = t >> 5;
  const int g = t >> 7, tl = t & 127;  // warpgroup = tile slot, thread within it
  const int bar = 1 + g;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + F_MISC + 16);
  const uint32_t mbar = tc::smem_u32(sm + F_MISC) + 8 * g;
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(sm + F_MISC), 1);
    tc::mbar_init(tc::smem_u32(sm + F_MISC) + 8, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row = tmem + 256 * g + ((uint32_t)((warp & 3) * 32) << 16);  // this thread's lane of its slot

  // tiles of views with a net, in order; this CTA takes every gridDim.x-th one, two at a time
  const int64_t n_tiles = S / kTM;
  const float* loaded = nullptr;
  uint32_t phase = 0u;
  bool pending = false;  // an MMA commit of this warpgroup's slot not yet waited for
  bool ok = true;
  int64_t next = blockIdx.x;
  auto next_tile = [&](Slot& sl) {
    sl.s0 = -1;
    while (next < n_tiles) {
      const int64_t s0 = next * kTM;
      next += gridDim.x;
      const int v = view_of_slot(P, s0);
      if (P.v[v].has_deform && P.v[v].deform.tc == (BF16 ? 2 : 1)) {
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
      stage_split<BF16, kThreadsF>(sm + F_W1, D.weights, H, Kf, n_in, H, D.n_feat);
      for (int l = 1; l < n; ++l)
        stage_split<BF16, kThreadsF>(sm + F_WH + (l - 1) * 2 * kH * kH * 2, D.weights + layer_offset(D, l), H, H, H,
                                     H, H);
      stage_split<BF16, kThreadsF>(sm + F_WO, D.weights + layer_offset(D, n), 16, H, H, 3, H);
      tc::fence_smem_to_async();
      __syncthreads();
      loaded = D.weights;
    }
    const Slot sl = slot[g];
    if (sl.s0 >= 0) {
      const int64_t s0 = sl.s0;
      // layer 1's operand: the features (FP32 feature-major) as 16-bit values and rounding
      // remainders in the slot's tensor memory, and the pose bias
      float xr[kKf];
#pragma unroll
      for (int k = 0; k < kKf; ++k) xr[k] = k < D.n_feat ? P.ws.feat_d[(int64_t)k * S_cap + s0 + tl] : 0.0f;
      // every global read of the tile is issued here, ahead of its chain: the pose bias beside
      // the features, the output stage's inputs (sample liveness, v_t) under the MMAs (the
      // same reads at their points of use cost 0.28 of 1.56 ms per step)
      const float pb = tl < H ? P.v[sl.view].deform.pose_bias[tl] : 0.0f;  // H <= 128
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) tc::split2<BF16>(xr[2 * c], xr[2 * c + 1], hi[c], lo[c]);
      const int64_t gs = s0 + tl;
      const bool live = P.ws.s_ray[gs] >= 0;
      const float vt0 = P.ws.s_vt[gs], vt1 = P.ws.s_vt[S_cap + gs], vt2 = P.ws.s_vt[2 * S_cap + gs];
      if (Kf == 32) {
        tc::tmem_st16(row + T_HI, hi);
        tc::tmem_st16(row + T_LO, lo);
      } else {
        uint32_t h8[8], l8[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          h8[c] = hi[c];
          l8[c] = lo[c];
        }
        tc::tmem_st8(row + T_HI, h8);
        tc::tmem_st8(row + T_LO, l8);
      }
      if (P.deform_store) {
        for (int k = 0; k < Kf; k += 8)
          *reinterpret_cast<uint4*>(P.ws.def_x + (s0 / kTM) * kXTile + tc::kmajor_offset(tl, k, Kf)) =
              make_uint4(hi[k / 2], hi[k / 2 + 1], hi[k / 2 + 2], hi[k / 2 + 3]);
      }
      float* bias = reinterpret_cast<float*>(sm + F_BIAS) + g * kH;
      if (tl < H) bias[tl] = pb;
      tc::fence_smem_to_async();
      tc::fence_before_sync();
      wg_sync(bar);
      if (tl == 0) {
        tc::fence_after_sync();
        issue_split<BF16>(tmem + 256 * g, tmem + 256 * g + T_HI, tmem + 256 * g + T_LO, sbase + F_W1, Kf, H);
        tc::commit_to(mbar);
      }
      pending = true;
      // layers 1..n: epilogue of layer l, then issue layer l+1
      for (int l = 0; l <= n; ++l) {
        ok = wg_and(bar, tc::mbar_wait(mbar, phase, P.wait_limit));
        if (!ok) break;
        phase ^= 1u;
        pending = false;
        tc::fence_after_sync();
        if (l < n) {
          const float* bias = reinterpret_cast<const float*>(sm + F_BIAS) + g * kH;
          uint8_t* gh = P.ws.def_h + ((int64_t)l * (S_cap / kTM) + s0 / kTM) * kHTile;
          for (int c = 0; c < H; c += 32) {
            float v[32];
            tc::tmem_ld32(row + c, v);
            if (l == 0) {
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] += bias[c + i];
            }
            uint32_t hh[16], ll[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
              tc::split2<BF16>(fmaxf(v[2 * q], 0.f), fmaxf(v[2 * q + 1], 0.f), hh[q], ll[q]);
            // h_l as the next layer's A operand (values and remainders) and, rounded, for the
            // backward (its weight-gradient operand; its sign is the ReLU decision taken here)
            tc::tmem_st16(row + T_HI + c / 2, hh);
            tc::tmem_st16(row + T_LO + c / 2, ll);
            if (P.deform_store) {
#pragma unroll
              for (int c8 = 0; c8 < 4; ++c8)
                *reinterpret_cast<uint4*>(gh + tc::kmajor_offset(tl, c + 8 * c8, H)) =
                    make_uint4(hh[4 * c8], hh[4 * c8 + 1], hh[4 * c8 + 2], hh[4 * c8 + 3]);
            }
          }
          tc::fence_before_sync();
          wg_sync(bar);
          if (tl == 0) {
            tc::fence_after_sync();
            if (l + 1 < n)
              issue_split<BF16>(tmem + 256 * g, tmem + 256 * g + T_HI, tmem + 256 * g + T_LO,
                                sbase + F_WH + l * 2 * kH * kH * 2, H, H);
            else
              issue_split<BF16>(tmem + 256 * g, tmem + 256 * g + T_HI, tmem + 256 * g + T_LO, sbase + F_WO, H, 16);
            tc::commit_to(mbar);
          }
          pending = true;
        } else {
          float v[16];
          tc::tmem_ld16(row, v);
          if (live) {
            P.ws.s_vc[gs] = vt0 + v[0];
            P.ws.s_vc[S_cap + gs] = vt1 + v[1];
            P.ws.s_vc[2 * S_cap + gs] = vt2 + v[2];
          }
          tc::fence_before_sync();
        }
      }
    }
    ok = __syncthreads_and(ok);  // both slots' chains done (or one gave up)
  }
  if (!ok) {
    if (t == 0) atomicOr(P.status, kStatusTimeout);
    // let this warpgroup's outstanding MMAs finish (bounded) before their tensor memory is freed
    if (tl == 0 && pending && !tc::mbar_wait(mbar, phase, kDrainLimit)) atomicOr(P.status, kStatusDrainTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------------ backward
// Adjoint MMA: D (128 x N) = G (smem, 128 x K, K-major) * W with W the forward weight
// [K rows][N columns] as staged for the forward (K-major in its own layout), read as an
// MN-major operand: column groups 128 B apart, row groups N * 16 B apart.
template <bool BF16>
__device__ __forceinline__ void issue_adjoint(uint32_t d_tmem, uint32_t a_saddr, uint32_t w_saddr, int K, int N) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, BF16) | (1u << 16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(w_saddr + kk * 32 * N, N * 16, 128);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

// Weight-gradient MMA over the 128 samples of a tile: D (M = a_units x N = b_units) (+)=
// A^T B, A and B [128 samples][units] K-major tiles read as MN-major operands (unit groups
// 128 B apart, sample groups units * 16 B apart).
template <bool BF16>
__device__ __forceinline__ void issue_dw(uint32_t d_tmem, uint32_t a_saddr, int a_units, uint32_t b_saddr,
                                         int b_units, bool accumulate) {
  const uint32_t idesc = tc::idesc_f16(kTM, b_units, BF16) | (1u << 15) | (1u << 16);
  for (int kk = 0; kk < kTM / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 32 * a_units, a_units * 16, 128);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 32 * b_units, b_units * 16, 128);
    tc::mma_f16(d_tmem, ad, bd, idesc, (accumulate || kk > 0) ? 1u : 0u);
  }
}

// Per 16-bit half of a stored ReLU output w (each half +0, -0 or positive): 0xFFFF where the
// half is positive, else 0 (one packed half-precision compare).
template <bool BF16>
__device__ __forceinline__ uint32_t positive_halves(uint32_t w) {
  if constexpr (BF16) {
    return __hgt2_mask(*reinterpret_cast<const __nv_bfloat162*>(&w),
                       __nv_bfloat162(__float2bfloat16(0.0f), __float2bfloat16(0.0f)));
  } else {
    return __hgt2_mask(*reinterpret_cast<const __half2*>(&w), __half2(__float2half(0.0f), __float2half(0.0f)));
  }
}

// The adjoint chain: per tile, dL/d(delta v) (the stored dL/dv_c, padded to 16 columns)
// -> g_n = (g_out W_out) . [h_n > 0] -> g_{l} = (g_{l+1} W_{l+1}) . [h_l > 0] -> dL/df =
// g_1 W_1f.  The ReLU masks come from the forward's stored h tiles; every g tile (and the
// padded g_out tile) is stored for the weight-gradient kernel; dL/df is written FP32
// feature-major for the scatter into the net's tables.  Two tiles in flight, as the forward.
template <bool BF16>
__global__ void __launch_bounds__(kThreadsF, 1) k_deform_chain_tc(const __grid_constant__ Plan P) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  const int t = threadIdx.x, warp = t >> 5;
  const int g = t >> 7, tl = t & 127;  // warpgroup = tile slot, thread within it
  const int bar = 1 + g;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 16);
  const uint32_t mbar = tc::smem_u32(sm + OFF_MISC) + 8 * g;
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(sm + OFF_MISC), 1);
    tc::mbar_init(tc::smem_u32(sm + OFF_MISC) + 8, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row = tmem + 256 * g + ((uint32_t)((warp & 3) * 32) << 16);  // this thread's lane of its slot
  const int64_t tiles_cap = S_cap / kTM;
  const int64_t n_tiles = S / kTM;
  const float* loaded = nullptr;
  uint32_t phase = 0u;
  bool pending = false;
  bool ok = true;
  int64_t next = blockIdx.x;
  auto next_tile = [&](Slot& sl) {
    sl.s0 = -1;
    while (next < n_tiles) {
      const int64_t s0 = next * kTM;
      next += gridDim.x;
      const int v = view_of_slot(P, s0);
      if (P.v[v].has_deform && P.v[v].deform.tc == (BF16 ? 2 : 1)) {
        sl.s0 = s0;
        sl.view = v;
        return;
      }
    }
  };
  // The warpgroups meet at a block barrier only where a net's weights are staged: between
  // stagings each runs its slots' chains at its own pace (a warpgroup that gave up walks on
  // without work, so both reach every staging barrier and leave the loop together).
  Slot slot[2];
  while (true) {
    next_tile(slot[0]);
    next_tile(slot[1]);
    if (slot[0].s0 < 0) break;
    const DeformDev& D = P.v[slot[0].view].deform;
    if (slot[1].s0 >= 0 && P.v[slot[1].view].deform.weights != D.weights) {
      next -= gridDim.x;
      slot[1].s0 = -1;
    }
    const int H = kH, n = D.n_hidden, Kf = kKf;
    if (D.weights != loaded) {
      ok = __syncthreads_and(ok);
      if (!ok) break;
      const int n_in = D.n_feat + D.pose_dim;
      stage<BF16, kThreadsF>(sm + OFF_W1, D.weights, H, Kf, n_in, H, D.n_feat);
      for (int l = 1; l < n; ++l)
        stage<BF16, kThreadsF>(sm + OFF_WH + (l - 1) * kH * kH * 2, D.weights + layer_offset(D, l), H, H, H, H, H);
      stage<BF16, kThreadsF>(sm + OFF_WO, D.weights + layer_offset(D, n), 16, H, H, 3, H);
      tc::fence_smem_to_async();
      __syncthreads();
      loaded = D.weights;
    }
    const Slot sl = slot[g];
    if (ok && sl.s0 >= 0) {
      const int64_t T = sl.s0 / kTM;
      // the ReLU mask rows (this thread's row of the stored h tile) of the next stage, loaded
      // one stage ahead so that they arrive under the MMAs (the first stage's beside dL/dv_c)
      uint4 mrow[16];
      if (n >= 1) {
        const uint8_t* hg = P.ws.def_h + ((int64_t)(n - 1) * tiles_cap + T) * kHTile;
#pragma unroll
        for (int c = 0; c < 16; ++c) mrow[c] = __ldg(reinterpret_cast<const uint4*>(hg + tc::kmajor_offset(tl, 8 * c, H)));
      }
      // g_out tile: dL/dv_c (3 columns) padded to 16, in smem and stored
      {
        const int64_t gs = sl.s0 + tl;
        float v[16];
        // scaled by 1 / loss_norm before rounding to 16 bits (the deltas of a mean loss are
        // small enough to lose FP16 precision), unscaled in FP32 on the way out
        const float in_scale = 1.0f / P.loss_norm;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = i < 3 ? P.ws.dvc[(int64_t)i * S_cap + gs] * in_scale : 0.0f;
        uint4 lo, hi;
        lo.x = tc::pack2<BF16>(v[0], v[1]);
        lo.y = tc::pack2<BF16>(v[2], v[3]);
        lo.z = tc::pack2<BF16>(v[4], v[5]);
        lo.w = tc::pack2<BF16>(v[6], v[7]);
        hi.x = hi.y = hi.z = hi.w = 0u;
        uint8_t* go = sm + OFF_X + g * kXTile;
        *reinterpret_cast<uint4*>(go + tc::kmajor_offset(tl, 0, 16)) = lo;
        *reinterpret_cast<uint4*>(go + tc::kmajor_offset(tl, 8, 16)) = hi;
        uint8_t* gg = P.ws.def_gout + T * kGoTile;
        *reinterpret_cast<uint4*>(gg + tc::kmajor_offset(tl, 0, 16)) = lo;
        *reinterpret_cast<uint4*>(gg + tc::kmajor_offset(tl, 8, 16)) = hi;
      }
      tc::fence_smem_to_async();
      tc::fence_before_sync();
      wg_sync(bar);
      if (tl == 0) {
        tc::fence_after_sync();
        issue_adjoint<BF16>(tmem + 256 * g, sbase + OFF_X + g * kXTile, sbase + OFF_WO, 16, H);
        tc::commit_to(mbar);
      }
      pending = true;
      // stage e = 0..n-1: mask with h_{n-1-e}, store g, issue the next adjoint; stage n: dL/df
      for (int e = 0; e <= n; ++e) {
        ok = wg_and(bar, tc::mbar_wait(mbar, phase, P.wait_limit));
        if (!ok) break;
        phase ^= 1u;
        pending = false;
        tc::fence_after_sync();
        if (e < n) {
          const int li = n - 1 - e;
          uint8_t* gsm = sm + OFF_HB + g * kHTile;
          uint8_t* gg = P.ws.def_g + ((int64_t)li * tiles_cap + T) * kHTile;
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            float v[32];
            tc::tmem_ld32(row + 32 * q4, v);
#pragma unroll
            for (int c8 = 0; c8 < 4; ++c8) {
              // pack, then clear the halves whose stored activation is not positive
              const uint4 m = mrow[4 * q4 + c8];
              const float* x = v + 8 * c8;
              uint4 q;
              q.x = tc::pack2<BF16>(x[0], x[1]) & positive_halves<BF16>(m.x);
              q.y = tc::pack2<BF16>(x[2], x[3]) & positive_halves<BF16>(m.y);
              q.z = tc::pack2<BF16>(x[4], x[5]) & positive_halves<BF16>(m.z);
              q.w = tc::pack2<BF16>(x[6], x[7]) & positive_halves<BF16>(m.w);
              const int c = 32 * q4 + 8 * c8;
              *reinterpret_cast<uint4*>(gsm + tc::kmajor_offset(tl, c, H)) = q;
              *reinterpret_cast<uint4*>(gg + tc::kmajor_offset(tl, c, H)) = q;
            }
          }
          if (li > 0) {
            const uint8_t* hn = P.ws.def_h + ((int64_t)(li - 1) * tiles_cap + T) * kHTile;
#pragma unroll
            for (int c = 0; c < 16; ++c)
              mrow[c] = __ldg(reinterpret_cast<const uint4*>(hn + tc::kmajor_offset(tl, 8 * c, H)));
          }
          tc::fence_smem_to_async();
          tc::fence_before_sync();
          wg_sync(bar);
          if (tl == 0) {
            tc::fence_after_sync();
            if (li > 0)
              issue_adjoint<BF16>(tmem + 256 * g, sbase + OFF_HB + g * kHTile, sbase + OFF_WH + (li - 1) * kH * kH * 2,
                                  H, H);
            else
              issue_adjoint<BF16>(tmem + 256 * g, sbase + OFF_HB + g * kHTile, sbase + OFF_W1, H, Kf);
            tc::commit_to(mbar);
          }
          pending = true;
        } else {
          const int64_t gs = sl.s0 + tl;
          for (int c = 0; c < Kf; c += 16) {
            float v[16];
            tc::tmem_ld16(row + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c + i < D.n_feat) P.ws.dfeat_d[(int64_t)(c + i) * S_cap + gs] = v[i] * P.loss_norm;
          }
          tc::fence_before_sync();
        }
      }
    }
  }
  if (!ok) {
    if (tl == 0) atomicOr(P.status, kStatusTimeout);
    if (tl == 0 && pending && !tc::mbar_wait(mbar, phase, kDrainLimit)) atomicOr(P.status, kStatusDrainTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Weight gradients of the net, accumulated in tensor memory over every tile the CTA visits:
//   dW_l (l = 1..n-1) += g_l^T h_{l-1}    (128 x 128 each, columns 128 (l - 1))
//   dW_out^T         += h_n^T g_out      (128 x 16, columns 384)
//   dW_1f            += g_1^T x          (128 x 32, columns 400)
//   dW_1p            += g_1^T Theta      (128 x 80, columns 432; Theta = the view's pose in
//                                          every row, the pose columns of W_1)
// then written as this CTA's partial (summed over CTAs by k_deform_reduce).  The operand
// pairs of the CTA's tiles form one sequence; the stored tiles of pairs p+1 and p+2 arrive by
// bulk copies into the other two of three buffers while pair p's MMAs run (pair p+2's as soon
// as pair p-1's MMAs have released its buffer); a tile's last pair (g_1, x) also feeds dW_1p
// from the same g_1 tile, so each tile takes n + 1 pairs.  Theta is rewritten when the view
// changes, after the MMAs in flight have drained.
constexpr uint32_t C_DWO = 384, C_DW1F = 400, C_DW1P = 432;
constexpr int kDwBufs = 3;                                 // operand pair buffers
constexpr uint32_t D_BUF = 0;                              // kDwBufs x 2 x [128 x 128] operand buffers
constexpr uint32_t D_THETA = D_BUF + 2 * kDwBufs * kHTile;   // [128 x 80]
constexpr uint32_t D_MISC = D_THETA + kTM * kDeformTcMaxPose * 2;   // 2 kDwBufs mbarriers + TMEM base
constexpr uint32_t kSmemDw = D_MISC + 64 + 1024;
static_assert(16 * kDwBufs + 4 <= 64, "the mbarriers and the tensor-memory base fit the misc block");
static_assert(kSmemDw <= 227 * 1024, "the weight-gradient kernel's buffers fit one CTA");

// One operand pair of the weight-gradient sequence.
struct DwPair {
  const uint8_t* a;   // [128 samples][a_units] stored tile
  const uint8_t* b;   // [128 samples][b_units] stored tile
  int a_units, b_units;
  uint32_t dcol;      // accumulator columns
};

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) k_deform_dw_tc(const __grid_constant__ Plan P) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  const int t = threadIdx.x, warp = t >> 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + D_MISC + 16 * kDwBufs);
  const uint32_t mbar0 = tc::smem_u32(sm + D_MISC);                 // MMAs of buffer b done: mbar0 + 8 b
  const uint32_t lbar0 = tc::smem_u32(sm + D_MISC + 8 * kDwBufs);   // copies into buffer b landed: lbar0 + 8 b
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) {
    for (int b = 0; b < kDwBufs; ++b) {
      tc::mbar_init(mbar0 + 8 * b, 1);
      tc::mbar_init(lbar0 + 8 * b, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int64_t tiles_cap = S_cap / kTM;
  const int64_t n_tiles = S <= S_cap ? S / kTM : 0;
  uint32_t phase[kDwBufs] = {}, lphase[kDwBufs] = {};
  bool pending[kDwBufs] = {}, loading[kDwBufs] = {};
  bool ok = true;
  bool any = false;
  int theta_view = -1;
  const DeformDev* Dp = nullptr;
  __shared__ int s_ok, s_any;          // warp 0's outcome, for the read-out by every warp
  __shared__ const DeformDev* s_dp;

  // the sequence: tiles T = blockIdx.x, +gridDim.x, ... of views with this kind of net;
  // per tile n + 1 pairs
  auto tile_view = [&](int64_t T) -> int {
    for (; T < n_tiles; T += gridDim.x) {
      const int v = view_of_slot(P, T * kTM);
      if (P.v[v].has_deform && P.v[v].deform.tc == (BF16 ? 2 : 1)) return v;
    }
    return -1;
  };
  auto first_tile = [&](int64_t T) -> int64_t {
    for (; T < n_tiles; T += gridDim.x) {
      const int v = view_of_slot(P, T * kTM);
      if (P.v[v].has_deform && P.v[v].deform.tc == (BF16 ? 2 : 1)) return T;
    }
    return n_tiles;
  };
  auto pair_of = [&](int64_t T, int i, int n) -> DwPair {
    const uint8_t* hb = P.ws.def_h;
    const uint8_t* gb = P.ws.def_g;
    auto H_ = [&](int l) { return hb + ((int64_t)l * tiles_cap + T) * kHTile; };
    auto G_ = [&](int l) { return gb + ((int64_t)l * tiles_cap + T) * kHTile; };
    if (i == 0) return DwPair{H_(n - 1), P.ws.def_gout + T * kGoTile, kH, 16, C_DWO};
    if (i < n) return DwPair{G_(n - i), H_(n - i - 1), kH, kH, 128u * (uint32_t)(n - i - 1)};
    return DwPair{G_(0), P.ws.def_x + T * kXTile, kH, kKf, C_DW1F};
  };
  // one thread: bulk copies of a pair's stored tiles into buffer b
  auto load_pair = [&](const DwPair& q, int b) {
    if (t == 0) {
      const uint32_t abytes = (uint32_t)(kTM * q.a_units * 2), bbytes = (uint32_t)(kTM * q.b_units * 2);
      tc::mbar_expect_tx(lbar0 + 8 * b, abytes + bbytes);
      tc::bulk_g2s(sbase + D_BUF + (2 * b) * kHTile, q.a, abytes, lbar0 + 8 * b);
      tc::bulk_g2s(sbase + D_BUF + (2 * b + 1) * kHTile, q.b, bbytes, lbar0 + 8 * b);
    }
    loading[b] = true;
  };
  // warp 0: buffer b's MMAs have completed (bounded)
  auto drain = [&](int b) -> bool {
    if (!pending[b]) return true;
    const bool got = tc::mbar_wait(mbar0 + 8 * b, phase[b], P.wait_limit);
    if (!__all_sync(0xffffffffu, got)) return false;
    phase[b] ^= 1u;
    pending[b] = false;
    return true;
  };

  // the sequence runs in warp 0 alone (its waits are warp votes, not block barriers); the
  // other warps join for the partial's read-out
  if (warp == 0) {
    // a position in the sequence: tile T (view v), pair i
    struct Pos {
      int64_t T;
      int i, v;
    };
    auto advance = [&](Pos q) -> Pos {
      if (++q.i > P.v[q.v].deform.n_hidden) {
        q.T = first_tile(q.T + gridDim.x);
        q.i = 0;
        q.v = q.T < n_tiles ? tile_view(q.T) : -1;
      }
      return q;
    };
    Pos cur{first_tile(blockIdx.x), 0, -1};
    if (cur.T < n_tiles) cur.v = tile_view(cur.T);
    Pos ahead = cur;  // the next pair to load
    int p = 0, lp = 0;  // pairs issued, pairs loaded; pair p in buffer p % kDwBufs
    for (; lp < kDwBufs - 1 && ahead.T < n_tiles; ++lp) {
      load_pair(pair_of(ahead.T, ahead.i, P.v[ahead.v].deform.n_hidden), lp % kDwBufs);
      ahead = advance(ahead);
    }
    while (cur.T < n_tiles && ok) {
      const DeformDev& D = P.v[cur.v].deform;
      const int n = D.n_hidden, i = cur.i;
      const int b = p % kDwBufs;
      Dp = &D;
      if (i == 0 && cur.v != theta_view) {
        // Theta rows = this view's pose, padded to 80 columns, once the MMAs that read the
        // previous Theta have completed
        for (int q = 0; q < kDwBufs && ok; ++q) ok = drain(q);
        if (!ok) break;
        for (int k = 0; k < kDeformTcMaxPose; k += 8) {
          float x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) x[u] = k + u < D.pose_dim ? D.pose[k + u] : 0.0f;
          uint4 q;
          q.x = tc::pack2<BF16>(x[0], x[1]);
          q.y = tc::pack2<BF16>(x[2], x[3]);
          q.z = tc::pack2<BF16>(x[4], x[5]);
          q.w = tc::pack2<BF16>(x[6], x[7]);
          for (int r = t; r < kTM; r += 32)  // four rows per lane
            *reinterpret_cast<uint4*>(sm + D_THETA + tc::kmajor_offset(r, k, kDeformTcMaxPose)) = q;
        }
        tc::fence_smem_to_async();
        __syncwarp();
        theta_view = cur.v;
      }
      // keep kDwBufs - 1 pairs loading ahead (the sequence runs on into the next tiles): pair
      // lp goes into the buffer that pair lp - kDwBufs = p - 1 releases when its MMAs complete
      if (ahead.T < n_tiles) {
        const int bl = lp % kDwBufs;
        if (!(ok = drain(bl))) break;
        load_pair(pair_of(ahead.T, ahead.i, P.v[ahead.v].deform.n_hidden), bl);
        ahead = advance(ahead);
        ++lp;
      }
      // this pair's tiles have landed: issue its MMAs
      const DwPair q = pair_of(cur.T, i, n);
      ok = tc::mbar_wait(lbar0 + 8 * b, lphase[b], P.wait_limit);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      lphase[b] ^= 1u;
      loading[b] = false;
      if (t == 0) {
        tc::fence_after_sync();
        issue_dw<BF16>(tmem + q.dcol, sbase + D_BUF + (2 * b) * kHTile, q.a_units,
                       sbase + D_BUF + (2 * b + 1) * kHTile, q.b_units, any);
        if (i == n)  // the pose columns from the same g_1 tile
          issue_dw<BF16>(tmem + C_DW1P, sbase + D_BUF + (2 * b) * kHTile, kH, sbase + D_THETA, kDeformTcMaxPose,
                         any);
        tc::commit_to(mbar0 + 8 * b);
      }
      pending[b] = true;
      ++p;
      if (i == n) any = true;  // every accumulator has been written once
      cur = advance(cur);
    }
    for (int b = 0; b < kDwBufs && ok; ++b) ok = drain(b);
    if (!ok) {
      if (t == 0) atomicOr(P.status, kStatusTimeout);
      // let this CTA's MMAs and copies in flight finish (bounded) before its tensor memory and
      // shared memory are released
      for (int b = 0; b < kDwBufs; ++b) {
        if (pending[b] && !tc::mbar_wait(mbar0 + 8 * b, phase[b], kDrainLimit))
          atomicOr(P.status, kStatusDrainTimeout);
        if (loading[b] && !tc::mbar_wait(lbar0 + 8 * b, lphase[b], kDrainLimit))
          atomicOr(P.status, kStatusDrainTimeout);
      }
    }
    if (t == 0) {
      s_ok = ok;
      s_any = any;
      s_dp = Dp;
    }
  }  // warp 0
  tc::fence_before_sync();
  __syncthreads();
  ok = s_ok;
  any = s_any;
  Dp = s_dp;
  if (ok && Dp) {
    // write this CTA's partial: lane t is row t of every accumulator
    tc::fence_after_sync();
    const DeformDev& D = *Dp;
    const int n = D.n_hidden, n_in = D.n_feat + D.pose_dim;
    const float out_scale = P.loss_norm;   // the chain's deltas carry 1 / loss_norm
    float* part = D.dw_scratch + (int64_t)blockIdx.x * D.n_w;
    const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
    for (int l = 1; l < n; ++l) {
      float* dst = part + (int64_t)kH * n_in + (int64_t)(l - 1) * kH * kH + (int64_t)t * kH;
      for (int c = 0; c < kH; c += 16) {
        float v16[16];
        tc::tmem_ld16(row + 128u * (l - 1) + c, v16);
#pragma unroll
        for (int u = 0; u < 16; ++u) dst[c + u] = any ? v16[u] * out_scale : 0.0f;
      }
    }
    {
      float v16[16];
      tc::tmem_ld16(row + C_DWO, v16);
      float* dst = part + layer_offset(D, n);
      for (int c = 0; c < 3; ++c) dst[c * kH + t] = any ? v16[c] * out_scale : 0.0f;
    }
    for (int c = 0; c < kKf; c += 16) {
      float v16[16];
      tc::tmem_ld16(row + C_DW1F + c, v16);
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (c + u < D.n_feat) part[(int64_t)t * n_in + c + u] = any ? v16[u] * out_scale : 0.0f;
    }
    for (int c = 0; c < kDeformTcMaxPose; c += 16) {
      float v16[16];
      tc::tmem_ld16(row + C_DW1P + c, v16);
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (c + u < D.pose_dim) part[(int64_t)t * n_in + D.n_feat + c + u] = any ? v16[u] * out_scale : 0.0f;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

template <bool BF16>
static cudaError_t backward_tc(const Plan& P, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_deform_chain_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  k_deform_chain_tc<BF16><<<num_sms, kThreadsF, kSmem, s>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_deform_dw_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDw);
  if (e != cudaSuccess) return e;
  k_deform_dw_tc<BF16><<<num_sms, kThreads, kSmemDw, s>>>(P);
  return cudaGetLastError();
}

template <bool BF16>
static cudaError_t forward_tc(const Plan& P, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_deform_fwd_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF);
  if (e != cudaSuccess) return e;
  k_deform_fwd_tc<BF16><<<num_sms, kThreadsF, kSmemF, s>>>(P);
  return cudaGetLastError();
}

static void tc_kinds(const Plan& P, bool& f16, bool& bf16) {
  f16 = bf16 = false;
  for (int v = 0; v < P.n_views; ++v) {
    if (!P.v[v].has_deform) continue;
    if (P.v[v].deform.tc == 1) f16 = true;
    if (P.v[v].deform.tc == 2) bf16 = true;
  }
}

cudaError_t launch_deform_backward_tc(const Plan& P, int num_sms, cudaStream_t s) {
  bool f16, bf16;
  tc_kinds(P, f16, bf16);
  cudaError_t e = cudaSuccess;
  if (bf16) e = backward_tc<true>(P, num_sms, s);
  if (e == cudaSuccess && f16) e = backward_tc<false>(P, num_sms, s);
  return e;
}

cudaError_t launch_deform_forward_tc(const Plan& P, int num_sms, cudaStream_t s) {
  bool f16, bf16;
  tc_kinds(P, f16, bf16);
  cudaError_t e = cudaSuccess;
  if (bf16) e = forward_tc<true>(P, num_sms, s);
  if (e == cudaSuccess && f16) e = forward_tc<false>(P, num_sms, s);
  return e;
}

}  // namespace invr
