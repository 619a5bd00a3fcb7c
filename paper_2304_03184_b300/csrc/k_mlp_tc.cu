// Geometry + colour MLPs on the 5th-generation tensor cores (tcgen05, kind::f16): FP16 or
// BF16 operands, FP32 accumulation in tensor memory (the mixed-precision path; Sec. 4.2
// geometry MLP E_g and colour MLP E_c).
//
// One CTA = 128 threads = one warpgroup; a tile is 128 samples, thread t owns sample t,
// which is row t of every MMA (M = 128) and lane t of tensor memory.  Per tile the five
// layers run as a chain through two 16 KB operand buffers P and Q:
//   X [128 x in] (P) -> D = X W1^T (N 64)  -> ReLU -> H1 (Q)
//   H1 (Q)           -> D = H1 W2^T (N 64) -> ReLU -> H2 (P)
//   H2 (P)           -> D = H2 W3^T (N 16) -> sigma = exp(o_0); O = (0, o_1..o_15) (Q)
//   O (Q)            -> D = O W4p^T (N 64) -> ReLU -> H4 (Q, over O)
//   H4 (Q)           -> D = H4 W5p^T (N 16) -> rgb = sigmoid(z_0..z_2)
// One elected thread issues each layer's MMAs (K = 16 per instruction) into one 64-column
// accumulator and commits them to an mbarrier; all threads wait, read their row from tensor
// memory (one tcgen05.ld of 64 columns), apply the activation in FP32 and write the next
// operand row in the K-major layout.  The encoder writes the features as 16-bit operand
// tiles, so a tile's X arrives by one TMA copy (a 3-D box of its 16 row groups); the copy of
// the CTA's next tile is issued as soon as layer 3 has read P, and land while layers 4 and 5
// run.  Weights (padded: W4p gets a zero column for o_0, W5p 13 zero rows) arrive as the
// field's 16-bit weight image (written from the FP32 weights by k_prep_w16 before each
// launch) by one bulk copy per CTA and field.  50 KB of shared memory and 64
// tensor-memory columns per CTA: four CTAs per SM overlap their chains.  Every mbarrier
// wait is bounded; a timeout sets the status word, and the CTA waits (bounded) for its
// own copies and MMAs in flight, frees its tensor memory and exits.
#include <cuda.h>

#include "invr_internal.cuh"
#include "tc_ptx.cuh"

namespace invr {

namespace {

constexpr int kTM = 128;             // samples per tile = MMA M
constexpr int kThreadsTC = 128;
constexpr int kCtasPerSm = 4;
constexpr uint32_t kTmemCols = 64;   // one accumulator, reused by every layer
constexpr uint32_t kWaitLimit = 1u << 22;  // polls of try_wait (bounded: a few seconds)

// shared-memory plan (bytes)
constexpr uint32_t OFF_W1 = 0;                       // 64 x 32
constexpr uint32_t OFF_W2 = OFF_W1 + 64 * 32 * 2;    // 64 x 64
constexpr uint32_t OFF_W3 = OFF_W2 + 64 * 64 * 2;    // 16 x 64
constexpr uint32_t OFF_W4 = OFF_W3 + 16 * 64 * 2;    // 64 x 16
constexpr uint32_t OFF_W5 = OFF_W4 + 64 * 16 * 2;    // 16 x 64
constexpr uint32_t OFF_P = OFF_W5 + 16 * 64 * 2;     // 128 x 64: X, then H2
constexpr uint32_t OFF_Q = OFF_P + kTM * 64 * 2;     // 128 x 64: H1, then O, then H4
constexpr uint32_t OFF_MISC = OFF_Q + kTM * 64 * 2;  // 2 mbarriers (16 B) + TMEM base (4 B)
constexpr uint32_t kSmemTC = OFF_MISC + 64;
static_assert(kCtasPerSm * (kSmemTC + 1024) <= 228 * 1024, "four CTAs per SM");
static_assert(kCtasPerSm * kTmemCols <= 512, "tensor memory of four CTAs");

struct TcArgs {
  CUtensorMap xmap[2];      // TMA maps of the 16-bit feature tiles for in = 16, 32 (plan path)
  const void* feat;         // 16-bit operand tiles (feat16_offset), or FP32 [in][ld] (points)
  float* out;               // [4][ld]
  const int32_t* view_base; // per-view tile-aligned sample ranges (device) or null
  int64_t ld;
  int64_t n;                // samples when view_base is null
  int n_views;
  uint32_t wait_limit;      // polls per bounded wait (0: give up at once)
  unsigned* status;
  FieldDev f[kMaxViews];
};

struct WOff {
  int w1, w2, w3, w4, w5;
  __device__ explicit WOff(int in) {
    w1 = 0;
    w2 = in * kHidden;
    w3 = w2 + kHidden * kHidden;
    w4 = w3 + kGeoOut * kHidden;
    w5 = w4 + kColHidden * (kGeoOut - 1);
  }
};

// Stage one (padded) weight matrix [N][K] as a K-major 16-bit operand.
template <bool BF16, int N, int K>
__device__ __forceinline__ void stage_weight(uint8_t* dst, const float* __restrict__ W, int layer, int in,
                                             const WOff& off) {
  for (int e = threadIdx.x; e < N * K / 2; e += blockDim.x) {
    const int o = (2 * e) / K, k = (2 * e) % K;
    float a = 0.0f, b = 0.0f;
    switch (layer) {
      case 1: a = W[off.w1 + o * in + k]; b = W[off.w1 + o * in + k + 1]; break;
      case 2: a = W[off.w2 + o * kHidden + k]; b = W[off.w2 + o * kHidden + k + 1]; break;
      case 3: a = W[off.w3 + o * kHidden + k]; b = W[off.w3 + o * kHidden + k + 1]; break;
      case 4:  // column 0 of W4p is zero: o_0 does not feed the colour MLP
        a = k == 0 ? 0.0f : W[off.w4 + o * (kGeoOut - 1) + k - 1];
        b = W[off.w4 + o * (kGeoOut - 1) + k];
        break;
      default:  // rows 3..15 of W5p are zero
        a = o < 3 ? W[off.w5 + o * kColHidden + k] : 0.0f;
        b = o < 3 ? W[off.w5 + o * kColHidden + k + 1] : 0.0f;
        break;
    }
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_offset(o, k, K)) = tc::pack2<BF16>(a, b);
  }
}

// All threads of the CTA: the field's weight image (`bytes` from global `src`) into shared
// memory at `dst` by one bulk copy, its completion awaited on mbarrier `bar` (bounded);
// every MMA that read the previous weights has completed.  The barrier's phase lives in
// shared memory (`phase`, flipped by thread 0), not in a register of the tile loop.  On a
// time-out the copy is drained (bounded) before returning false, so no write of it can land
// after the CTA leaves.
__device__ __forceinline__ bool load_weights(uint32_t dst, const uint8_t* src, int bytes, uint32_t bar,
                                             uint32_t& phase, uint32_t wait_limit, unsigned* status) {
  __syncthreads();
  const uint32_t ph = phase;
  if (threadIdx.x == 0) {
    tc::mbar_expect_tx(bar, (uint32_t)bytes);
    tc::bulk_g2s(dst, src, (uint32_t)bytes, bar);
  }
  const bool got = tc::mbar_wait(bar, ph, wait_limit);
  if (!__syncthreads_and(got)) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusTimeout);
      if (!tc::mbar_wait(bar, ph, kWaitLimit)) atomicOr(status, kStatusDrainTimeout);
    }
    __syncthreads();
    return false;
  }
  if (threadIdx.x == 0) phase = ph ^ 1u;  // read by all threads at the next call, after its barrier
  return true;
}

// One thread: issue D(tmem) = A(smem, 128 x K) * B(smem, N x K)^T as K/16 MMAs.
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N,
                                            bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

// Read the 64 accumulator columns of this thread's row, apply ReLU, store as row t of a
// K = 64 16-bit operand.
template <bool BF16>
__device__ __forceinline__ void relu_row64(uint32_t taddr, uint8_t* dst, int t) {
  float v[64];
  tc::tmem_ld64(taddr, v);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 q;
    q.x = tc::pack2<BF16>(fmaxf(v[8 * c + 0], 0.f), fmaxf(v[8 * c + 1], 0.f));
    q.y = tc::pack2<BF16>(fmaxf(v[8 * c + 2], 0.f), fmaxf(v[8 * c + 3], 0.f));
    q.z = tc::pack2<BF16>(fmaxf(v[8 * c + 4], 0.f), fmaxf(v[8 * c + 5], 0.f));
    q.w = tc::pack2<BF16>(fmaxf(v[8 * c + 6], 0.f), fmaxf(v[8 * c + 7], 0.f));
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8 * c, 64)) = q;
  }
}

// Operand writes done by every thread -> visible to the tensor core; TMEM reads ordered.
__device__ __forceinline__ void operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
}

// The CTA's tiles: from `tile` on in steps of gridDim.x, the first whose view has this
// kernel's MLP kind (uniform over the CTA), or n_tiles; v follows the view (cursor).
__device__ __forceinline__ int64_t next_tile(const TcArgs& A, const int32_t* vb, int64_t tile, int64_t n_tiles,
                                             int kind, int& v) {
  for (; tile < n_tiles; tile += gridDim.x) {
    v = advance_view(vb, A.n_views, tile * kTM, v);
    if (A.f[v].mlp_kind == kind) return tile;
  }
  return n_tiles;
}

// One warp (lane 0 works): tile `tile`'s X [128 x in] as one TMA box of its 16 row groups.
__device__ __forceinline__ void load_x(const TcArgs& A, int64_t tile, int in, uint32_t dst, uint32_t bar) {
  if ((threadIdx.x & 31) == 0) {
    tc::mbar_expect_tx(bar, 16u * 16u * (uint32_t)in);
    tc::tma_load_3d(dst, &A.xmap[in == 32 ? 1 : 0], 0, (int)tile, 0, bar);
  }
  __syncwarp();
}

// TILES: the plan's 16-bit operand tiles (one TMA copy each, prefetched); else FP32 feature-major
// points converted by the threads.
template <bool BF16, bool TILES>
__global__ void __launch_bounds__(kThreadsTC, kCtasPerSm) k_mlp_fwd_tc(const __grid_constant__ TcArgs A) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ int32_t vb[kMaxViews + 1];  // view sample bases
  __shared__ uint32_t s_wphase;          // phase of the weight-image barrier
  if (A.view_base && (int64_t)A.view_base[A.n_views] > A.ld) return;  // overflow flagged by the scan
  const int t = threadIdx.x, warp = t >> 5;
  if (t <= A.n_views) vb[t] = A.view_base ? A.view_base[t] : 0;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 16);
  const uint32_t mbar = tc::smem_u32(sm + OFF_MISC);       // MMA completion
  const uint32_t xbar = tc::smem_u32(sm + OFF_MISC + 8);   // X copies landed
  const uint32_t wbar = tc::smem_u32(sm + OFF_MISC + 24);  // weight image landed
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(xbar, 1);
    tc::mbar_init(wbar, 1);
    s_wphase = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row_taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const int kind = BF16 ? kMlpBF16 : kMlpF16;

  const int64_t S = A.view_base ? (int64_t)A.view_base[A.n_views] : A.n;
  const int64_t n_tiles = (S + kTM - 1) / kTM;
  const float* loaded = nullptr;
  uint32_t phase = 0, xphase = 0;
  bool ok = true;
  bool mma_pending = false, x_pending = false;

  int vn = 0;  // view of the next tile to process
  int64_t tile = next_tile(A, vb, blockIdx.x, n_tiles, kind, vn);
  if (TILES && warp == 0 && tile < n_tiles) load_x(A, tile, A.f[vn].mlp_in, sbase + OFF_P, xbar);
  x_pending = TILES && tile < n_tiles;

  while (tile < n_tiles) {
    const int64_t s0 = tile * kTM;
    const FieldDev& F = A.f[vn];
    const int64_t nxt = next_tile(A, vb, tile + gridDim.x, n_tiles, kind, vn);
    if (F.weights != loaded) {
      // the field's weight image by one bulk copy (every MMA that read the previous field's
      // weights has completed: the last tile waited for them)
      if (!load_weights(sbase + OFF_W1, F.w16, kW16Bytes, wbar, s_wphase, A.wait_limit, A.status)) {
        ok = false;
        break;
      }
      loaded = F.weights;
    }
    const int in = F.mlp_in;
    const int valid = (int)(S - s0 < kTM ? S - s0 : kTM);
    if constexpr (!TILES) {
      // ---- X: this thread's FP32 features (feature-major in global) -> row t
      const float* feat = static_cast<const float*>(A.feat);
      for (int j = 0; j < in / 8; ++j) {
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = t < valid ? feat[(int64_t)(8 * j + i) * A.ld + s0 + t] : 0.0f;
        uint4 q;
        q.x = tc::pack2<BF16>(x[0], x[1]);
        q.y = tc::pack2<BF16>(x[2], x[3]);
        q.z = tc::pack2<BF16>(x[4], x[5]);
        q.w = tc::pack2<BF16>(x[6], x[7]);
        *reinterpret_cast<uint4*>(sm + OFF_P + tc::kmajor_offset(t, 8 * j, in)) = q;
      }
    }
    operands_ready();  // converted X (points path) visible to the tensor core
    if constexpr (TILES) {
      ok = tc::mbar_wait(xbar, xphase, A.wait_limit);
      if (!__syncthreads_and(ok)) { ok = false; break; }
      xphase ^= 1u;
      x_pending = false;
    }
    // ---- layer 1
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem, sbase + OFF_P, sbase + OFF_W1, in, 64, BF16);
      tc::commit_to(mbar);
    }
    mma_pending = true;
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    phase ^= 1u;
    mma_pending = false;
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr, sm + OFF_Q, t);
    operands_ready();
    // ---- layer 2
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem, sbase + OFF_Q, sbase + OFF_W2, 64, 64, BF16);
      tc::commit_to(mbar);
    }
    mma_pending = true;
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    phase ^= 1u;
    mma_pending = false;
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr, sm + OFF_P, t);
    operands_ready();
    // ---- layer 3: geometry output o (16)
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem, sbase + OFF_P, sbase + OFF_W3, 64, 16, BF16);
      tc::commit_to(mbar);
    }
    mma_pending = true;
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    phase ^= 1u;
    mma_pending = false;
    tc::fence_after_sync();
    // P (H2) has been read: the next tile's X may land there now
    if (TILES && nxt < n_tiles) {
      if (warp == 0) load_x(A, nxt, A.f[vn].mlp_in, sbase + OFF_P, xbar);
      x_pending = true;
    }
    float o[16];
    tc::tmem_ld16(row_taddr, o);
    const float sigma = expf(o[0]);
    {
      uint4 lo, hi;
      lo.x = tc::pack2<BF16>(0.0f, o[1]);
      lo.y = tc::pack2<BF16>(o[2], o[3]);
      lo.z = tc::pack2<BF16>(o[4], o[5]);
      lo.w = tc::pack2<BF16>(o[6], o[7]);
      hi.x = tc::pack2<BF16>(o[8], o[9]);
      hi.y = tc::pack2<BF16>(o[10], o[11]);
      hi.z = tc::pack2<BF16>(o[12], o[13]);
      hi.w = tc::pack2<BF16>(o[14], o[15]);
      *reinterpret_cast<uint4*>(sm + OFF_Q + tc::kmajor_offset(t, 0, 16)) = lo;
      *reinterpret_cast<uint4*>(sm + OFF_Q + tc::kmajor_offset(t, 8, 16)) = hi;
    }
    operands_ready();
    // ---- layer 4: colour hidden
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem, sbase + OFF_Q, sbase + OFF_W4, 16, 64, BF16);
      tc::commit_to(mbar);
    }
    mma_pending = true;
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    phase ^= 1u;
    mma_pending = false;
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr, sm + OFF_Q, t);  // H4 over O (read by the completed layer 4)
    operands_ready();
    // ---- layer 5: colour output
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem, sbase + OFF_Q, sbase + OFF_W5, 64, 16, BF16);
      tc::commit_to(mbar);
    }
    mma_pending = true;
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    phase ^= 1u;
    mma_pending = false;
    tc::fence_after_sync();
    float z[16];
    tc::tmem_ld16(row_taddr, z);
    if (t < valid) {
      const int64_t gs = s0 + t;
      A.out[gs] = sigma;
      A.out[A.ld + gs] = 1.0f / (1.0f + expf(-z[0]));
      A.out[2 * A.ld + gs] = 1.0f / (1.0f + expf(-z[1]));
      A.out[3 * A.ld + gs] = 1.0f / (1.0f + expf(-z[2]));
    }
    tc::fence_before_sync();
    __syncthreads();  // every thread is done with this tile's TMEM and operands
    tile = nxt;
  }
  if (!ok) {
    // a wait gave up: record it, then let this CTA's MMAs and copies in flight finish
    // (bounded) before the tensor memory and shared memory they write are released
    if (t == 0) atomicOr(A.status, kStatusTimeout);
    if (mma_pending && !tc::mbar_wait(mbar, phase, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
    if (x_pending && !tc::mbar_wait(xbar, xphase, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool BF16, bool TILES>
cudaError_t launch_tc(const TcArgs& A, int num_sms, cudaStream_t s) {
  cudaFuncSetAttribute(k_mlp_fwd_tc<BF16, TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC);
  k_mlp_fwd_tc<BF16, TILES><<<num_sms * kCtasPerSm, kThreadsTC, kSmemTC, s>>>(A);
  return cudaGetLastError();
}


// ====================================================================== training forward
// The training forward of a 16-bit field with split operands: every tensor-core product is
// formed as hi*hi + lo*hi + hi*lo of a 16-bit value and the 16-bit remainder of its rounding
// (tc::split2), three MMAs into one FP32 accumulator.  The ReLU decisions of the network are
// then taken at about twice the 16-bit precision: a pre-activation that rounds across zero in
// plain 16-bit arithmetic flips its unit's gradient path in the backward, and these flips,
// not the 16-bit rounding of values, are what carries the gradient error of the plain 16-bit
// chain.  The kernel writes sigma, rgb and the ReLU decisions (one bit per hidden unit of H1,
// H2, H4; [6][ld] words) that the backward applies.
//
// Layers 1 (X -> H1), 2 (H1 -> H2), 3 (H2 -> o) and 4 (O -> H4) run on the tensor cores; the
// colour output z = W5 H4 (3 x 64) is formed by each thread in FP32 from its FP32 ReLU values
// (192 FMAs per sample instead of a fifth MMA stage).  Hidden activations never touch shared
// memory: each epilogue writes its row's hi and lo halves into tensor memory, from which the
// next layer's MMAs read their A operand.  Per CTA 128 tensor-memory columns (accumulator
// [0,64), activations hi [64,96), lo [96,128)) and 49 KB of shared memory (W1..W4 hi and lo,
// W5 in FP32, one tile of X hi and lo): four CTAs per SM.  The CTA converts the weights itself
// (a bulk copy of a prepared split image measured 5.6% slower).  X hi/lo arrive by two TMA boxes;
// the next tile's are issued once layer 1 has read this tile's.
constexpr int kCtasSplit = 4;
constexpr uint32_t kTmemSplit = 128;
constexpr uint32_t T_ACC = 0, T_HI = 64, T_LO = 96;
constexpr uint32_t S_WHI = 0;                    // W1..W4 at the OFF_W* offsets
constexpr uint32_t S_WLO = OFF_W5;               // 16,384: the same layout, remainders
constexpr uint32_t S_W5 = 2 * OFF_W5;            // W5 FP32 [3][64]
constexpr uint32_t S_XHI = S_W5 + 1024;          // [128 x in]
constexpr uint32_t S_XLO = S_XHI + kTM * 32 * 2;
constexpr uint32_t S_MISC = S_XLO + kTM * 32 * 2;
constexpr uint32_t kSmemSplit = S_MISC + 64;
static_assert(kCtasSplit * (kSmemSplit + 1024) <= 228 * 1024, "four CTAs per SM");
static_assert(kCtasSplit * kTmemSplit <= 512, "tensor memory of four CTAs");

struct SplitArgs {
  CUtensorMap xmap[2][2];   // [in == 32][hi, lo]: TMA maps of the feature tiles and their remainders
  float* out;               // [4][ld]
  uint32_t* mask;           // [6][ld]: ReLU decisions of H1 (words 0, 1), H2 (2, 3), H4 (4, 5)
  uint32_t* ticket;         // work counter of this launch (zero at launch)
  const int32_t* view_base;
  int64_t ld;
  int n_views;
  uint32_t wait_limit;
  unsigned* status;
  FieldDev f[kMaxViews];
};

// Stage one (padded) weight matrix [N][K] as K-major 16-bit values and remainders.
template <bool BF16, int N, int K>
__device__ __forceinline__ void stage_weight_split(uint8_t* hi, uint8_t* lo, const float* __restrict__ W,
                                                   int layer, int in, const WOff& off) {
  for (int e = threadIdx.x; e < N * K / 2; e += blockDim.x) {
    const int o = (2 * e) / K, k = (2 * e) % K;
    float a = 0.0f, b = 0.0f;
    switch (layer) {
      case 1: a = W[off.w1 + o * in + k]; b = W[off.w1 + o * in + k + 1]; break;
      case 2: a = W[off.w2 + o * kHidden + k]; b = W[off.w2 + o * kHidden + k + 1]; break;
      case 3: a = W[off.w3 + o * kHidden + k]; b = W[off.w3 + o * kHidden + k + 1]; break;
      default:  // column 0 of W4p is zero: o_0 does not feed the colour MLP
        a = k == 0 ? 0.0f : W[off.w4 + o * (kGeoOut - 1) + k - 1];
        b = W[off.w4 + o * (kGeoOut - 1) + k];
        break;
    }
    uint32_t h, l;
    tc::split2<BF16>(a, b, h, l);
    *reinterpret_cast<uint32_t*>(hi + tc::kmajor_offset(o, k, K)) = h;
    *reinterpret_cast<uint32_t*>(lo + tc::kmajor_offset(o, k, K)) = l;
  }
}

template <bool BF16>
__device__ void stage_weights_split(uint8_t* sm, const FieldDev& F) {
  const WOff off(F.mlp_in);
  uint8_t* hi = sm + S_WHI;
  uint8_t* lo = sm + S_WLO;
  if (F.mlp_in == 16)
    stage_weight_split<BF16, 64, 16>(hi + OFF_W1, lo + OFF_W1, F.weights, 1, 16, off);
  else
    stage_weight_split<BF16, 64, 32>(hi + OFF_W1, lo + OFF_W1, F.weights, 1, 32, off);
  stage_weight_split<BF16, 64, 64>(hi + OFF_W2, lo + OFF_W2, F.weights, 2, F.mlp_in, off);
  stage_weight_split<BF16, 16, 64>(hi + OFF_W3, lo + OFF_W3, F.weights, 3, F.mlp_in, off);
  stage_weight_split<BF16, 64, 16>(hi + OFF_W4, lo + OFF_W4, F.weights, 4, F.mlp_in, off);
  float* w5 = reinterpret_cast<float*>(sm + S_W5);
  for (int e = threadIdx.x; e < 3 * kColHidden; e += blockDim.x) w5[e] = F.weights[off.w5 + e];
}

// One thread: D = A B^T over K as split products, A in shared memory (the X tile).
__device__ __forceinline__ void issue_split_ss(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                               uint32_t b_lo, int K, int N, bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ah = tc::smem_desc(a_hi + kk * 256, 128, K * 16);
    const uint64_t al = tc::smem_desc(a_lo + kk * 256, 128, K * 16);
    const uint64_t bh = tc::smem_desc(b_hi + kk * 256, 128, K * 16);
    const uint64_t bl = tc::smem_desc(b_lo + kk * 256, 128, K * 16);
    tc::mma_f16(d, ah, bh, idesc, kk > 0 ? 1u : 0u);
    tc::mma_f16(d, al, bh, idesc, 1u);
    tc::mma_f16(d, ah, bl, idesc, 1u);
  }
}

// One thread: the same with A in tensor memory (8 columns per K step of 16).
__device__ __forceinline__ void issue_split_ts(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                               uint32_t b_lo, int K, int N, bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t bh = tc::smem_desc(b_hi + kk * 256, 128, K * 16);
    const uint64_t bl = tc::smem_desc(b_lo + kk * 256, 128, K * 16);
    tc::mma_f16_ts(d, a_hi + kk * 8, bh, idesc, kk > 0 ? 1u : 0u);
    tc::mma_f16_ts(d, a_lo + kk * 8, bh, idesc, 1u);
    tc::mma_f16_ts(d, a_hi + kk * 8, bl, idesc, 1u);
  }
}

// This thread's 64 accumulator columns (two loads, one wait).
__device__ __forceinline__ void tmem_ld64_pair(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]),
        "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]),
        "=r"(r[62]), "=r"(r[63])
      : "r"(taddr + 32)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of a 64-unit ReLU layer: ReLU of this thread's 64 accumulator columns into `h`
// (FP32), written as hi and lo halves into its tensor-memory lane (32 columns each, waited
// for once), and the decisions z > 0 as two 32-bit masks (bit j of m[w] = unit 32 w + j).
template <bool BF16, bool STORE>
__device__ __forceinline__ void relu_split64(uint32_t row, float (&h)[64], uint32_t (&m)[2]) {
  tmem_ld64_pair(row + T_ACC, h);
  // one compare per unit gives an all-ones / all-zeros word: it sets the unit's mask bit and
  // zeroes the value where z <= 0 (two logic operations, no selects or shifts)
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (h[32 * w + j] > 0.0f) bits |= 1u << j;
      else h[32 * w + j] = 0.0f;
    }
    m[w] = bits;
  }
  if constexpr (STORE) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) tc::split2<BF16>(h[32 * q + 2 * c], h[32 * q + 2 * c + 1], hi[c], lo[c]);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
              row + T_HI + 16 * q),
          "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]), "r"(hi[7]), "r"(hi[8]),
          "r"(hi[9]), "r"(hi[10]), "r"(hi[11]), "r"(hi[12]), "r"(hi[13]), "r"(hi[14]), "r"(hi[15])
          : "memory");
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
              row + T_LO + 16 * q),
          "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]), "r"(lo[8]),
          "r"(lo[9]), "r"(lo[10]), "r"(lo[11]), "r"(lo[12]), "r"(lo[13]), "r"(lo[14]), "r"(lo[15])
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
}

// Tensor-memory writes and reads of every thread done -> the tensor core may go on.
__device__ __forceinline__ void tmem_ready() {
  tc::fence_before_sync();
  __syncthreads();
}

// One thread: the next tile of this kernel's MLP kind by the launch's work counter (tiles are
// handed out in increasing order, so a CTA's tiles increase too), or n_tiles.  Dynamic: CTAs
// that run faster take more tiles (with a fixed stride, CTAs with equal tile counts finished
// up to 50% apart).
__device__ __forceinline__ int64_t grab_tile(const SplitArgs& A, const int32_t* vb, int64_t n_tiles, int kind) {
  for (;;) {
    const int64_t tile = (int64_t)atomicAdd(A.ticket, 1u);
    if (tile >= n_tiles) return n_tiles;
    if (A.f[view_of_slot(vb, A.n_views, tile * kTM)].mlp_kind == kind) return tile;
  }
}

// One thread: X hi and lo of tile `tile` as two TMA boxes.
__device__ __forceinline__ void load_x_split(const SplitArgs& A, int64_t tile, int in, uint32_t sbase, uint32_t bar) {
  const int w = in == 32 ? 1 : 0;
  tc::mbar_expect_tx(bar, 2u * 16u * 16u * (uint32_t)in);
  tc::tma_load_3d(sbase + S_XHI, &A.xmap[w][0], 0, (int)tile, 0, bar);
  tc::tma_load_3d(sbase + S_XLO, &A.xmap[w][1], 0, (int)tile, 0, bar);
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsTC, kCtasSplit) k_mlp_fwd_split_tc(const __grid_constant__ SplitArgs A) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ int32_t vb[kMaxViews + 1];
  __shared__ int64_t s_next;  // thread 0's next tile, read by all after the next barrier
  if ((int64_t)A.view_base[A.n_views] > A.ld) return;  // overflow flagged by the scan
  const int t = threadIdx.x, warp = t >> 5;
  if (t <= A.n_views) vb[t] = A.view_base[t];
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S_MISC + 16);
  const uint32_t mbar = tc::smem_u32(sm + S_MISC);
  const uint32_t xbar = tc::smem_u32(sm + S_MISC + 8);
  const uint32_t sbase = tc::smem_u32(sm);
  const float* w5 = reinterpret_cast<const float*>(sm + S_W5);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemSplit);
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(xbar, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
  const int kind = BF16 ? kMlpBF16 : kMlpF16;
  const int64_t S = (int64_t)A.view_base[A.n_views];
  const int64_t n_tiles = (S + kTM - 1) / kTM;
  const float* loaded = nullptr;
  uint32_t phase = 0, xphase = 0;
  bool ok = true, mma_pending = false, x_pending = false;

  __syncthreads();  // vb
  if (t == 0) {
    const int64_t first = grab_tile(A, vb, n_tiles, kind);
    if (first < n_tiles) {
      load_x_split(A, first, A.f[view_of_slot(vb, A.n_views, first * kTM)].mlp_in, sbase, xbar);
      x_pending = true;
    }
    s_next = first;
  }
  __syncthreads();
  int64_t tile = s_next;
  int vn = tile < n_tiles ? view_of_slot(vb, A.n_views, tile * kTM) : 0;

#define INVR_SPLIT_WAIT()                                     \
  mma_pending = true;                                         \
  ok = tc::mbar_wait(mbar, phase, A.wait_limit);              \
  if (!__syncthreads_and(ok)) { ok = false; break; }          \
  phase ^= 1u;                                                \
  mma_pending = false;                                        \
  tc::fence_after_sync();

  while (tile < n_tiles) {
    const int64_t s0 = tile * kTM;
    const FieldDev& F = A.f[vn];
    if (F.weights != loaded) {
      __syncthreads();
      stage_weights_split<BF16>(sm, F);
      loaded = F.weights;
      tc::fence_smem_to_async();
    }
    const int in = F.mlp_in;
    const int valid = (int)(S - s0 < kTM ? S - s0 : kTM);
    tmem_ready();
    ok = tc::mbar_wait(xbar, xphase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    xphase ^= 1u;
    x_pending = false;
    uint32_t m1[2], m2[2], m4[2];
    float h[64];
    // ---- layer 1: X (shared memory) -> H1
    if (t == 0) {
      tc::fence_after_sync();
      issue_split_ss(tmem + T_ACC, sbase + S_XHI, sbase + S_XLO, sbase + S_WHI + OFF_W1, sbase + S_WLO + OFF_W1,
                     in, 64, BF16);
      tc::commit_to(mbar);
    }
    INVR_SPLIT_WAIT();
    // X has been read: thread 0 takes the CTA's next tile, whose X lands while layers 2..4 run
    if (t == 0) {
      const int64_t nt = grab_tile(A, vb, n_tiles, kind);
      if (nt < n_tiles) {
        load_x_split(A, nt, A.f[view_of_slot(vb, A.n_views, nt * kTM)].mlp_in, sbase, xbar);
        x_pending = true;
      }
      s_next = nt;
    }
    relu_split64<BF16, true>(row, h, m1);
    tmem_ready();
    // ---- layer 2: H1 (tensor memory) -> H2
    if (t == 0) {
      tc::fence_after_sync();
      issue_split_ts(tmem + T_ACC, tmem + T_HI, tmem + T_LO, sbase + S_WHI + OFF_W2, sbase + S_WLO + OFF_W2, 64,
                     64, BF16);
      tc::commit_to(mbar);
    }
    INVR_SPLIT_WAIT();
    relu_split64<BF16, true>(row, h, m2);
    tmem_ready();
    // ---- layer 3: H2 -> o (16)
    if (t == 0) {
      tc::fence_after_sync();
      issue_split_ts(tmem + T_ACC, tmem + T_HI, tmem + T_LO, sbase + S_WHI + OFF_W3, sbase + S_WLO + OFF_W3, 64,
                     16, BF16);
      tc::commit_to(mbar);
    }
    INVR_SPLIT_WAIT();
    float sigma;
    {
      float o[16];
      tc::tmem_ld16(row + T_ACC, o);
      sigma = expf(o[0]);
      o[0] = 0.0f;  // o_0 does not feed the colour MLP (W4p has a zero column for it)
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) tc::split2<BF16>(o[2 * c], o[2 * c + 1], hi[c], lo[c]);
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(row + T_HI),
                   "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]), "r"(hi[7])
                   : "memory");
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(row + T_LO),
                   "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7])
                   : "memory");
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tmem_ready();
    // ---- layer 4: O -> H4; colour z = W5 H4 in FP32 by each thread
    if (t == 0) {
      tc::fence_after_sync();
      issue_split_ts(tmem + T_ACC, tmem + T_HI, tmem + T_LO, sbase + S_WHI + OFF_W4, sbase + S_WLO + OFF_W4, 16,
                     64, BF16);
      tc::commit_to(mbar);
    }
    INVR_SPLIT_WAIT();
    relu_split64<BF16, false>(row, h, m4);
    float z[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < kColHidden; j += 4) {
        const float4 w = *reinterpret_cast<const float4*>(w5 + c * kColHidden + j);  // one 16-byte broadcast load
        z[c] = fmaf(w.x, h[j], z[c]);
        z[c] = fmaf(w.y, h[j + 1], z[c]);
        z[c] = fmaf(w.z, h[j + 2], z[c]);
        z[c] = fmaf(w.w, h[j + 3], z[c]);
      }
    if (t < valid) {
      const int64_t gs = s0 + t;
      A.out[gs] = sigma;
      A.out[A.ld + gs] = 1.0f / (1.0f + expf(-z[0]));
      A.out[2 * A.ld + gs] = 1.0f / (1.0f + expf(-z[1]));
      A.out[3 * A.ld + gs] = 1.0f / (1.0f + expf(-z[2]));
      A.mask[gs] = m1[0];
      A.mask[A.ld + gs] = m1[1];
      A.mask[2 * A.ld + gs] = m2[0];
      A.mask[3 * A.ld + gs] = m2[1];
      A.mask[4 * A.ld + gs] = m4[0];
      A.mask[5 * A.ld + gs] = m4[1];
    }
    tile = s_next;  // written by thread 0 before this tile's layer-2 barrier
    if (tile < n_tiles) vn = advance_view(vb, A.n_views, tile * kTM, vn);
  }
#undef INVR_SPLIT_WAIT
  if (!ok) {
    if (t == 0) atomicOr(A.status, kStatusTimeout);
    if (mma_pending && !tc::mbar_wait(mbar, phase, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
    if (x_pending && !tc::mbar_wait(xbar, xphase, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemSplit);
  }
}

// ====================================================================== weight images
// A 16-bit field's MLP weights as the shared-memory image the render forward above and the
// backward copy in with one bulk copy per CTA: the padded W1..W5 as 16-bit K-major operands
// (the layout of OFF_W1..OFF_W5 here and of the backward's weights).  Rewritten from the FP32
// weights before each forward (the optimiser changes them every step; the backward reads the
// image its training forward wrote, with the same weights): one launch for every 16-bit field
// of the call, one block per matrix and field.
static_assert(OFF_P == (uint32_t)kW16Bytes, "weight image = OFF_W1..OFF_W5");

struct PrepArgs {
  int n;
  FieldDev f[kMaxViews];
};

template <bool BF16>
__device__ __forceinline__ void prep_w16(const FieldDev& F) {
  const WOff off(F.mlp_in);
  uint8_t* plain = F.w16;
  switch (blockIdx.x) {
    case 0:
      if (F.mlp_in == 16) stage_weight<BF16, 64, 16>(plain + OFF_W1, F.weights, 1, 16, off);
      else stage_weight<BF16, 64, 32>(plain + OFF_W1, F.weights, 1, 32, off);
      break;
    case 1: stage_weight<BF16, 64, 64>(plain + OFF_W2, F.weights, 2, F.mlp_in, off); break;
    case 2: stage_weight<BF16, 16, 64>(plain + OFF_W3, F.weights, 3, F.mlp_in, off); break;
    case 3: stage_weight<BF16, 64, 16>(plain + OFF_W4, F.weights, 4, F.mlp_in, off); break;
    default: stage_weight<BF16, 16, 64>(plain + OFF_W5, F.weights, 5, F.mlp_in, off); break;
  }
}

constexpr int kPrepBlocks = 5;

// blockIdx.x: the matrix, blockIdx.y: the field.
__global__ void __launch_bounds__(256) k_prep_w16(const __grid_constant__ PrepArgs A) {
  const FieldDev& F = A.f[blockIdx.y];
  if (F.mlp_kind == kMlpBF16) prep_w16<true>(F);
  else prep_w16<false>(F);
}

cudaError_t launch_prep_w16(const PrepArgs& A, cudaStream_t s) {
  if (A.n > 0) k_prep_w16<<<dim3(kPrepBlocks, A.n), 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_prep_w16(const FieldDev& f, cudaStream_t s) {
  PrepArgs A{};
  A.n = f.mlp_kind == kMlpF32 ? 0 : 1;
  A.f[0] = f;
  return launch_prep_w16(A, s);
}

}  // namespace

// Every 16-bit field of the plan (once each), in one launch.
cudaError_t launch_prep_w16_plan(const Plan& P, cudaStream_t s) {
  PrepArgs A{};
  for (int v = 0; v < P.n_views; ++v) {
    const FieldDev& F = P.v[v].field;
    bool seen = false;
    for (int u = 0; u < v; ++u) seen = seen || P.v[u].field.weights == F.weights;
    if (!seen && F.mlp_kind != kMlpF32) A.f[A.n++] = F;
  }
  return launch_prep_w16(A, s);
}

bool encode_feat16_map(void* map, const void* feat, int64_t S_cap, int in) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<Encode>(fn);
  }
  if (S_cap % kTile != 0 || (in != 16 && in != 32)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)in * 8, (cuuint64_t)(S_cap / kTile), 16};
  const cuuint64_t strides[2] = {512, (cuuint64_t)S_cap * 4};
  const cuuint32_t box[3] = {(cuuint32_t)in * 8, 1, 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(feat), dims,
                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool plan_has_kind(const Plan& P, int kind) {
  for (int v = 0; v < P.n_views; ++v)
    if (P.v[v].field.mlp_kind == kind) return true;
  return false;
}

cudaError_t launch_mlp_fwd_tc(const Plan& P, int num_sms, cudaStream_t s) {
  TcArgs A{};
  A.feat = P.ws.feat;
  A.out = P.ws.out;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n_views = P.n_views;
  A.wait_limit = P.wait_limit;
  A.status = P.status;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  if (!encode_feat16_map(&A.xmap[0], P.ws.feat, P.ws.S_cap, 16) ||
      !encode_feat16_map(&A.xmap[1], P.ws.feat, P.ws.S_cap, 32))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;  // the weight images: launch_prep_w16_plan, before this launch
  if (plan_has_kind(P, kMlpBF16)) e = launch_tc<true, true>(A, num_sms, s);
  if (e == cudaSuccess && plan_has_kind(P, kMlpF16)) e = launch_tc<false, true>(A, num_sms, s);
  return e;
}

cudaError_t preload_mlp_points_tc() {
  cudaError_t e =
      cudaFuncSetAttribute(k_mlp_fwd_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_fwd_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC);
  cudaFuncAttributes a;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_prep_w16);
  return e;
}

cudaError_t launch_mlp_fwd_split_tc(const Plan& P, int num_sms, cudaStream_t s) {
  SplitArgs A{};
  A.out = P.ws.out;
  A.mask = P.ws.mlp_mask;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n_views = P.n_views;
  A.wait_limit = P.wait_limit;
  A.status = P.status;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  uint8_t* feat = static_cast<uint8_t*>(P.ws.feat);
  for (int w = 0; w < 2; ++w)
    for (int h = 0; h < 2; ++h)
      if (!encode_feat16_map(&A.xmap[w][h], feat + (h ? feat16_lo_offset(P.ws.S_cap) : 0), P.ws.S_cap,
                             w ? 32 : 16))
        return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;  // the weight images: launch_prep_w16_plan, before this launch
  if (plan_has_kind(P, kMlpBF16)) {
    A.ticket = P.ws.tickets + kTicketSplitFwd;
    e = cudaMemsetAsync(A.ticket, 0, sizeof(uint32_t), s);
    cudaFuncSetAttribute(k_mlp_fwd_split_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSplit);
    if (e == cudaSuccess) k_mlp_fwd_split_tc<true><<<num_sms * kCtasSplit, kThreadsTC, kSmemSplit, s>>>(A);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && plan_has_kind(P, kMlpF16)) {
    A.ticket = P.ws.tickets + kTicketSplitFwd + 1;
    e = cudaMemsetAsync(A.ticket, 0, sizeof(uint32_t), s);
    cudaFuncSetAttribute(k_mlp_fwd_split_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSplit);
    if (e == cudaSuccess) k_mlp_fwd_split_tc<false><<<num_sms * kCtasSplit, kThreadsTC, kSmemSplit, s>>>(A);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_mlp_points_tc(const FieldDev& f, int64_t n, const float* feat, float* out, unsigned* status,
                                 uint32_t wait_limit, int num_sms, cudaStream_t s) {
  TcArgs A{};
  A.wait_limit = wait_limit;
  A.feat = feat;
  A.out = out;
  A.ld = n;
  A.n = n;
  A.n_views = 1;
  A.status = status;
  A.f[0] = f;
  if (n <= 0) return cudaSuccess;
  const cudaError_t e = launch_prep_w16(f, s);
  if (e != cudaSuccess) return e;
  return f.mlp_kind == kMlpBF16 ? launch_tc<true, false>(A, num_sms, s) : launch_tc<false, false>(A, num_sms, s);
}

}  // namespace invr
