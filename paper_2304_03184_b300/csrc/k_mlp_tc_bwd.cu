// Backward of the geometry + colour MLPs on the tcgen05 tensor cores, 16-bit operands (the
// field's FP16 or BF16) with FP32 accumulation (mixed-precision fields).  The incoming
// dL/d(outputs) are multiplied by in_scale (the inverse of the loss's mean normalisation,
// so per-sample gradients are O(1) and do not underflow FP16) and the FP32 results (dX,
// dW) by out_scale on the way out.
//
// One CTA = one warpgroup of 128 threads; per 128-sample tile (thread t = sample t):
//   recompute  X -> H1 -> H2 -> O -> H4          (4 chained MMAs, M = 128, ReLU epilogues)
//   adjoint    dZ -> dH4 -> dO -> dH2 -> dH1 -> dX (5 chained MMAs; each reads the forward
//              weight as an MN-major operand; ReLU masks read back from the stored activations)
//   weights    dW5^T += H4^T dZ, dW4 += dH4^T O, dW3^T += H2^T dO, dW2 += dH2^T H1,
//              dW1 += dH1^T X: M = 64 MMAs with K = the 128 samples, issued next to the
//              chain and accumulated in tensor memory over every tile the CTA visits.
// The weight-gradient MMAs read the [sample][unit] activation buffers as MN-major operands
// (each 8 x 16-byte core matrix holds 8 units of 8 samples), so no transposed copies exist.
// Each masked delta is written over the activation that masks it (dH4 over H4, dH2 over H2,
// dH1 over H1), and dO over dZ, once the MMAs that read them have completed.  X arrives as
// the encoder's 16-bit operand tile by bulk copies into one of two buffers: the next tile's
// copies are issued when this tile's have landed and run under its whole chain; the next
// tile's dL/d(outputs) are loaded into registers at the same point.  90 KB of shared memory:
// two CTAs per SM.
// The accumulated dW are read out once per field (M = 64 accumulator: row r in TMEM lane
// 32 (r / 16) + r % 16) and added to the gradient buffer with one atomic per weight per CTA.
// dL/dX (the encoding features' gradient) is written FP32 feature-major for the hash
// scatter.  All waits are bounded; a timeout sets the status word, and the CTA waits
// (bounded) for its copies and MMAs in flight, frees its tensor memory and returns.
#include "mlp_tc_common.cuh"

namespace invr {

namespace {

using namespace mlp_tc;

constexpr int kThreadsB = 128;
constexpr uint32_t kTmemColsB = 256;
// tensor-memory columns
constexpr uint32_t C_CHAIN = 0;     // 64: the chain's current layer
constexpr uint32_t C_DW2 = 64;      // 64
constexpr uint32_t C_DW1 = 128;     // 32
constexpr uint32_t C_DW4 = 160;     // 16
constexpr uint32_t C_DW3T = 176;    // 16
constexpr uint32_t C_DW5T = 192;    // 16

// shared-memory plan (bytes); [n][k] = K-major operand with n rows and k columns.  The
// transposed products of the adjoint chain read the forward weights as MN-major operands.
constexpr uint32_t B_W1 = 0;                   // [64][32] forward weights (W4p, W5p padded)
constexpr uint32_t B_W2 = B_W1 + 64 * 32 * 2;  // [64][64]
constexpr uint32_t B_W3 = B_W2 + 64 * 64 * 2;  // [16][64]
constexpr uint32_t B_W4 = B_W3 + 16 * 64 * 2;  // [64][16]
constexpr uint32_t B_W5 = B_W4 + 16 * 64 * 2;  // [16][64]
constexpr uint32_t B_X = B_W5 + 16 * 64 * 2;   // 2 x [128][32]: this tile's X and the next
constexpr uint32_t B_H1 = B_X + 2 * kTM * 32 * 2;  // [128][64], later dH1
constexpr uint32_t B_H2 = B_H1 + kTM * 64 * 2;     // [128][64], later dH2
constexpr uint32_t B_O = B_H2 + kTM * 64 * 2;      // [128][16]
constexpr uint32_t B_H4 = B_O + kTM * 16 * 2;      // [128][64], later dH4
constexpr uint32_t B_DZ = B_H4 + kTM * 64 * 2;     // [128][16], later dO
constexpr uint32_t B_MISC = B_DZ + kTM * 16 * 2;   // 2 mbarriers + TMEM base
constexpr uint32_t B_DH4 = B_H4;
constexpr uint32_t B_DH2 = B_H2;
constexpr uint32_t B_DH1 = B_H1;
constexpr uint32_t B_DO = B_DZ;
constexpr uint32_t kSmemB = B_MISC + 64;         // 90 KB: two CTAs per SM
static_assert(2 * (kSmemB + 1024) <= 228 * 1024, "two CTAs per SM");

struct TcBwdArgs {
  const void* feat;         // 16-bit operand tiles of the encoding features (feat16_offset)
  const float* dout;        // [4][ld]: dL/do_0, dL/dz_rgb
  float* dfeat;             // [in][ld]
  const int32_t* s_ray;     // padding marker (< 0) or null
  const int32_t* view_base;
  int64_t ld;
  int n_views;
  float in_scale;           // applied to dL/d(outputs) before rounding to 16 bit
  float out_scale;          // applied to dX and dW (FP32) on the way out
  uint32_t wait_limit;      // polls per bounded wait (0: give up at once)
  unsigned* status;
  FieldDev f[kMaxViews];
};

// One thread: weight-gradient MMA, D (M = 64 rows x N) += A^T B over the tile's 128 samples.
// A (rows = M units) and B (rows = N units) are [sample][units] K-major activation buffers
// read MN-major: unit groups 128 B apart, sample groups units*16 B apart.
__device__ __forceinline__ void issue_dw(uint32_t d_tmem, uint32_t a_saddr, int a_units, uint32_t b_saddr,
                                         int b_units, int N, bool accumulate, bool bf16) {
  const uint32_t idesc = tc::idesc_f16(64, N, bf16) | (1u << 15) | (1u << 16);
  for (int kk = 0; kk < kTM / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 32 * a_units, a_units * 16, 128);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 32 * b_units, b_units * 16, 128);
    tc::mma_f16(d_tmem, ad, bd, idesc, (accumulate || kk > 0) ? 1u : 0u);
  }
}

template <bool BF16>
__device__ void stage_bwd_weights(uint8_t* sm, const FieldDev& F) {
  const WOff off(F.mlp_in);
  const int in = F.mlp_in;
  if (in == 16)
    stage<BF16, false, 64, 16>(sm + B_W1, F.weights, off, in, 1);
  else
    stage<BF16, false, 64, 32>(sm + B_W1, F.weights, off, in, 1);
  stage<BF16, false, 64, 64>(sm + B_W2, F.weights, off, in, 2);
  stage<BF16, false, 16, 64>(sm + B_W3, F.weights, off, in, 3);
  stage<BF16, false, 64, 16>(sm + B_W4, F.weights, off, in, 4);
  stage<BF16, false, 16, 64>(sm + B_W5, F.weights, off, in, 5);
}

// One thread: adjoint-chain MMA D (128 x N) = dY (smem, 128 x K, K-major) * W, with W the
// forward weight [K rows][N columns] (K-major in its own layout) read as an MN-major
// operand: column groups 128 B apart, row groups N*16 B apart.
__device__ __forceinline__ void issue_adjoint(uint32_t d_tmem, uint32_t a_saddr, uint32_t w_saddr, int K, int N,
                                              bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16) | (1u << 16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(w_saddr + kk * 32 * N, N * 16, 128);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

// Read the M = 64 weight-gradient accumulators and add them to the field's gradient buffer.
__device__ void flush_dw(uint32_t tmem, const FieldDev& F, float scale) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const int row = warp * 16 + lane;  // valid for lane < 16
  const WOff off(F.mlp_in);
  const int in = F.mlp_in;
  float* G = F.grad_weights;
  float v[16];
  // dW2 [64 out][64 in]
  for (int c = 0; c < 4; ++c) {
    tc::tmem_ld16(taddr + C_DW2 + 16 * c, v);
    if (lane < 16)
      for (int j = 0; j < 16; ++j) atomicAdd(G + off.w2 + row * kHidden + 16 * c + j, v[j] * scale);
  }
  // dW1 [64 out][in]
  for (int c = 0; c < in / 16; ++c) {
    tc::tmem_ld16(taddr + C_DW1 + 16 * c, v);
    if (lane < 16)
      for (int j = 0; j < 16; ++j) atomicAdd(G + off.w1 + row * in + 16 * c + j, v[j] * scale);
  }
  // dW4p [64 out][16 in], column 0 is padding
  tc::tmem_ld16(taddr + C_DW4, v);
  if (lane < 16)
    for (int j = 1; j < 16; ++j) atomicAdd(G + off.w4 + row * (kGeoOut - 1) + j - 1, v[j] * scale);
  // dW3^T [64 in][16 out]
  tc::tmem_ld16(taddr + C_DW3T, v);
  if (lane < 16)
    for (int j = 0; j < 16; ++j) atomicAdd(G + off.w3 + j * kHidden + row, v[j] * scale);
  // dW5p^T [64 in][16 out], outputs 3..15 are padding
  tc::tmem_ld16(taddr + C_DW5T, v);
  if (lane < 16)
    for (int j = 0; j < 3; ++j) atomicAdd(G + off.w5 + j * kColHidden + row, v[j] * scale);
}

// The CTA's tiles: from `tile` on in steps of gridDim.x, the first whose view has this
// kernel's MLP kind (uniform over the CTA), or n_tiles.
__device__ __forceinline__ int64_t next_tile(const TcBwdArgs& A, int64_t tile, int64_t n_tiles, int kind) {
  for (; tile < n_tiles; tile += gridDim.x)
    if (A.f[view_of_slot(A.view_base, A.n_views, tile * kTM)].mlp_kind == kind) return tile;
  return n_tiles;
}

// One thread: the 16 bulk copies of tile `tile`'s X (one row group of 8 samples each).
__device__ __forceinline__ void load_x(const TcBwdArgs& A, int64_t tile, uint32_t dst, uint32_t bar) {
  const uint32_t group = (uint32_t)A.f[view_of_slot(A.view_base, A.n_views, tile * kTM)].mlp_in * 16;
  tc::mbar_expect_tx(bar, 16 * group);
  const uint8_t* src = static_cast<const uint8_t*>(A.feat);
  for (int g = 0; g < 16; ++g) tc::bulk_g2s(dst + g * group, src + feat16_group_offset(A.ld, tile, g), group, bar);
}

// This thread's dL/do_0 and dL/dz_rgb of tile `tile` (zero for padding), scaled by in_scale.
__device__ __forceinline__ void load_dout(const TcBwdArgs& A, int64_t tile, int64_t S, int t, float (&d)[4]) {
  const int64_t s = tile * kTM + t;
  const bool live = s < S && (!A.s_ray || A.s_ray[s] >= 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = live ? A.dout[(int64_t)i * A.ld + s] * A.in_scale : 0.0f;
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsB, 2) k_mlp_bwd_tc(const __grid_constant__ TcBwdArgs A) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((int64_t)A.view_base[A.n_views] > A.ld) return;  // overflow flagged by the scan
  const int t = threadIdx.x, warp = t >> 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + B_MISC + 16);
  const uint32_t mbar = tc::smem_u32(sm + B_MISC);      // MMA completion
  const uint32_t xbar = tc::smem_u32(sm + B_MISC + 8);  // X copies landed
  const uint32_t sb = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemColsB);
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(xbar, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row_t = tmem + ((uint32_t)(warp * 32) << 16);
  const int kind = BF16 ? kMlpBF16 : kMlpF16;

  const int64_t S = (int64_t)A.view_base[A.n_views];
  const int64_t n_tiles = (S + kTM - 1) / kTM;
  int cur = -1;            // view whose field's weights are staged
  bool dw_live = false;    // weight-gradient accumulators hold data
  uint32_t phase = 0, xphase = 0, xbuf = 0;
  bool ok = true, mma_pending = false, x_pending = false;

  int64_t tile = next_tile(A, blockIdx.x, n_tiles, kind);
  float dnext[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (tile < n_tiles) {
    if (t == 0) load_x(A, tile, sb + B_X, xbar);
    x_pending = true;
    load_dout(A, tile, S, t, dnext);
  }

  // wait for the MMAs committed last; all threads, bounded
#define INVR_CHAIN_WAIT()                                   \
  mma_pending = true;                                       \
  ok = tc::mbar_wait(mbar, phase, A.wait_limit);            \
  if (!__syncthreads_and(ok)) { ok = false; break; }        \
  phase ^= 1u;                                              \
  mma_pending = false;                                      \
  tc::fence_after_sync();

  while (tile < n_tiles) {
    const int64_t s0 = tile * kTM;
    const int v = view_of_slot(A.view_base, A.n_views, s0);
    const FieldDev& F = A.f[v];
    const int64_t nxt = next_tile(A, tile + gridDim.x, n_tiles, kind);
    if (cur < 0 || F.weights != A.f[cur].weights) {
      if (dw_live) {
        if (t == 0) tc::commit_to(mbar);
        INVR_CHAIN_WAIT();
        flush_dw(tmem, A.f[cur], A.out_scale);
        tc::fence_before_sync();
        __syncthreads();
        dw_live = false;
      }
      stage_bwd_weights<BF16>(sm, F);
      cur = v;
    }
    const int in = F.mlp_in;
    const int valid = (int)(S - s0 < kTM ? S - s0 : kTM);
    const uint32_t bx = B_X + xbuf * (kTM * 32 * 2);
    // ---- dZ row (dL/dz for rgb; zero for the padded outputs) and dL/do_0 of this tile
    const float do0 = dnext[0];
    {
      float dz[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) dz[i] = i < 3 ? dnext[1 + i] : 0.0f;
      row16_out<BF16>(dz, sm + B_DZ, t);
    }
    operands_ready();
    ok = tc::mbar_wait(xbar, xphase, A.wait_limit);
    if (!__syncthreads_and(ok)) { ok = false; break; }
    xphase ^= 1u;
    x_pending = false;
    // the next tile's X (into the other buffer) and dL/d(outputs) arrive under this chain
    if (nxt < n_tiles) {
      if (t == 0) load_x(A, nxt, sb + B_X + (xbuf ^ 1u) * (kTM * 32 * 2), xbar);
      x_pending = true;
      load_dout(A, nxt, S, t, dnext);
    }
    // ---- recompute: H1
    if (t == 0) {
      tc::fence_after_sync();
      issue_chain(tmem + C_CHAIN, sb + bx, sb + B_W1, in, 64, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, false>(row_t + C_CHAIN, sm + B_H1, nullptr, t);
    operands_ready();
    // ---- H2
    if (t == 0) {
      tc::fence_after_sync();
      issue_chain(tmem + C_CHAIN, sb + B_H1, sb + B_W2, 64, 64, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, false>(row_t + C_CHAIN, sm + B_H2, nullptr, t);
    operands_ready();
    // ---- O = (0, o_1..o_15)
    if (t == 0) {
      tc::fence_after_sync();
      issue_chain(tmem + C_CHAIN, sb + B_H2, sb + B_W3, 64, 16, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    {
      float o[16];
      tc::tmem_ld16(row_t + C_CHAIN, o);
      o[0] = 0.0f;
      row16_out<BF16>(o, sm + B_O, t);
    }
    operands_ready();
    // ---- H4
    if (t == 0) {
      tc::fence_after_sync();
      issue_chain(tmem + C_CHAIN, sb + B_O, sb + B_W4, 16, 64, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, false>(row_t + C_CHAIN, sm + B_H4, nullptr, t);
    operands_ready();
    // ---- dH4 = (dZ W5p) * [H4 > 0] (over H4);  dW5p^T += H4^T dZ
    if (t == 0) {
      tc::fence_after_sync();
      issue_adjoint(tmem + C_CHAIN, sb + B_DZ, sb + B_W5, 16, 64, BF16);
      issue_dw(tmem + C_DW5T, sb + B_H4, 64, sb + B_DZ, 16, 16, dw_live, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, true>(row_t + C_CHAIN, sm + B_DH4, sm + B_H4, t);
    operands_ready();
    // ---- dO = dH4 W4p (o_0 slot carries dL/do_0; over dZ);  dW4p += dH4^T O
    if (t == 0) {
      tc::fence_after_sync();
      issue_adjoint(tmem + C_CHAIN, sb + B_DH4, sb + B_W4, 64, 16, BF16);
      issue_dw(tmem + C_DW4, sb + B_DH4, 64, sb + B_O, 16, 16, dw_live, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    {
      float d[16];
      tc::tmem_ld16(row_t + C_CHAIN, d);
      d[0] = do0;
      row16_out<BF16>(d, sm + B_DO, t);
    }
    operands_ready();
    // ---- dH2 = (dO W3) * [H2 > 0] (over H2);  dW3^T += H2^T dO
    if (t == 0) {
      tc::fence_after_sync();
      issue_adjoint(tmem + C_CHAIN, sb + B_DO, sb + B_W3, 16, 64, BF16);
      issue_dw(tmem + C_DW3T, sb + B_H2, 64, sb + B_DO, 16, 16, dw_live, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, true>(row_t + C_CHAIN, sm + B_DH2, sm + B_H2, t);
    operands_ready();
    // ---- dH1 = (dH2 W2) * [H1 > 0] (over H1);  dW2 += dH2^T H1
    if (t == 0) {
      tc::fence_after_sync();
      issue_adjoint(tmem + C_CHAIN, sb + B_DH2, sb + B_W2, 64, 64, BF16);
      issue_dw(tmem + C_DW2, sb + B_DH2, 64, sb + B_H1, 64, 64, dw_live, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    row64_out<BF16, true>(row_t + C_CHAIN, sm + B_DH1, sm + B_H1, t);
    operands_ready();
    // ---- dX = dH1 W1;  dW1 += dH1^T X
    if (t == 0) {
      tc::fence_after_sync();
      issue_adjoint(tmem + C_CHAIN, sb + B_DH1, sb + B_W1, 64, in, BF16);
      issue_dw(tmem + C_DW1, sb + B_DH1, 64, sb + bx, in, in, dw_live, BF16);
      tc::commit_to(mbar);
    }
    INVR_CHAIN_WAIT();
    dw_live = true;
    if (in == 32) {
      float d[32];
      tc::tmem_ld32(row_t + C_CHAIN, d);
      if (t < valid)
#pragma unroll
        for (int j = 0; j < 32; ++j) A.dfeat[(int64_t)j * A.ld + s0 + t] = d[j] * A.out_scale;
    } else {
      float d[16];
      tc::tmem_ld16(row_t + C_CHAIN, d);
      if (t < valid)
#pragma unroll
        for (int j = 0; j < 16; ++j) A.dfeat[(int64_t)j * A.ld + s0 + t] = d[j] * A.out_scale;
    }
    tc::fence_before_sync();
    __syncthreads();
    xbuf ^= 1u;
    tile = nxt;
  }
#undef INVR_CHAIN_WAIT
  if (ok && dw_live) {
    tc::fence_after_sync();
    flush_dw(tmem, A.f[cur], A.out_scale);  // every MMA completed at the last chain wait
  }
  if (!ok) {
    // a wait gave up: record it, then let this CTA's MMAs and copies in flight finish
    // (bounded) before the tensor memory and shared memory they write are released
    if (t == 0) atomicOr(A.status, kStatusTimeout);
    if (mma_pending) tc::mbar_wait(mbar, phase, kWaitLimit);
    if (x_pending) tc::mbar_wait(xbar, xphase, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemColsB);
  }
}

}  // namespace

cudaError_t launch_mlp_bwd_tc(const Plan& P, int num_sms, cudaStream_t s) {
  TcBwdArgs A{};
  A.feat = P.ws.feat;
  A.dout = P.ws.dout;
  A.dfeat = P.ws.dfeat;
  A.s_ray = P.ws.s_ray;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n_views = P.n_views;
  // dL/dout carries the loss's 1 / (3 R); take it out of the 16-bit operands
  A.in_scale = P.grad_scale / P.loss_norm;
  A.out_scale = P.loss_norm;
  A.wait_limit = P.wait_limit;
  A.status = P.status;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  cudaError_t e = cudaSuccess;
  if (plan_has_kind(P, kMlpBF16)) {
    cudaFuncSetAttribute(k_mlp_bwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemB);
    k_mlp_bwd_tc<true><<<num_sms * 2, kThreadsB, kSmemB, s>>>(A);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && plan_has_kind(P, kMlpF16)) {
    cudaFuncSetAttribute(k_mlp_bwd_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemB);
    k_mlp_bwd_tc<false><<<num_sms * 2, kThreadsB, kSmemB, s>>>(A);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace invr
