// Geometry + colour MLPs on the 5th-generation tensor cores (tcgen05, kind::f16): FP16 or
// BF16 operands, FP32 accumulation in tensor memory (the mixed-precision path; Sec. 4.2
// geometry MLP E_g and colour MLP E_c).
//
// One CTA = 128 threads = one warpgroup; a tile is 128 samples, thread t owns sample t,
// which is row t of every MMA (M = 128) and lane t of tensor memory.  Per tile the five
// layers run as a chain:
//   X [128 x in]  -> D1 = X W1^T (N 64)  -> ReLU -> H1 (smem, 16-bit)
//   H1            -> D2 = H1 W2^T (N 64) -> ReLU -> H2
//   H2            -> D3 = H2 W3^T (N 16) -> sigma = exp(o_0); O = (0, o_1..o_15)
//   O             -> D4 = O W4p^T (N 64) -> ReLU -> H4 (reuses H1)
//   H4            -> D5 = H4 W5p^T (N 16) -> rgb = sigmoid(z_0..z_2)
// One elected thread issues each layer's MMAs (K = 16 per instruction) and commits them to
// an mbarrier; all threads wait, read their row from tensor memory (tcgen05.ld 32x32b),
// apply the activation in FP32, and write the next operand row in the K-major layout.
// Weights (padded: W4p gets a zero column for o_0, W5p 13 zero rows) are converted to 16
// bit and staged in shared memory once per field.  Several CTAs per SM overlap their
// chains.  Every mbarrier wait is bounded; a timeout sets the status word and the CTA frees
// its tensor memory and exits.
#include "invr_internal.cuh"
#include "tc_ptx.cuh"

namespace invr {

namespace {

constexpr int kTM = 128;             // samples per tile = MMA M
constexpr int kThreadsTC = 128;
constexpr uint32_t kTmemCols = 128;  // D1/D3/D5 in columns 0..63, D2/D4 in 64..127
constexpr uint32_t kWaitLimit = 1u << 22;  // polls of try_wait (bounded: a few seconds)

// shared-memory plan (bytes)
constexpr uint32_t OFF_W1 = 0;                       // 64 x 32
constexpr uint32_t OFF_W2 = OFF_W1 + 64 * 32 * 2;    // 64 x 64
constexpr uint32_t OFF_W3 = OFF_W2 + 64 * 64 * 2;    // 16 x 64
constexpr uint32_t OFF_W4 = OFF_W3 + 16 * 64 * 2;    // 64 x 16
constexpr uint32_t OFF_W5 = OFF_W4 + 64 * 16 * 2;    // 16 x 64
constexpr uint32_t OFF_X = OFF_W5 + 16 * 64 * 2;     // 128 x 32
constexpr uint32_t OFF_H1 = OFF_X + kTM * 32 * 2;    // 128 x 64 (H1, then H4)
constexpr uint32_t OFF_H2 = OFF_H1 + kTM * 64 * 2;   // 128 x 64
constexpr uint32_t OFF_O = OFF_H2 + kTM * 64 * 2;    // 128 x 16
constexpr uint32_t OFF_MISC = OFF_O + kTM * 16 * 2;  // mbarrier (8 B) + TMEM base (4 B)
constexpr uint32_t kSmemTC = OFF_MISC + 64 + 4096;   // + guard band

struct TcArgs {
  const float* feat;        // [in][ld] FP32
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

template <bool BF16>
__device__ void stage_weights(uint8_t* sm, const FieldDev& F) {
  const WOff off(F.mlp_in);
  if (F.mlp_in == 16)
    stage_weight<BF16, 64, 16>(sm + OFF_W1, F.weights, 1, 16, off);
  else
    stage_weight<BF16, 64, 32>(sm + OFF_W1, F.weights, 1, 32, off);
  stage_weight<BF16, 64, 64>(sm + OFF_W2, F.weights, 2, F.mlp_in, off);
  stage_weight<BF16, 16, 64>(sm + OFF_W3, F.weights, 3, F.mlp_in, off);
  stage_weight<BF16, 64, 16>(sm + OFF_W4, F.weights, 4, F.mlp_in, off);
  stage_weight<BF16, 16, 64>(sm + OFF_W5, F.weights, 5, F.mlp_in, off);
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

// Read 64 accumulator columns of this thread's row, apply ReLU, store as row t of a K=64
// 16-bit operand.
template <bool BF16>
__device__ __forceinline__ void relu_row64(uint32_t taddr, uint8_t* dst, int t) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(taddr + 16 * c, v);
    uint4 lo, hi;
    lo.x = tc::pack2<BF16>(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f));
    lo.y = tc::pack2<BF16>(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f));
    lo.z = tc::pack2<BF16>(fmaxf(v[4], 0.f), fmaxf(v[5], 0.f));
    lo.w = tc::pack2<BF16>(fmaxf(v[6], 0.f), fmaxf(v[7], 0.f));
    hi.x = tc::pack2<BF16>(fmaxf(v[8], 0.f), fmaxf(v[9], 0.f));
    hi.y = tc::pack2<BF16>(fmaxf(v[10], 0.f), fmaxf(v[11], 0.f));
    hi.z = tc::pack2<BF16>(fmaxf(v[12], 0.f), fmaxf(v[13], 0.f));
    hi.w = tc::pack2<BF16>(fmaxf(v[14], 0.f), fmaxf(v[15], 0.f));
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 16 * c, 64)) = lo;
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 16 * c + 8, 64)) = hi;
  }
}

// Operand writes done by every thread -> visible to the tensor core; TMEM reads ordered.
__device__ __forceinline__ void operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsTC, 3) k_mlp_fwd_tc(const __grid_constant__ TcArgs A) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if (A.view_base && (int64_t)A.view_base[A.n_views] > A.ld) return;  // overflow flagged by the scan
  const int t = threadIdx.x, warp = t >> 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 8);
  const uint32_t mbar = tc::smem_u32(sm + OFF_MISC);
  const uint32_t sbase = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
  if (t == 0) tc::mbar_init(mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t row_taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const int kind = BF16 ? kMlpBF16 : kMlpF16;

  const int64_t S = A.view_base ? (int64_t)A.view_base[A.n_views] : A.n;
  const int64_t n_tiles = (S + kTM - 1) / kTM;
  const float* loaded = nullptr;
  uint32_t phase = 0;
  bool ok = true;

  for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int64_t s0 = tile * kTM;
    const FieldDev& F = A.f[A.view_base ? view_of_slot(A.view_base, A.n_views, s0) : 0];
    if (F.mlp_kind != kind) continue;  // uniform over the CTA
    if (F.weights != loaded) {
      __syncthreads();
      stage_weights<BF16>(sm, F);
      loaded = F.weights;
    }
    const int in = F.mlp_in;
    const int valid = (int)(S - s0 < kTM ? S - s0 : kTM);
    // ---- X: this thread's features (FP32, feature-major in global) -> row t
    for (int j = 0; j < in / 8; ++j) {
      float x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = t < valid ? A.feat[(int64_t)(8 * j + i) * A.ld + s0 + t] : 0.0f;
      uint4 q;
      q.x = tc::pack2<BF16>(x[0], x[1]);
      q.y = tc::pack2<BF16>(x[2], x[3]);
      q.z = tc::pack2<BF16>(x[4], x[5]);
      q.w = tc::pack2<BF16>(x[6], x[7]);
      *reinterpret_cast<uint4*>(sm + OFF_X + tc::kmajor_offset(t, 8 * j, in)) = q;
    }
    operands_ready();
    // ---- layer 1
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem + 0, sbase + OFF_X, sbase + OFF_W1, in, 64, BF16);
      tc::commit_to(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr + 0, sm + OFF_H1, t);
    operands_ready();
    // ---- layer 2
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem + 64, sbase + OFF_H1, sbase + OFF_W2, 64, 64, BF16);
      tc::commit_to(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr + 64, sm + OFF_H2, t);
    operands_ready();
    // ---- layer 3: geometry output o (16)
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem + 0, sbase + OFF_H2, sbase + OFF_W3, 64, 16, BF16);
      tc::commit_to(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    float o[16];
    tc::tmem_ld16(row_taddr + 0, o);
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
      *reinterpret_cast<uint4*>(sm + OFF_O + tc::kmajor_offset(t, 0, 16)) = lo;
      *reinterpret_cast<uint4*>(sm + OFF_O + tc::kmajor_offset(t, 8, 16)) = hi;
    }
    operands_ready();
    // ---- layer 4: colour hidden
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem + 64, sbase + OFF_O, sbase + OFF_W4, 16, 64, BF16);
      tc::commit_to(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    relu_row64<BF16>(row_taddr + 64, sm + OFF_H1, t);
    operands_ready();
    // ---- layer 5: colour output
    if (t == 0) {
      tc::fence_after_sync();
      issue_layer(tmem + 16, sbase + OFF_H1, sbase + OFF_W5, 64, 16, BF16);
      tc::commit_to(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, A.wait_limit);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after_sync();
    float z[16];
    tc::tmem_ld16(row_taddr + 16, z);
    if (t < valid) {
      const int64_t gs = s0 + t;
      A.out[gs] = sigma;
      A.out[A.ld + gs] = 1.0f / (1.0f + expf(-z[0]));
      A.out[2 * A.ld + gs] = 1.0f / (1.0f + expf(-z[1]));
      A.out[3 * A.ld + gs] = 1.0f / (1.0f + expf(-z[2]));
    }
    tc::fence_before_sync();
    __syncthreads();  // every thread is done with this tile's TMEM and operands
  }
  if (!ok) {
    // a wait gave up: record it, then let the pending MMAs finish (bounded) before the
    // tensor memory they write is freed
    if (t == 0) atomicOr(A.status, kStatusTimeout);
    tc::mbar_wait(mbar, phase ^ 1u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool BF16>
cudaError_t launch_tc(const TcArgs& A, int num_sms, cudaStream_t s) {
  cudaFuncSetAttribute(k_mlp_fwd_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC);
  k_mlp_fwd_tc<BF16><<<num_sms * 3, kThreadsTC, kSmemTC, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

bool plan_has_kind(const Plan& P, int kind) {
  for (int v = 0; v < P.n_views; ++v)
    if (P.v[v].field.mlp_kind == kind) return true;
  return false;
}

cudaError_t launch_mlp_fwd_tc(const Plan& P, int num_sms, cudaStream_t s) {
  TcArgs A{};
  A.feat = static_cast<const float*>(P.ws.feat);
  A.out = P.ws.out;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n_views = P.n_views;
  A.wait_limit = P.wait_limit;
  A.status = P.status;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  cudaError_t e = cudaSuccess;
  if (plan_has_kind(P, kMlpBF16)) e = launch_tc<true>(A, num_sms, s);
  if (e == cudaSuccess && plan_has_kind(P, kMlpF16)) e = launch_tc<false>(A, num_sms, s);
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
  return f.mlp_kind == kMlpBF16 ? launch_tc<true>(A, num_sms, s) : launch_tc<false>(A, num_sms, s);
}

}  // namespace invr
