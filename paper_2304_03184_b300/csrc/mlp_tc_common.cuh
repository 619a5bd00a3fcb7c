// Pieces shared by the tensor-core MLP kernels (forward and backward): the weight layout
// of W1..W5, staging of (padded, optionally transposed) weights as 16-bit K-major
// operands, MMA chains over K, and the ReLU epilogue from tensor memory.
#pragma once

#include "invr_internal.cuh"
#include "tc_ptx.cuh"

namespace invr {
namespace mlp_tc {

constexpr int kTM = 128;                     // samples per tile = MMA M of the chain
constexpr uint32_t kWaitLimit = 1u << 22;    // polls of try_wait (bounded: a few seconds)

// Offsets of W1..W5 in the flat FP32 weight array (row-major [out][in]).
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

// Element [o][k] of padded layer `layer` (1..5): W4p has a zero column 0 (o_0 does not feed
// the colour MLP), W5p has zero rows 3..15.
__device__ __forceinline__ float padded_weight(const float* __restrict__ W, const WOff& off, int in, int layer,
                                               int o, int k) {
  switch (layer) {
    case 1: return W[off.w1 + o * in + k];
    case 2: return W[off.w2 + o * kHidden + k];
    case 3: return W[off.w3 + o * kHidden + k];
    case 4: return k == 0 ? 0.0f : W[off.w4 + o * (kGeoOut - 1) + k - 1];
    default: return o < 3 ? W[off.w5 + o * kColHidden + k] : 0.0f;
  }
}

// Stage padded layer `layer` ([OUT][IN]) as a 16-bit K-major operand with N rows and K
// columns: the matrix itself (N = OUT, K = IN) or, if TRANS, its transpose (N = IN, K = OUT).
// Threads tid = 0..nthr-1 share the work.
template <bool BF16, bool TRANS, int N, int K>
__device__ __forceinline__ void stage(uint8_t* dst, const float* __restrict__ W, const WOff& off, int in,
                                      int layer, int tid, int nthr) {
  for (int e = tid; e < N * K / 2; e += nthr) {
    const int n = (2 * e) / K, k = (2 * e) % K;
    const float a = TRANS ? padded_weight(W, off, in, layer, k, n) : padded_weight(W, off, in, layer, n, k);
    const float b =
        TRANS ? padded_weight(W, off, in, layer, k + 1, n) : padded_weight(W, off, in, layer, n, k + 1);
    *reinterpret_cast<uint32_t*>(dst + tc::kmajor_offset(n, k, K)) = tc::pack2<BF16>(a, b);
  }
}

// One thread: D(tmem) (+)= A(smem, 128 x K, K-major) * B(smem, N x K, K-major)^T.
__device__ __forceinline__ void issue_chain(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N,
                                            bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = tc::smem_desc(a_saddr + kk * 256, 128, K * 16);
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
  }
}

// Read 64 accumulator columns of this thread's row (one tcgen05.ld); write max(v, 0) as row t
// of a K = 64 16-bit operand.
template <bool BF16>
__device__ __forceinline__ void row64_relu(uint32_t taddr, uint8_t* dst, int t) {
  float v[64];
  tc::tmem_ld64(taddr, v);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float* x = v + 8 * c;
    uint4 q;
    q.x = tc::pack2<BF16>(fmaxf(x[0], 0.0f), fmaxf(x[1], 0.0f));
    q.y = tc::pack2<BF16>(fmaxf(x[2], 0.0f), fmaxf(x[3], 0.0f));
    q.z = tc::pack2<BF16>(fmaxf(x[4], 0.0f), fmaxf(x[5], 0.0f));
    q.w = tc::pack2<BF16>(fmaxf(x[6], 0.0f), fmaxf(x[7], 0.0f));
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8 * c, 64)) = q;
  }
}

// Read 64 accumulator columns of this thread's row; write each value where its unit's ReLU
// decision (bit j of m[j / 32], from the training forward) is positive, else 0, as row t of
// a K = 64 16-bit operand.
template <bool BF16>
__device__ __forceinline__ void row64_masked(uint32_t taddr, uint8_t* dst, uint32_t m0, uint32_t m1, int t) {
  float v[64];
  tc::tmem_ld64(taddr, v);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t b = (c < 4 ? m0 : m1) >> (8 * (c & 3));
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = ((b >> i) & 1u) ? v[8 * c + i] : 0.0f;
    uint4 q;
    q.x = tc::pack2<BF16>(x[0], x[1]);
    q.y = tc::pack2<BF16>(x[2], x[3]);
    q.z = tc::pack2<BF16>(x[4], x[5]);
    q.w = tc::pack2<BF16>(x[6], x[7]);
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8 * c, 64)) = q;
  }
}

// Write a row of 16 values as row t of a K = 16 16-bit operand.
template <bool BF16>
__device__ __forceinline__ void row16_out(const float (&v)[16], uint8_t* dst, int t) {
  uint4 lo, hi;
  lo.x = tc::pack2<BF16>(v[0], v[1]);
  lo.y = tc::pack2<BF16>(v[2], v[3]);
  lo.z = tc::pack2<BF16>(v[4], v[5]);
  lo.w = tc::pack2<BF16>(v[6], v[7]);
  hi.x = tc::pack2<BF16>(v[8], v[9]);
  hi.y = tc::pack2<BF16>(v[10], v[11]);
  hi.z = tc::pack2<BF16>(v[12], v[13]);
  hi.w = tc::pack2<BF16>(v[14], v[15]);
  *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 0, 16)) = lo;
  *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8, 16)) = hi;
}

// Operand writes done by every thread -> visible to the tensor core; TMEM reads ordered.
__device__ __forceinline__ void operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
}

}  // namespace mlp_tc
}  // namespace invr
