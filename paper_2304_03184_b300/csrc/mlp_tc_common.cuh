// Pieces shared by the tensor-core MLP kernels (forward and backward): the weight layout
// of W1..W5, MMA chains over K, and the ReLU epilogue from tensor memory.
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

// One thread: D(tmem) = A(tmem, 128 x K: 8 columns per K step of 16) * B(smem, N x K, K-major)^T.
__device__ __forceinline__ void issue_chain_ts(uint32_t d_tmem, uint32_t a_tmem, uint32_t b_saddr, int K, int N,
                                               bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t bd = tc::smem_desc(b_saddr + kk * 256, 128, K * 16);
    tc::mma_f16_ts(d_tmem, a_tmem + kk * 8, bd, idesc, kk > 0 ? 1u : 0u);
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

// The epilogues below write the next MMA's 16-bit A operand row t twice when TS: into shared
// memory (K-major layout, for the weight-gradient MMAs) and into this thread's tensor-memory
// lane at column `aop` (packed pairs, for the chain MMA, which then reads A from tensor
// memory and leaves the shared-memory bandwidth to B).

// Store 32 packed words as row t of a K = 64 operand (and in tensor memory if TS).
template <bool TS>
__device__ __forceinline__ void put_row64(const uint32_t (&w)[32], uint8_t* dst, int t, uint32_t aop) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8 * c, 64)) =
        make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
  if constexpr (TS) tc::tmem_st32(aop, w);
}

// Read 64 accumulator columns of this thread's row (one tcgen05.ld); write max(v, 0).
template <bool BF16, bool TS>
__device__ __forceinline__ void row64_relu(uint32_t taddr, uint8_t* dst, int t, uint32_t aop) {
  float v[64];
  tc::tmem_ld64(taddr, v);
  uint32_t w[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) w[c] = tc::pack2<BF16>(fmaxf(v[2 * c], 0.0f), fmaxf(v[2 * c + 1], 0.0f));
  put_row64<TS>(w, dst, t, aop);
}

// Read 64 accumulator columns of this thread's row; write each value where its unit's ReLU
// decision (bit j of m[j / 32], from the training forward) is positive, else 0.
template <bool BF16, bool TS>
__device__ __forceinline__ void row64_masked(uint32_t taddr, uint8_t* dst, uint32_t m0, uint32_t m1, int t,
                                             uint32_t aop) {
  float v[64];
  tc::tmem_ld64(taddr, v);
  uint32_t w[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t b = (c < 16 ? m0 : m1) >> (2 * (c & 15));
    w[c] = tc::pack2<BF16>((b & 1u) ? v[2 * c] : 0.0f, (b & 2u) ? v[2 * c + 1] : 0.0f);
  }
  put_row64<TS>(w, dst, t, aop);
}

// Write a row of 16 values as row t of a K = 16 16-bit operand (and in tensor memory if TS).
template <bool BF16, bool TS>
__device__ __forceinline__ void row16_out(const float (&v)[16], uint8_t* dst, int t, uint32_t aop) {
  uint32_t w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = tc::pack2<BF16>(v[2 * c], v[2 * c + 1]);
  *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 0, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(t, 8, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
  if constexpr (TS) tc::tmem_st8(aop, w);
}

// Operand writes done by every thread -> visible to the tensor core; TMEM reads ordered.
__device__ __forceinline__ void operands_ready() {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
}

}  // namespace mlp_tc
}  // namespace invr
