// Backward of the geometry + colour MLPs on the tcgen05 tensor cores, 16-bit operands (the
// field's FP16 or BF16) with FP32 accumulation (mixed-precision fields).  The incoming
// dL/d(outputs) are multiplied by in_scale (the inverse of the loss's mean normalisation,
// so per-sample gradients are O(1) and do not underflow FP16) and the FP32 results (dX,
// dW) by out_scale on the way out.
//
// Per 128-sample tile (epilogue thread t = sample t, row t of every M = 128 MMA):
//   recompute  X -> H1 -> H2 -> O -> H4          (4 chained MMAs, ReLU epilogues)
//   adjoint    dZ -> dH4 -> dO -> dH2 -> dH1 -> dX (5 chained MMAs; each reads the forward
//              weight as an MN-major operand; the ReLU decisions are the training forward's,
//              taken on split products, one bit per unit and sample)
// Every chain MMA after the first reads its A operand from tensor memory: each epilogue
// writes its 16-bit row twice, into shared memory for the weight-gradient MMAs and into its
// tensor-memory lane for the next chain MMA, which then streams only B from shared memory.
//   weights    dW5^T += H4^T dZ, dW4 += dH4^T O, dW3^T += H2^T dO, dW2 += dH2^T H1,
//              dW1 += dH1^T X: M = 64 MMAs with K = the 128 samples, accumulated in tensor
//              memory over every tile the CTA visits.
// The weight-gradient MMAs read the [sample][unit] activation buffers as MN-major operands
// (each 8 x 16-byte core matrix holds 8 units of 8 samples), so no transposed copies exist.
//
// Warp roles.  A tcgen05.mma instruction costs its issuing thread ~60 clocks whatever its
// size (N <= 128), and a tile needs 65 of them, so one CTA = 4 epilogue warps + 1 issuer
// warp.  The issuer waits for the epilogue's "operands ready" mbarrier (128 arrivals), issues
// a stage's chain MMAs, commits them to the "accumulator ready" mbarrier, and only then
// issues that stage's weight-gradient MMAs, which run while the epilogue works; the next
// commit (tracking every earlier MMA) retires them.  The buffers are assigned so that an
// epilogue never writes what the current stage's weight-gradient MMAs read: dH4 into its
// own buffer, dO over dZ, dH2 over H4, dH1 over H2.  The issuer also moves X: the encoder's
// 16-bit operand tile arrives by one TMA copy into one of two buffers, the next tile's
// copy issued once this tile's first MMA has retired the previous tile's last
// weight-gradient MMAs.  Epilogue threads load the next tile's dL/d(outputs) and padding
// markers into registers under the chain (unconditionally; the padding selection is
// applied when they are used).  106 KB of shared memory and 160 threads: two CTAs per SM.
// The accumulated dW are read out once per field, after the issuer's "flush" commit (M = 64
// accumulator: row r in TMEM lane 32 (r / 16) + r % 16), and added to the gradient buffer
// with one atomic per weight per CTA.  dL/dX (the encoding features' gradient) is written
// FP32 feature-major for the hash scatter.  All waits are bounded: a role that gives up sets
// the status word and leaves its loop (the other role's waits then give up in turn), and the
// issuer retires its MMAs and copies (bounded) before the tensor memory is freed.
#include <cuda.h>

#include "mlp_tc_common.cuh"

namespace invr {

namespace {

using namespace mlp_tc;

constexpr int kEpi = 128;       // epilogue threads (warps 0..3)
constexpr int kThreadsB = 160;  // + the issuer warp (warp 4)
constexpr uint32_t kTmemColsB = 256;
// tensor-memory columns
constexpr uint32_t C_CHAIN = 0;     // 64: the chain's current layer
constexpr uint32_t C_DW2 = 64;      // 64
constexpr uint32_t C_DW1 = 128;     // 32
constexpr uint32_t C_DW4 = 160;     // 16
constexpr uint32_t C_DW3T = 176;    // 16
constexpr uint32_t C_DW5T = 192;    // 16
constexpr uint32_t C_AOP = 208;     // 32: the chain MMA's A operand (16-bit, packed in pairs)

// shared-memory plan (bytes); [n][k] = K-major operand with n rows and k columns.  The
// transposed products of the adjoint chain read the forward weights as MN-major operands.
constexpr uint32_t B_W1 = 0;                   // [64][32] forward weights (W4p, W5p padded)
constexpr uint32_t B_W2 = B_W1 + 64 * 32 * 2;  // [64][64]
constexpr uint32_t B_W3 = B_W2 + 64 * 64 * 2;  // [16][64]
constexpr uint32_t B_W4 = B_W3 + 16 * 64 * 2;  // [64][16]
constexpr uint32_t B_W5 = B_W4 + 16 * 64 * 2;  // [16][64]
constexpr uint32_t B_X = B_W5 + 16 * 64 * 2;   // 2 x [128][32]: this tile's X and the next
constexpr uint32_t B_H1 = B_X + 2 * kTM * 32 * 2;  // [128][64]
constexpr uint32_t B_H2 = B_H1 + kTM * 64 * 2;     // [128][64], later dH1
constexpr uint32_t B_O = B_H2 + kTM * 64 * 2;      // [128][16]
constexpr uint32_t B_H4 = B_O + kTM * 16 * 2;      // [128][64], later dH2
constexpr uint32_t B_DZ = B_H4 + kTM * 64 * 2;     // [128][16], later dO
constexpr uint32_t B_DH4 = B_DZ + kTM * 16 * 2;    // [128][64]
constexpr uint32_t B_MISC = B_DH4 + kTM * 64 * 2;  // 5 mbarriers + TMEM base
constexpr uint32_t B_DO = B_DZ;
constexpr uint32_t B_DH2 = B_H4;
constexpr uint32_t B_DH1 = B_H2;
constexpr uint32_t kSmemB = B_MISC + 64;         // 106 KB: two CTAs per SM
static_assert(B_X == (uint32_t)kW16Bytes, "W1..W5 = the field's weight image");
static_assert(2 * (kSmemB + 1024) <= 228 * 1024, "two CTAs per SM");

struct TcBwdArgs {
  CUtensorMap xmap[2];      // TMA maps of the 16-bit feature tiles for in = 16, 32
  const void* feat;         // 16-bit operand tiles of the encoding features (feat16_offset)
  const float* dout;        // [4][ld]: dL/do_0, dL/dz_rgb
  float* dfeat;             // [in][ld]
  const int32_t* s_ray;     // padding marker (< 0) or null
  const uint32_t* mask;     // [6][ld] ReLU decisions of H1, H2, H4 from the training forward
  const int32_t* view_base;
  int view_lo, view_hi;     // the views whose tiles this launch takes (ranges are whole tiles)
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

// One thread: adjoint-chain MMA D (128 x N) = dY * W, with W the forward weight [K rows][N
// columns] (K-major in its own layout) read as an MN-major operand (column groups 128 B
// apart, row groups N*16 B apart) and dY in tensor memory: 8 columns per K step of 16.
__device__ __forceinline__ void issue_adjoint_ts(uint32_t d_tmem, uint32_t a_tmem, uint32_t w_saddr, int K, int N,
                                                 bool bf16) {
  const uint32_t idesc = tc::idesc_f16(kTM, N, bf16) | (1u << 16);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t bd = tc::smem_desc(w_saddr + kk * 32 * N, N * 16, 128);
    tc::mma_f16_ts(d_tmem, a_tmem + kk * 8, bd, idesc, kk > 0 ? 1u : 0u);
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
// kernel's MLP kind (uniform over the CTA), or n_tiles; v follows the view (cursor).
__device__ __forceinline__ int64_t next_tile(const TcBwdArgs& A, const int32_t* vb, int64_t tile, int64_t n_tiles,
                                             int kind, int& v) {
  for (; tile < n_tiles; tile += gridDim.x) {
    v = advance_view(vb, A.n_views, tile * kTM, v);
    if (A.f[v].mlp_kind == kind) return tile;
  }
  return n_tiles;
}

// The issuer warp (lane 0 works): tile `tile`'s X [128 x in] as one TMA box of its 16 row
// groups.
__device__ __forceinline__ void load_x(const TcBwdArgs& A, int64_t tile, int in, uint32_t dst, uint32_t bar) {
  if ((threadIdx.x & 31) == 0) {
    tc::mbar_expect_tx(bar, 16u * 16u * (uint32_t)in);
    tc::tma_load_3d(dst, &A.xmap[in == 32 ? 1 : 0], 0, (int)tile, 0, bar);
  }
  __syncwarp();
}

// This thread's raw dL/do_0, dL/dz_rgb, ReLU decisions and padding marker of tile `tile`
// (slot < S: view ranges are whole tiles).  No load depends on another, so all stay in
// flight under the chain; padding slots (marker < 0) are zeroed where the values are used.
__device__ __forceinline__ void load_dout(const TcBwdArgs& A, int64_t tile, int t, float (&d)[4], uint32_t (&m)[6],
                                          int& ray) {
  const int64_t s = tile * kTM + t;
  ray = A.s_ray ? A.s_ray[s] : 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = A.dout[(int64_t)i * A.ld + s];
#pragma unroll
  for (int i = 0; i < 6; ++i) m[i] = A.mask[(int64_t)i * A.ld + s];
}

// Epilogue thread: this thread's writes to MMA operands (shared memory) and reads of the
// accumulator (tensor memory) are done; count it in the issuer's "operands ready" barrier.
__device__ __forceinline__ void epi_arrive(uint32_t bar) {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsB, 2) k_mlp_bwd_tc(const __grid_constant__ TcBwdArgs A) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ int32_t vb[kMaxViews + 1];  // view sample bases
  if ((int64_t)A.view_base[A.n_views] > A.ld) return;  // overflow flagged by the scan
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t <= A.n_views) vb[t] = A.view_base[t];
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + B_MISC + 40);
  const uint32_t acc_bar = tc::smem_u32(sm + B_MISC);        // chain accumulator ready (commit)
  const uint32_t opr_bar = tc::smem_u32(sm + B_MISC + 8);    // operands ready (128 epilogue arrivals)
  const uint32_t x_bar = tc::smem_u32(sm + B_MISC + 16);     // X copies landed
  const uint32_t flush_bar = tc::smem_u32(sm + B_MISC + 24); // every MMA retired: dW may be read
  const uint32_t drain_bar = tc::smem_u32(sm + B_MISC + 32); // every MMA retired (exit)
  const uint32_t w_bar = tc::smem_u32(sm + B_MISC + 48);     // weight image landed
  const uint32_t sb = tc::smem_u32(sm);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemColsB);
  if (t == 0) {
    tc::mbar_init(acc_bar, 1);
    tc::mbar_init(opr_bar, kEpi);
    tc::mbar_init(x_bar, 1);
    tc::mbar_init(flush_bar, 1);
    tc::mbar_init(drain_bar, 1);
    tc::mbar_init(w_bar, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int kind = BF16 ? kMlpBF16 : kMlpF16;
  const int64_t S = (int64_t)vb[A.view_hi];
  const int64_t n_tiles = (S + kTM - 1) / kTM;
  const int64_t t_lo = (int64_t)vb[A.view_lo] / kTM;  // view ranges start on a tile boundary
  int v_first = A.view_lo;
  const int64_t first = next_tile(A, vb, t_lo + blockIdx.x, n_tiles, kind, v_first);
  bool ok = true;

  if (warp == 4) {
    // ================================================================ issuer warp
    uint32_t opr_ph = 0, acc_ph = 0, x_ph = 0, xbuf = 0;
    bool x_pending = false, dw_live = false;
    int cur = -1;
    int64_t tile = first;
    int vn = v_first;  // view of the next tile to process
    if (tile < n_tiles) {
      load_x(A, tile, A.f[vn].mlp_in, sb + B_X, x_bar);
      x_pending = true;
    }
    // wait for the epilogue's next "operands ready", then order the MMAs after it
#define INVR_OPR_WAIT()                                   \
  if (!(ok = tc::mbar_wait(opr_bar, opr_ph, A.wait_limit))) break; \
  opr_ph ^= 1u;                                           \
  tc::fence_after_sync();
    // commit the chain MMAs issued so far to the epilogue's barrier
#define INVR_ACC_COMMIT()                  \
  if (lane == 0) tc::commit_to(acc_bar);   \
  acc_ph ^= 1u;
    while (tile < n_tiles) {
      const int v = vn;
      const FieldDev& F = A.f[v];
      const int64_t nxt = next_tile(A, vb, tile + gridDim.x, n_tiles, kind, vn);
      if (cur >= 0 && F.weights != A.f[cur].weights && dw_live) {
        if (lane == 0) tc::commit_to(flush_bar);  // the epilogue reads the old field's dW out
        dw_live = false;
      }
      cur = v;
      const int in = F.mlp_in;
      const uint32_t bx = B_X + xbuf * (kTM * 32 * 2);
      // ---- S1 recompute H1 (needs: dZ rows, the previous tile's last TMEM read, weights)
      INVR_OPR_WAIT();
      if (!(ok = tc::mbar_wait(x_bar, x_ph, A.wait_limit))) break;
      x_ph ^= 1u;
      x_pending = false;
      if (lane == 0) issue_chain(tmem + C_CHAIN, sb + bx, sb + B_W1, in, 64, BF16);
      INVR_ACC_COMMIT();
      // once S1 retires, so have the previous tile's weight-gradient MMAs (they read the
      // other X buffer): the next tile's X may land there
      if (nxt < n_tiles) {
        if (!(ok = tc::mbar_wait(acc_bar, acc_ph ^ 1u, A.wait_limit))) break;
        load_x(A, nxt, A.f[vn].mlp_in, sb + B_X + (xbuf ^ 1u) * (kTM * 32 * 2), x_bar);
        x_pending = true;
      }
      // ---- S2 H2, S3 O, S4 H4
      INVR_OPR_WAIT();
      if (lane == 0) issue_chain_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W2, 64, 64, BF16);
      INVR_ACC_COMMIT();
      INVR_OPR_WAIT();
      if (lane == 0) issue_chain_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W3, 64, 16, BF16);
      INVR_ACC_COMMIT();
      INVR_OPR_WAIT();
      if (lane == 0) issue_chain_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W4, 16, 64, BF16);
      INVR_ACC_COMMIT();
      // ---- S5 dH4 = (dZ W5p) [H4 > 0];  dW5p^T += H4^T dZ
      INVR_OPR_WAIT();
      if (lane == 0) issue_adjoint_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W5, 16, 64, BF16);
      INVR_ACC_COMMIT();
      if (lane == 0) issue_dw(tmem + C_DW5T, sb + B_H4, 64, sb + B_DZ, 16, 16, dw_live, BF16);
      // ---- S6 dO = dH4 W4p  (dW4p += dH4^T O is issued after S9)
      INVR_OPR_WAIT();
      if (lane == 0) issue_adjoint_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W4, 64, 16, BF16);
      INVR_ACC_COMMIT();
      // ---- S7 dH2 = (dO W3) [H2 > 0];  dW3^T += H2^T dO
      INVR_OPR_WAIT();
      if (lane == 0) issue_adjoint_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W3, 16, 64, BF16);
      INVR_ACC_COMMIT();
      if (lane == 0) issue_dw(tmem + C_DW3T, sb + B_H2, 64, sb + B_DO, 16, 16, dw_live, BF16);
      // ---- S8 dH1 = (dH2 W2) [H1 > 0];  dW2 += dH2^T H1
      INVR_OPR_WAIT();
      if (lane == 0) issue_adjoint_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W2, 64, 64, BF16);
      INVR_ACC_COMMIT();
      if (lane == 0) issue_dw(tmem + C_DW2, sb + B_DH2, 64, sb + B_H1, 64, 64, dw_live, BF16);
      // ---- S9 dX = dH1 W1;  dW1 += dH1^T X
      INVR_OPR_WAIT();
      if (lane == 0) issue_adjoint_ts(tmem + C_CHAIN, tmem + C_AOP, sb + B_W1, 64, in, BF16);
      INVR_ACC_COMMIT();
      if (lane == 0) {
        issue_dw(tmem + C_DW1, sb + B_DH1, 64, sb + bx, in, in, dw_live, BF16);
        // dW4 reads dH4 and O, which stay untouched until the next tile's S3 and S5 epilogues;
        // issued here, under the dX epilogue, instead of after S6's short one
        issue_dw(tmem + C_DW4, sb + B_DH4, 64, sb + B_O, 16, 16, dw_live, BF16);
      }
      dw_live = true;
      __syncwarp();
      xbuf ^= 1u;
      tile = nxt;
    }
#undef INVR_OPR_WAIT
#undef INVR_ACC_COMMIT
    if (ok && dw_live && lane == 0) tc::commit_to(flush_bar);  // the last field's dW
    if (!ok && lane == 0) atomicOr(A.status, kStatusTimeout);
    // retire every MMA and copy of this CTA (bounded) before the tensor memory is freed
    if (lane == 0) tc::commit_to(drain_bar);
    if (!tc::mbar_wait(drain_bar, 0, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
    if (x_pending && !tc::mbar_wait(x_bar, x_ph, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
  } else {
    // ================================================================ epilogue warps
    const uint32_t row_t = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t acc_ph = 0, fl_ph = 0, w_ph = 0;
    bool dw_live = false, w_pending = false;
    int cur = -1;
    int64_t tile = first;
    int vn = v_first;  // view of the next tile to process
    float dnext[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t mnext[6] = {0u, 0u, 0u, 0u, 0u, 0u}, m[6];
    int ray_next = -1;
    if (tile < n_tiles) load_dout(A, tile, t, dnext, mnext, ray_next);
#define INVR_ACC_WAIT()                                   \
  if (!(ok = tc::mbar_wait(acc_bar, acc_ph, A.wait_limit))) break; \
  acc_ph ^= 1u;                                           \
  tc::fence_after_sync();
    while (tile < n_tiles) {
      const int64_t s0 = tile * kTM;
      const int v = vn;
      const FieldDev& F = A.f[v];
      const int64_t nxt = next_tile(A, vb, tile + gridDim.x, n_tiles, kind, vn);
      if (cur < 0 || F.weights != A.f[cur].weights) {
        if (dw_live) {
          if (!(ok = tc::mbar_wait(flush_bar, fl_ph, A.wait_limit))) break;
          fl_ph ^= 1u;
          tc::fence_after_sync();
          flush_dw(tmem, A.f[cur], A.out_scale);
          dw_live = false;
        }
        // the field's weight image by one bulk copy (every MMA has retired, or none was issued)
        if (t == 0) {
          tc::mbar_expect_tx(w_bar, (uint32_t)kW16Bytes);
          tc::bulk_g2s(sb + B_W1, F.w16, (uint32_t)kW16Bytes, w_bar);
        }
        w_pending = true;
        if (!(ok = tc::mbar_wait(w_bar, w_ph, A.wait_limit))) break;
        w_ph ^= 1u;
        w_pending = false;
        cur = v;
      }
      const int in = F.mlp_in;
      const int valid = (int)(S - s0 < kTM ? S - s0 : kTM);
      // ---- dZ row (dL/dz for rgb; zero for the padded outputs) and dL/do_0 of this tile
      const bool live = t < valid && ray_next >= 0;
      const float do0 = live ? dnext[0] * A.in_scale : 0.0f;
#pragma unroll
      for (int i = 0; i < 6; ++i) m[i] = mnext[i];
      float dz[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) dz[i] = (i < 3 && live) ? dnext[1 + i] * A.in_scale : 0.0f;
      row16_out<BF16, false>(dz, sm + B_DZ, t, 0u);
      epi_arrive(opr_bar);
      // ---- S1: H1
      INVR_ACC_WAIT();
      if (nxt < n_tiles) load_dout(A, nxt, t, dnext, mnext, ray_next);
      row64_relu<BF16, true>(row_t + C_CHAIN, sm + B_H1, t, row_t + C_AOP);
      epi_arrive(opr_bar);
      // ---- S2: H2
      INVR_ACC_WAIT();
      row64_relu<BF16, true>(row_t + C_CHAIN, sm + B_H2, t, row_t + C_AOP);
      epi_arrive(opr_bar);
      // ---- S3: O = (0, o_1..o_15)
      INVR_ACC_WAIT();
      {
        float o[16];
        tc::tmem_ld16(row_t + C_CHAIN, o);
        o[0] = 0.0f;
        row16_out<BF16, true>(o, sm + B_O, t, row_t + C_AOP);
      }
      epi_arrive(opr_bar);
      // ---- S4: H4
      INVR_ACC_WAIT();
      row64_relu<BF16, false>(row_t + C_CHAIN, sm + B_H4, t, 0u);
      {
        // the adjoint chain starts from dZ: S5's A operand
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) w[c] = tc::pack2<BF16>(dz[2 * c], dz[2 * c + 1]);
        tc::tmem_st8(row_t + C_AOP, w);
      }
      epi_arrive(opr_bar);
      // ---- S5: dH4
      INVR_ACC_WAIT();
      row64_masked<BF16, true>(row_t + C_CHAIN, sm + B_DH4, m[4], m[5], t, row_t + C_AOP);
      epi_arrive(opr_bar);
      // ---- S6: dO (o_0 slot carries dL/do_0), over dZ
      INVR_ACC_WAIT();
      {
        float d[16];
        tc::tmem_ld16(row_t + C_CHAIN, d);
        d[0] = do0;
        row16_out<BF16, true>(d, sm + B_DO, t, row_t + C_AOP);
      }
      epi_arrive(opr_bar);
      // ---- S7: dH2, over H4
      INVR_ACC_WAIT();
      row64_masked<BF16, true>(row_t + C_CHAIN, sm + B_DH2, m[2], m[3], t, row_t + C_AOP);
      epi_arrive(opr_bar);
      // ---- S8: dH1, over H2
      INVR_ACC_WAIT();
      row64_masked<BF16, true>(row_t + C_CHAIN, sm + B_DH1, m[0], m[1], t, row_t + C_AOP);
      epi_arrive(opr_bar);
      // ---- S9: dX -> dL/dfeat (its TMEM read is covered by the next tile's first arrival)
      INVR_ACC_WAIT();
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
      dw_live = true;
      tile = nxt;
    }
#undef INVR_ACC_WAIT
    if (ok && dw_live) {
      ok = tc::mbar_wait(flush_bar, fl_ph, A.wait_limit);
      tc::fence_after_sync();
      if (ok) flush_dw(tmem, A.f[cur], A.out_scale);
    }
    if (!ok) atomicOr(A.status, kStatusTimeout);
    // a weight copy still in flight must land before the shared memory is released
    if (w_pending && !tc::mbar_wait(w_bar, w_ph, kWaitLimit)) atomicOr(A.status, kStatusDrainTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemColsB);
  }
}

}  // namespace

// The tiles of views [P.view_lo, P.view_hi).
cudaError_t launch_mlp_bwd_tc(const Plan& P, int num_sms, cudaStream_t s) {
  TcBwdArgs A{};
  A.view_lo = P.view_lo;
  A.view_hi = P.view_hi;
  A.feat = P.ws.feat;
  A.dout = P.ws.dout;
  A.dfeat = P.ws.dfeat;
  A.s_ray = P.ws.s_ray;
  A.mask = P.ws.mlp_mask;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n_views = P.n_views;
  // dL/dout carries the loss's 1 / (3 R); take it out of the 16-bit operands
  A.in_scale = P.grad_scale / P.loss_norm;
  A.out_scale = P.loss_norm;
  A.wait_limit = P.wait_limit;
  A.status = P.status;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  if (!encode_feat16_map(&A.xmap[0], P.ws.feat, P.ws.S_cap, 16) ||
      !encode_feat16_map(&A.xmap[1], P.ws.feat, P.ws.S_cap, 32))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;  // the weight images its training forward wrote (same weights)
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
