// Geometry + colour MLPs in FP32 (the plain-precision path; Sec. 4.2 "geometry MLP E_g
// and color MLP E_c").  Shapes: in (16|32) -> 64 -> 64 -> 16 (ReLU hidden, no biases),
// sigma = exp(o_0); o_1..o_15 -> 64 (ReLU) -> 3, sigmoid.
//
// Persistent CTAs of 256 threads walk 128-sample tiles.  A tile's activations live in
// shared memory as [units][128 samples] (row stride 132 floats: rows stay 16-byte aligned);
// each layer is a small SIMT GEMM in which a thread owns (rows/16) x 8 outputs: two runs
// of 4 samples, read as two float4 per input row, so a 64-row layer does 32 FMAs per three
// 16-byte shared loads.  The colour layers are padded to 16-wide (W4 gets a zero
// column for o_0, W5 gets 13 zero rows) so every dimension is a multiple of 16.
//
// Backward (per tile): the forward activations are recomputed from the stored encoding
// features, then deltas flow back layer by layer (in place over the activations), and the
// weight gradients dW = sum_s delta_s a_s^T are accumulated in registers across all tiles
// a CTA visits, flushed once per field with atomics.
//
// Bound: FP32 FMA pipe (9216 padded multiply-adds per sample forward, ~3x backward).
#include "invr_internal.cuh"

namespace invr {

namespace {

constexpr int kTS = 128;   // samples per tile
constexpr int kLD = 132;   // activation row stride (floats; a multiple of 4)
constexpr int kThreads = 256;

struct MlpArgs {
  const float* feat;        // [IN][ld]
  float* out;               // [4][ld]
  const float* dout;        // [4][ld]: dL/do_0, dL/dz_rgb
  float* dfeat;             // [IN][ld]
  const int32_t* s_ray;     // padding marker (< 0) or null
  const int32_t* view_base; // per-view tile-aligned sample ranges (device) or null
  int64_t ld;
  int64_t n;                // samples when view_base is null
  int n_views;
  float grad_scale;
  FieldDev f[kMaxViews];
};

// Shared-memory plan (floats).
constexpr int kW1 = 0;                   // [IN][64]  (transposed)
constexpr int kW2 = kW1 + 32 * 64;       // [64][64]
constexpr int kW3 = kW2 + 64 * 64;       // [64][16]
constexpr int kW4 = kW3 + 64 * 16;       // [16][64]
constexpr int kW5 = kW4 + 16 * 64;       // [64][16]
constexpr int kWSize = kW5 + 64 * 16;    // 9216

struct WeightOffsets {
  int w1, w2, w3, w4, w5;
  __device__ WeightOffsets(int in) {
    w1 = 0;
    w2 = w1 + kHidden * in;
    w3 = w2 + kHidden * kHidden;
    w4 = w3 + kGeoOut * kHidden;
    w5 = w4 + kColHidden * (kGeoOut - 1);
  }
};

// Padded weight element [o][k] of layer `layer` (1-based) from the flat W1..W5 array.
__device__ __forceinline__ float padded_w(const float* W, const WeightOffsets& off, int in, int layer, int o, int k) {
  switch (layer) {
    case 1: return W[off.w1 + o * in + k];
    case 2: return W[off.w2 + o * kHidden + k];
    case 3: return W[off.w3 + o * kHidden + k];
    case 4: return k == 0 ? 0.0f : W[off.w4 + o * (kGeoOut - 1) + (k - 1)];
    default: return o < 3 ? W[off.w5 + o * kColHidden + k] : 0.0f;
  }
}

// Load the five (padded) layers: transposed copies [k][o] into Wt; if Wn is non-null also
// the [o][k] copies.
__device__ void load_weights(const float* __restrict__ W, int in, float* Wt, float* Wn) {
  const WeightOffsets off(in);
  const int outs[5] = {64, 64, 16, 64, 16};
  const int ins[5] = {in, 64, 64, 16, 64};
  const int base[5] = {kW1, kW2, kW3, kW4, kW5};
  for (int layer = 0; layer < 5; ++layer) {
    const int O = outs[layer], I = ins[layer];
    for (int e = threadIdx.x; e < O * I; e += blockDim.x) {
      const int o = e / I, k = e % I;
      const float w = padded_w(W, off, in, layer + 1, o, k);
      Wt[base[layer] + k * O + o] = w;
      if (Wn) Wn[base[layer] + o * I + k] = w;
    }
  }
}

// R consecutive floats of a shared-memory row (R = 1, 2 or 4; 4 R-byte aligned).
template <int R>
__device__ __forceinline__ void load_r(const float* p, float (&w)[R]) {
  if constexpr (R == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
  } else if constexpr (R == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    w[0] = q.x; w[1] = q.y;
  } else {
    w[0] = *p;
  }
}

// R consecutive floats of a global-memory row through the read-only path (same alignment).
template <int R>
__device__ __forceinline__ void ldg_r(const float* p, float (&w)[R]) {
  if constexpr (R == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
  } else if constexpr (R == 2) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    w[0] = q.x; w[1] = q.y;
  } else {
    w[0] = __ldg(p);
  }
}

// A thread's 8 samples of a tile: 4 sg .. 4 sg + 3 and 64 + 4 sg .. 64 + 4 sg + 3, so that
// the 16 sample groups of a warp read 256 contiguous bytes per float4 (no bank conflicts).
__device__ __forceinline__ int sample_of(int sg, int c) { return (c < 4 ? 4 * sg : 64 + 4 * sg) + (c & 3); }

__device__ __forceinline__ void load8(const float* row, int sg, float (&x)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(row + 4 * sg);
  const float4 b = *reinterpret_cast<const float4*>(row + 64 + 4 * sg);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

__device__ __forceinline__ void store8(float* row, int sg, const float (&v)[8]) {
  *reinterpret_cast<float4*>(row + 4 * sg) = make_float4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<float4*>(row + 64 + 4 * sg) = make_float4(v[4], v[5], v[6], v[7]);
}

// Y[o][s] = act(sum_k Wt[k][o] X[k][s]); thread owns rows og*R..og*R+R-1 and the 8 samples
// sample_of(sg, 0..7).
// 16-row layers: thread owns rows 4 og .. 4 og + 3 (og = t / 64, uniform per warp) and the
// samples 2 sg, 2 sg + 1 (sg = t % 64): one float2 of X and one float4 of W per input row
// for 8 FMAs, where the (rows/16) x 8 mapping would read 8 samples for one row.
template <int IN, bool RELU, bool GW>
__device__ __forceinline__ void layer_fwd16(const float* __restrict__ Wt, const float* __restrict__ X, float* Y) {
  const int og = threadIdx.x >> 6, sg = threadIdx.x & 63;
  float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
  for (int k = 0; k < IN; ++k) {
    const float2 x = *reinterpret_cast<const float2*>(X + k * kLD + 2 * sg);
    float w[4];
    if constexpr (GW)
      ldg_r<4>(Wt + k * 16 + og * 4, w);
    else
      load_r<4>(Wt + k * 16 + og * 4, w);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a][0] = fmaf(w[a], x.x, acc[a][0]);
      acc[a][1] = fmaf(w[a], x.y, acc[a][1]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
    *reinterpret_cast<float2*>(Y + (og * 4 + a) * kLD + 2 * sg) =
        RELU ? make_float2(fmaxf(acc[a][0], 0.0f), fmaxf(acc[a][1], 0.0f)) : make_float2(acc[a][0], acc[a][1]);
}

// Wt in shared memory, or in global memory (GW; L1-resident: every warp reads the same rows).
template <int OUT, int IN, bool RELU, bool GW = false>
__device__ __forceinline__ void layer_fwd(const float* __restrict__ Wt, const float* __restrict__ X, float* Y) {
  if constexpr (OUT == 16) {
    layer_fwd16<IN, RELU, GW>(Wt, X, Y);
    return;
  }
  constexpr int R = OUT / 16;
  const int og = threadIdx.x >> 4, sg = threadIdx.x & 15;
  float acc[R][8];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < IN; ++k) {
    float x[8], w[R];
    load8(X + k * kLD, sg, x);
    if constexpr (GW)
      ldg_r<R>(Wt + k * OUT + og * R, w);
    else
      load_r<R>(Wt + k * OUT + og * R, w);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(w[a], x[c], acc[a][c]);
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = RELU ? fmaxf(acc[a][c], 0.0f) : acc[a][c];
    store8(Y + (og * R + a) * kLD, sg, v);
  }
}

// dX[k][s] = (sum_o W[o][k] dY[o][s]) masked by (M[k][s] > 0); W in [OUT][IN] layout.
// Output to shared memory (stride kLD) or, if G != null, to global G[k*ld + s] (s < valid).
// dX may be M itself: each element's mask is read by the thread that then writes it.
// 16-row outputs (IN = 16, no mask) with the mapping of layer_fwd16: rows 4 kg .. 4 kg + 3,
// samples 2 sg, 2 sg + 1.
template <int OUT>
__device__ __forceinline__ void layer_bwd_in16(const float* __restrict__ Wn, const float* __restrict__ dY, float* dX,
                                               float* G, int64_t ld, int valid) {
  const int kg = threadIdx.x >> 6, sg = threadIdx.x & 63;
  float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
  for (int o = 0; o < OUT; ++o) {
    const float2 y = *reinterpret_cast<const float2*>(dY + o * kLD + 2 * sg);
    float w[4];
    load_r<4>(Wn + o * 16 + kg * 4, w);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a][0] = fmaf(w[a], y.x, acc[a][0]);
      acc[a][1] = fmaf(w[a], y.y, acc[a][1]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = kg * 4 + a, s = 2 * sg;
    if (G) {
      float* g = G + (int64_t)k * ld + s;
      if (s < valid) g[0] = acc[a][0];
      if (s + 1 < valid) g[1] = acc[a][1];
    } else {
      *reinterpret_cast<float2*>(dX + k * kLD + s) = make_float2(acc[a][0], acc[a][1]);
    }
  }
}

template <int OUT, int IN, bool MASK>
__device__ __forceinline__ void layer_bwd_in(const float* __restrict__ Wn, const float* __restrict__ dY, float* dX,
                                             const float* M, float* G, int64_t ld, int valid) {
  if constexpr (IN == 16 && !MASK) {
    layer_bwd_in16<OUT>(Wn, dY, dX, G, ld, valid);
    return;
  }
  constexpr int R = IN / 16;
  const int kg = threadIdx.x >> 4, sg = threadIdx.x & 15;
  float acc[R][8];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
#pragma unroll 4
  for (int o = 0; o < OUT; ++o) {
    float y[8], w[R];
    load8(dY + o * kLD, sg, y);
    load_r<R>(Wn + o * IN + kg * R, w);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(w[a], y[c], acc[a][c]);
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const int k = kg * R + a;
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = acc[a][c];
    if (MASK) {
      float m[8];
      load8(M + k * kLD, sg, m);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (!(m[c] > 0.0f)) v[c] = 0.0f;
    }
    if (G) {
      // G + k ld is 16-byte aligned: ld and the tile start are multiples of 128 samples
      float* g = G + (int64_t)k * ld;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int s = sample_of(sg, 4 * h);
        if (s + 4 <= valid) {
          *reinterpret_cast<float4*>(g + s) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (s + c < valid) g[s + c] = v[4 * h + c];
        }
      }
    } else {
      store8(dX + k * kLD, sg, v);
    }
  }
}

// acc[i][j] += sum_s dY[i][s] X[j][s]; thread owns rows ig*RI+a, columns jg+16c; the
// samples in order, 4 per step (one float4 per row).
template <int OUT, int IN>
__device__ __forceinline__ void acc_dw(const float* __restrict__ dY, const float* __restrict__ X, float* acc) {
  constexpr int RI = OUT / 16, CJ = IN / 16;
  const int ig = threadIdx.x >> 4, jg = threadIdx.x & 15;
#pragma unroll 2
  for (int s = 0; s < kTS; s += 4) {
    float4 y[RI], x[CJ];
#pragma unroll
    for (int a = 0; a < RI; ++a) y[a] = *reinterpret_cast<const float4*>(dY + (ig * RI + a) * kLD + s);
#pragma unroll
    for (int c = 0; c < CJ; ++c) x[c] = *reinterpret_cast<const float4*>(X + (jg + 16 * c) * kLD + s);
#pragma unroll
    for (int a = 0; a < RI; ++a)
#pragma unroll
      for (int c = 0; c < CJ; ++c) {
        float t = acc[a * CJ + c];
        t = fmaf(y[a].x, x[c].x, t);
        t = fmaf(y[a].y, x[c].y, t);
        t = fmaf(y[a].z, x[c].z, t);
        t = fmaf(y[a].w, x[c].w, t);
        acc[a * CJ + c] = t;
      }
  }
}

template <int OUT, int IN>
__device__ __forceinline__ void flush_dw(float* acc, float* G, const WeightOffsets& off, int in, int layer) {
  constexpr int RI = OUT / 16, CJ = IN / 16;
  const int ig = threadIdx.x >> 4, jg = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < RI; ++a)
#pragma unroll
    for (int c = 0; c < CJ; ++c) {
      const int i = ig * RI + a, j = jg + 16 * c;
      const float v = acc[a * CJ + c];
      acc[a * CJ + c] = 0.0f;
      int idx = -1;
      switch (layer) {
        case 1: idx = off.w1 + i * in + j; break;
        case 2: idx = off.w2 + i * kHidden + j; break;
        case 3: idx = off.w3 + i * kHidden + j; break;
        case 4: idx = j == 0 ? -1 : off.w4 + i * (kGeoOut - 1) + (j - 1); break;
        default: idx = i < 3 ? off.w5 + i * kColHidden + j : -1; break;
      }
      if (idx >= 0 && v != 0.0f) atomicAdd(G + idx, v);
    }
}

__device__ __forceinline__ void tile_range(const MlpArgs& A, int64_t& n_tiles) {
  const int64_t S = A.view_base ? (int64_t)A.view_base[A.n_views] : A.n;
  // a sample list longer than the workspace (flagged by the scan) is not processed
  n_tiles = (A.view_base && S > A.ld) ? 0 : (S + kTS - 1) / kTS;
}

__device__ __forceinline__ int tile_view(const MlpArgs& A, int64_t s0) {
  return A.view_base ? view_of_slot(A.view_base, A.n_views, s0) : 0;
}

__device__ __forceinline__ int tile_valid(const MlpArgs& A, int64_t s0) {
  const int64_t S = A.view_base ? (int64_t)A.view_base[A.n_views] : A.n;
  const int64_t rem = S - s0;
  return rem < kTS ? (int)rem : kTS;
}

// 4-byte asynchronous copy global -> shared (zero-filled when !valid; src is then not read).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most `pending` (0 or 1) of this thread's copy groups are in flight.
__device__ __forceinline__ void cp_async_wait(int pending) {
  if (pending) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// The tile's inputs, staged asynchronously (one copy group per tile, issued a tile ahead):
// X [in][kTS] (zero past `valid`) and, for the backward, dL/d(outputs) [4][kTS] and the
// padding markers [kTS].
__device__ void stage_inputs(const MlpArgs& A, int64_t s0, int in, float* X, float* Dp, int32_t* Rp) {
  const int valid = tile_valid(A, s0);
  for (int e = threadIdx.x; e < in * kTS; e += kThreads) {
    const int k = e / kTS, s = e % kTS;
    cp_async4(X + k * kLD + s, s < valid ? A.feat + (int64_t)k * A.ld + s0 + s : A.feat, s < valid);
  }
  if (Dp) {
    for (int e = threadIdx.x; e < 4 * kTS; e += kThreads) {
      const int i = e / kTS, s = e % kTS;
      cp_async4(Dp + i * kTS + s, s < valid ? A.dout + (int64_t)i * A.ld + s0 + s : A.dout, s < valid);
    }
    if (A.s_ray)
      for (int s = threadIdx.x; s < kTS; s += kThreads)
        cp_async4(Rp + s, s < valid ? A.s_ray + s0 + s : A.s_ray, s < valid);
  }
  cp_async_commit();
}

// The next tile of this CTA from `t` on (steps of gridDim.x) whose field runs in FP32.
__device__ __forceinline__ int64_t next_f32_tile(const MlpArgs& A, int64_t t, int64_t n_tiles) {
  for (; t < n_tiles; t += gridDim.x)
    if (A.f[tile_view(A, t * kTS)].mlp_kind == kMlpF32) return t;
  return n_tiles;
}

// X staged (and visible to every thread) on entry; Wt (global) the field's transposed
// weights.  Once layer 1 has read X, its buffer holds O (rows 0..15) and Z (rows 16..31).
template <int IN>
__device__ __forceinline__ void tile_forward(const MlpArgs& A, int64_t s0, int valid, const float* Wt, float* X,
                                             float* H1, float* H2) {
  float* O = X;
  float* Z = X + 16 * kLD;
  layer_fwd<64, IN, true, true>(Wt + kW1, X, H1);
  __syncthreads();
  layer_fwd<64, 64, true, true>(Wt + kW2, H1, H2);
  __syncthreads();
  layer_fwd<16, 64, false, true>(Wt + kW3, H2, O);
  __syncthreads();
  layer_fwd<64, 16, true, true>(Wt + kW4, O, H1);  // H4 reuses H1
  __syncthreads();
  layer_fwd<16, 64, false, true>(Wt + kW5, H1, Z);
  __syncthreads();
  if (threadIdx.x < kTS && (int)threadIdx.x < valid) {
    const int s = threadIdx.x;
    const int64_t gs = s0 + s;
    A.out[gs] = expf(O[s]);
    for (int c = 0; c < 3; ++c) A.out[(int64_t)(1 + c) * A.ld + gs] = 1.0f / (1.0f + expf(-Z[c * kLD + s]));
  }
  __syncthreads();
}

// Two CTAs per SM (99 KB of shared memory each): the weights are read from the field's
// transposed copy in global memory (L1-resident) instead of being staged per CTA.
__global__ void __launch_bounds__(kThreads, 2) k_mlp_fwd_f32(const __grid_constant__ MlpArgs A) {
  extern __shared__ float sm[];
  float* const X0 = sm;  // double-buffered inputs X0, X1
  float* const X1 = X0 + 32 * kLD;
  float* H1 = X1 + 32 * kLD;
  float* H2 = H1 + 64 * kLD;
  int64_t n_tiles;
  tile_range(A, n_tiles);
  int64_t t = next_f32_tile(A, blockIdx.x, n_tiles);
  if (t < n_tiles) stage_inputs(A, t * kTS, A.f[tile_view(A, t * kTS)].mlp_in, X0, nullptr, nullptr);
  for (int buf = 0; t < n_tiles; buf ^= 1) {
    const int64_t s0 = t * kTS;
    const FieldDev& F = A.f[tile_view(A, s0)];
    const int64_t tn = next_f32_tile(A, t + gridDim.x, n_tiles);
    float* const X = buf ? X1 : X0;
    // the other buffer was last read by the previous tile, which ended with a barrier
    if (tn < n_tiles) stage_inputs(A, tn * kTS, A.f[tile_view(A, tn * kTS)].mlp_in, buf ? X0 : X1, nullptr, nullptr);
    cp_async_wait(tn < n_tiles ? 1 : 0);
    __syncthreads();
    const int valid = tile_valid(A, s0);
    if (F.mlp_in == 16)
      tile_forward<16>(A, s0, valid, F.wt_f32, X, H1, H2);
    else
      tile_forward<32>(A, s0, valid, F.wt_f32, X, H1, H2);
    t = tn;
  }
}

// The padded, transposed weights of a field into its global copy Wt: one thread per element
// of the [k][o] layout (layer 1 with in = 16 leaves its rows 16..31 unused).
__global__ void __launch_bounds__(256) k_prep_wt(const float* __restrict__ W, int in, float* Wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kWSize) return;
  const WeightOffsets off(in);
  const int base[5] = {kW1, kW2, kW3, kW4, kW5}, outs[5] = {64, 64, 16, 64, 16}, ins[5] = {in, 64, 64, 16, 64};
  int layer = 4;
  while (layer > 0 && e < base[layer]) --layer;
  const int i = e - base[layer], k = i / outs[layer], o = i % outs[layer];
  if (k < ins[layer]) Wt[e] = padded_w(W, off, in, layer + 1, o, k);
}

// X, Dp (dL/d(outputs)) and Rp (padding markers) staged and visible on entry.
template <int IN>
__device__ __forceinline__ void tile_backward(const MlpArgs& A, int64_t s0, int valid, const float* Wt, const float* Wn, float* X,
                              const float* Dp, const int32_t* Rp, float* H1, float* H2, float* H4, float* O, float* D,
                              float* acc1, float* acc2, float* acc3, float* acc4, float* acc5) {
  layer_fwd<64, IN, true>(Wt + kW1, X, H1);
  __syncthreads();
  layer_fwd<64, 64, true>(Wt + kW2, H1, H2);
  __syncthreads();
  layer_fwd<16, 64, false>(Wt + kW3, H2, O);
  __syncthreads();
  layer_fwd<64, 16, true>(Wt + kW4, O, H4);
  // dZ (rows 0..2 from dL/dz_rgb, rows 3..15 zero) into D
  for (int e = threadIdx.x; e < 16 * kTS; e += blockDim.x) {
    const int i = e / kTS, s = e % kTS;
    float v = 0.0f;
    if (i < 3 && s < valid && (!A.s_ray || Rp[s] >= 0)) v = Dp[(1 + i) * kTS + s] * A.grad_scale;
    D[i * kLD + s] = v;
  }
  __syncthreads();
  acc_dw<16, 64>(D, H4, acc5);
  __syncthreads();
  layer_bwd_in<16, 64, true>(Wn + kW5, D, H4, H4, nullptr, 0, kTS);  // dH4 in place
  __syncthreads();
  acc_dw<64, 16>(H4, O, acc4);
  __syncthreads();
  layer_bwd_in<64, 16, false>(Wn + kW4, H4, D, nullptr, nullptr, 0, kTS);  // dO into D
  __syncthreads();
  for (int s = threadIdx.x; s < kTS; s += blockDim.x) {
    float v = 0.0f;
    if (s < valid && (!A.s_ray || Rp[s] >= 0)) v = Dp[s] * A.grad_scale;
    D[s] = v;  // row 0: dL/do_0 (the colour MLP does not read o_0)
  }
  __syncthreads();
  acc_dw<16, 64>(D, H2, acc3);
  __syncthreads();
  layer_bwd_in<16, 64, true>(Wn + kW3, D, H2, H2, nullptr, 0, kTS);  // dH2 in place
  __syncthreads();
  acc_dw<64, 64>(H2, H1, acc2);
  __syncthreads();
  layer_bwd_in<64, 64, true>(Wn + kW2, H2, H1, H1, nullptr, 0, kTS);  // dH1 in place
  __syncthreads();
  acc_dw<64, IN>(H1, X, acc1);
  layer_bwd_in<64, IN, false>(Wn + kW1, H1, nullptr, nullptr, A.dfeat + s0, A.ld, valid);
  __syncthreads();
}

__device__ __forceinline__ void flush_all(float* acc1, float* acc2, float* acc3, float* acc4, float* acc5, const FieldDev& F) {
  const WeightOffsets off(F.mlp_in);
  if (F.mlp_in == 16)
    flush_dw<64, 16>(acc1, F.grad_weights, off, 16, 1);
  else
    flush_dw<64, 32>(acc1, F.grad_weights, off, 32, 1);
  flush_dw<64, 64>(acc2, F.grad_weights, off, F.mlp_in, 2);
  flush_dw<16, 64>(acc3, F.grad_weights, off, F.mlp_in, 3);
  flush_dw<64, 16>(acc4, F.grad_weights, off, F.mlp_in, 4);
  flush_dw<16, 64>(acc5, F.grad_weights, off, F.mlp_in, 5);
}

__global__ void __launch_bounds__(kThreads) k_mlp_bwd_f32(const __grid_constant__ MlpArgs A) {
  extern __shared__ float sm[];
  float* Wt = sm;
  float* Wn = Wt + kWSize;
  float* const X0 = Wn + kWSize;  // double-buffered inputs: X, dL/d(outputs), padding markers
  float* const X1 = X0 + 32 * kLD;
  float* H1 = X1 + 32 * kLD;
  float* H2 = H1 + 64 * kLD;
  float* H4 = H2 + 64 * kLD;
  float* O = H4 + 64 * kLD;
  float* D = O + 16 * kLD;
  float* const D0 = D + 16 * kLD;
  float* const D1 = D0 + 4 * kTS;
  int32_t* const R0 = reinterpret_cast<int32_t*>(D1 + 4 * kTS);
  int32_t* const R1 = R0 + kTS;
  float acc1[8], acc2[16], acc3[4], acc4[4], acc5[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc1[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) acc2[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) acc3[i] = acc4[i] = acc5[i] = 0.0f;
  int64_t n_tiles;
  tile_range(A, n_tiles);
  int cur = -1;
  int64_t t = next_f32_tile(A, blockIdx.x, n_tiles);
  if (t < n_tiles) stage_inputs(A, t * kTS, A.f[tile_view(A, t * kTS)].mlp_in, X0, D0, R0);
  for (int buf = 0; t < n_tiles; buf ^= 1) {
    const int64_t s0 = t * kTS;
    const int v = tile_view(A, s0);
    const FieldDev& F = A.f[v];
    const int64_t tn = next_f32_tile(A, t + gridDim.x, n_tiles);
    float* const X = buf ? X1 : X0;
    const float* const Dp = buf ? D1 : D0;
    const int32_t* const Rp = buf ? R1 : R0;
    // the other buffers were last read by the previous tile, which ended with a barrier
    if (tn < n_tiles)
      stage_inputs(A, tn * kTS, A.f[tile_view(A, tn * kTS)].mlp_in, buf ? X0 : X1, buf ? D0 : D1, buf ? R0 : R1);
    if (cur < 0 || F.weights != A.f[cur].weights) {
      if (cur >= 0) flush_all(acc1, acc2, acc3, acc4, acc5, A.f[cur]);
      __syncthreads();
      load_weights(F.weights, F.mlp_in, Wt, Wn);
      cur = v;
    }
    cp_async_wait(tn < n_tiles ? 1 : 0);
    __syncthreads();
    const int valid = tile_valid(A, s0);
    if (F.mlp_in == 16)
      tile_backward<16>(A, s0, valid, Wt, Wn, X, Dp, Rp, H1, H2, H4, O, D, acc1, acc2, acc3, acc4, acc5);
    else
      tile_backward<32>(A, s0, valid, Wt, Wn, X, Dp, Rp, H1, H2, H4, O, D, acc1, acc2, acc3, acc4, acc5);
    t = tn;
  }
  if (cur >= 0) flush_all(acc1, acc2, acc3, acc4, acc5, A.f[cur]);
}

static_assert(kWSize == kWtF32, "size of the transposed weight copy");
constexpr size_t kFwdSmem = (size_t)(2 * 32 * kLD + 64 * kLD * 2) * sizeof(float);
static_assert(2 * (kFwdSmem + 1024) <= 228 * 1024, "two forward CTAs per SM");
constexpr size_t kBwdSmem =
    (size_t)(2 * kWSize + 2 * 32 * kLD + 64 * kLD * 3 + 16 * kLD * 2 + 2 * 4 * kTS + 2 * kTS) * sizeof(float);
static_assert(kBwdSmem <= 227 * 1024, "backward fits one CTA per SM");

MlpArgs plan_args(const Plan& P) {
  MlpArgs A{};
  A.feat = static_cast<const float*>(P.ws.feat);
  A.out = P.ws.out;
  A.dout = P.ws.dout;
  A.dfeat = P.ws.dfeat;
  A.s_ray = P.ws.s_ray;
  A.view_base = P.ws.view_base;
  A.ld = P.ws.S_cap;
  A.n = 0;
  A.n_views = P.n_views;
  A.grad_scale = P.grad_scale;
  for (int v = 0; v < P.n_views; ++v) A.f[v] = P.v[v].field;
  return A;
}

}  // namespace

// Persistent grids: two forward CTAs per SM, one backward CTA (221 KB of shared memory).
// Each FP32 field's transposed weight copy is rewritten before its forward (the weights
// change with every optimiser step).
cudaError_t launch_mlp_fwd_f32(const Plan& P, int num_sms, cudaStream_t s) {
  for (int v = 0; v < P.n_views; ++v) {
    const FieldDev& F = P.v[v].field;
    bool seen = false;
    for (int u = 0; u < v; ++u) seen = seen || P.v[u].field.weights == F.weights;
    if (F.mlp_kind == kMlpF32 && !seen) k_prep_wt<<<ceil_div(kWSize, 256), 256, 0, s>>>(F.weights, F.mlp_in, F.wt_f32);
  }
  cudaFuncSetAttribute(k_mlp_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  k_mlp_fwd_f32<<<num_sms * 2, kThreads, kFwdSmem, s>>>(plan_args(P));
  return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_f32(const Plan& P, int num_sms, cudaStream_t s) {
  cudaFuncSetAttribute(k_mlp_bwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
  k_mlp_bwd_f32<<<num_sms, kThreads, kBwdSmem, s>>>(plan_args(P));
  return cudaGetLastError();
}

cudaError_t launch_mlp_points_f32(const FieldDev& f, int64_t n, const float* feat, float* out, int num_sms,
                                  cudaStream_t s) {
  MlpArgs A{};
  A.feat = feat;
  A.out = out;
  A.ld = n;
  A.n = n;
  A.n_views = 1;
  A.grad_scale = 1.0f;
  A.f[0] = f;
  cudaFuncSetAttribute(k_mlp_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  if (n > 0) {
    k_prep_wt<<<ceil_div(kWSize, 256), 256, 0, s>>>(f.weights, f.mlp_in, f.wt_f32);
    k_mlp_fwd_f32<<<num_sms * 2, kThreads, kFwdSmem, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t preload_mlp_points_f32() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  return e != cudaSuccess ? e : cudaFuncGetAttributes(&a, k_prep_wt);
}

}  // namespace invr
