// Pose-conditioned deformation net of the human field (Sec. 4.2, after Eq. 4; sizes of
// Sec. 4.4), FP32 SIMT path.
//
//   v_t = DQB^{-1}(v) v (k_warp),  f = H^d(v_t) (k_encode on the net's own tables),
//   h_1 = ReLU(W_1 [f; theta]),  h_k = ReLU(W_k h_{k-1}) (k = 2..n),  delta v = W_out h_n,
//   v_c = v_t + delta v  (then the field's own encoding reads v_c).
//
// The pose part of the first layer is the same for every sample of a view, so it is folded
// into a per-view bias W_1[:, n_feat:] theta (k_deform_bias) and the first layer's K drops
// from n_feat + pose_dim to n_feat.
//
// Backward: dL/dv_c comes from the field's encoding (k_encode_dx: for every level and
// corner, the derivative of the trilinear weight in the point times the corner's
// features, N_l / 2 per unit of x); dL/d(delta v) = dL/dv_c.  k_deform_bwd recomputes the
// forward activations of a 32-sample tile in shared memory, propagates the deltas down the
// layers (ReLU masks from the recomputed activations), writes dL/df for the table scatter
// (k_encode_bwd on the net's tables) and accumulates the weight gradients of its tiles in a
// per-CTA partial buffer, summed once per call (k_deform_reduce).
//
// Bound: FP32 FMA pipe, ~2 x (n_feat H + (n-1) H^2 + 3 H) FLOP per sample forward (110 k at
// 32 / 4 x 128), ~3x that backward, plus per tile the staging of every layer's weights
// from L2 (forward 4 B x n_w per 64 samples; backward twice per 32 samples) and the
// read-modify-write of the CTA's weight-gradient partials (8 B x n_w per 32 samples).
#include "invr_internal.cuh"

namespace invr {

namespace {

constexpr int kThreads = 256;
constexpr int kFwdTS = 64, kFwdLD = 65;   // forward tile: samples, activation row stride
constexpr int kBwdTS = 32, kBwdLD = 33;   // backward tile

__device__ __forceinline__ int view_of_slot(const Plan& P, int64_t s) {
  int v = 0;
  while (v + 1 < P.n_views && s >= P.ws.view_base[v + 1]) ++v;
  return v;
}

__device__ __forceinline__ int64_t layer_offset(const DeformDev& D, int layer) {  // 0-based; n = output
  const int64_t n_in = D.n_feat + D.pose_dim;
  if (layer == 0) return 0;
  return (int64_t)D.hidden * n_in + (int64_t)(layer - 1) * D.hidden * D.hidden;
}

// A[k][n] = W[n][k0 + k] for n < N, k < K (transposed stage: out = W x); reads run along
// the rows of W.
__device__ __forceinline__ void stage_t(const float* __restrict__ W, int N, int K, int ldw, int k0, float* A) {
  for (int e = threadIdx.x; e < N * K; e += kThreads) {
    const int n = e / K, k = e - n * K;
    A[k * N + n] = __ldg(W + (int64_t)n * ldw + k0 + k);
  }
}

// A[k][n] = W[k][n] for k < K, n < N (natural stage: out = W^T g).
__device__ __forceinline__ void stage_n(const float* __restrict__ W, int N, int K, int ldw, float* A) {
  for (int e = threadIdx.x; e < N * K; e += kThreads) {
    const int k = e / N, n = e - k * N;
    A[e] = __ldg(W + (int64_t)k * ldw + n);
  }
}

// out[n][s] = act(sum_k A[k][n] in[k][s] + bias[n]) for n < N, s < TS; act = ReLU if relu,
// and out = 0 where mask[n][s] <= 0 if mask is given (the ReLU derivative of the backward).
// A thread owns 4 consecutive samples of every (GY)-th output row.
template <int TS, int LD>
__device__ __forceinline__ void tile_gemm(const float* __restrict__ A, int N, int K, const float* __restrict__ in,
                                          float* __restrict__ out, const float* __restrict__ bias, bool relu,
                                          const float* __restrict__ mask) {
  constexpr int GX = TS / 4;
  constexpr int GY = kThreads / GX;
  constexpr int R = (kDeformMaxHidden + GY - 1) / GY;
  const int tx = threadIdx.x % GX, ty = threadIdx.x / GX;
  float acc[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[r][j] = 0.0f;
  for (int k = 0; k < K; ++k) {
    const float* ik = in + k * LD + 4 * tx;
    const float a0 = ik[0], a1 = ik[1], a2 = ik[2], a3 = ik[3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = ty + r * GY;
      const float w = n < N ? A[k * N + n] : 0.0f;
      acc[r][0] = fmaf(w, a0, acc[r][0]);
      acc[r][1] = fmaf(w, a1, acc[r][1]);
      acc[r][2] = fmaf(w, a2, acc[r][2]);
      acc[r][3] = fmaf(w, a3, acc[r][3]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int n = ty + r * GY;
    if (n >= N) continue;
    const float b = bias ? bias[n] : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = 4 * tx + j;
      float v = acc[r][j] + b;
      if (relu) v = fmaxf(v, 0.0f);
      if (mask && !(mask[n * LD + s] > 0.0f)) v = 0.0f;
      out[n * LD + s] = v;
    }
  }
}

// part[o][i] += sum_s g[o][s] a[i][s] over the tile, for O rows and I columns (both
// multiples of 8): 8 x 8 register blocks, one read-modify-write of the CTA's partials.
__device__ __forceinline__ void accumulate_dw(const float* __restrict__ g, const float* __restrict__ a, int O, int I,
                                              float* __restrict__ part, int ldp) {
  const int bo_n = O / 8, bi_n = I / 8;
  for (int b = threadIdx.x; b < bo_n * bi_n; b += kThreads) {
    const int bo = b / bi_n, bi = b - bo * bi_n;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = 0.0f;
    for (int s = 0; s < kBwdTS; ++s) {
      float gv[8], av[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) gv[r] = g[(bo * 8 + r) * kBwdLD + s];
#pragma unroll
      for (int c = 0; c < 8; ++c) av[c] = a[(bi * 8 + c) * kBwdLD + s];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(gv[r], av[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float* row = part + (int64_t)(bo * 8 + r) * ldp + bi * 8;
#pragma unroll
      for (int c = 0; c < 8; ++c) row[c] += acc[r][c];
    }
  }
}

// ------------------------------------------------------------------ forward
__global__ void __launch_bounds__(kThreads) k_deform_bias(const __grid_constant__ Plan P) {
  const ViewDev& V = P.v[blockIdx.x];
  if (!V.has_deform) return;
  const DeformDev& D = V.deform;
  const int n_in = D.n_feat + D.pose_dim;
  for (int o = threadIdx.x; o < D.hidden; o += kThreads) {
    float b = 0.0f;
    for (int k = 0; k < D.pose_dim; ++k) b = fmaf(__ldg(D.weights + (int64_t)o * n_in + D.n_feat + k), D.pose[k], b);
    D.pose_bias[o] = b;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_deform_fwd(const __grid_constant__ Plan P) {
  extern __shared__ float sm[];
  float* A = sm;                                           // [<=128][<=128] staged weights
  float* fin = A + kDeformMaxHidden * kDeformMaxHidden;    // [n_feat][LD]
  float* h0 = fin + kDeformMaxFeat * kFwdLD;               // [H][LD]
  float* h1 = h0 + kDeformMaxHidden * kFwdLD;              // [H][LD]
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  const int64_t n_tiles = S / kFwdTS;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t s0 = t * kFwdTS;
    const ViewDev& V = P.v[view_of_slot(P, s0)];
    if (!V.has_deform || V.deform.tc) continue;
    const DeformDev& D = V.deform;
    const int H = D.hidden, n_in = D.n_feat + D.pose_dim;
    for (int e = threadIdx.x; e < D.n_feat * kFwdTS; e += kThreads) {
      const int k = e / kFwdTS, s = e - k * kFwdTS;
      fin[k * kFwdLD + s] = P.ws.feat_d[(int64_t)k * S_cap + s0 + s];
    }
    stage_t(D.weights, H, D.n_feat, n_in, 0, A);
    __syncthreads();
    tile_gemm<kFwdTS, kFwdLD>(A, H, D.n_feat, fin, h0, D.pose_bias, true, nullptr);
    __syncthreads();
    float* cur = h0;
    float* nxt = h1;
    for (int l = 1; l < D.n_hidden; ++l) {
      stage_t(D.weights + layer_offset(D, l), H, H, H, 0, A);
      __syncthreads();
      tile_gemm<kFwdTS, kFwdLD>(A, H, H, cur, nxt, nullptr, true, nullptr);
      __syncthreads();
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    stage_t(D.weights + layer_offset(D, D.n_hidden), 3, H, H, 0, A);
    __syncthreads();
    tile_gemm<kFwdTS, kFwdLD>(A, 3, H, cur, nxt, nullptr, false, nullptr);   // delta v -> nxt[0..2]
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * kFwdTS; e += kThreads) {
      const int a = e / kFwdTS, s = e - a * kFwdTS;
      const int64_t g = s0 + s;
      if (P.ws.s_ray[g] >= 0) P.ws.s_vc[a * S_cap + g] = P.ws.s_vt[a * S_cap + g] + nxt[a * kFwdLD + s];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ backward
// dL/dv_c of every sample of a view with a deformation net, from dL/dfeat of the field's
// encoding at v_c.
__global__ void __launch_bounds__(256) k_encode_dx(const __grid_constant__ Plan P) {
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    const ViewDev& V = P.v[view_of_slot(P, s)];
    if (!V.has_deform) continue;
    float d[3] = {0.0f, 0.0f, 0.0f};
    if (P.ws.s_ray[s] >= 0) {
      const FieldDev& F = V.field;
      const float x[3] = {P.ws.s_vc[s], P.ws.s_vc[S_cap + s], P.ws.s_vc[2 * S_cap + s]};
      const uint32_t tmask = (1u << F.log2T) - 1u;
      for (int l = 0; l < F.L; ++l) {
        const int res = F.res[l];
        const bool dense = (F.dense_mask >> l) & 1u;
        int c[3];
        float fr[3], sc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          c[a] = level_cell(x[a], res, fr[a]);
          sc[a] = (x[a] < -1.0f || x[a] > 1.0f) ? 0.0f : 0.5f * (float)res;
        }
        const float2 g = make_float2(P.ws.dfeat[(int64_t)(2 * l) * S_cap + s],
                                     P.ws.dfeat[(int64_t)(2 * l + 1) * S_cap + s]);
        const float2* tab = reinterpret_cast<const float2*>(F.tables) + ((size_t)l << F.log2T);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int b[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
          const uint32_t idx = vertex_index((uint32_t)(c[0] + b[0]), (uint32_t)(c[1] + b[1]), (uint32_t)(c[2] + b[2]),
                                            res, dense, tmask);
          const float2 e = __ldg(tab + idx);
          const float ge = fmaf(g.x, e.x, g.y * e.y);
          const float w[3] = {b[0] ? fr[0] : 1.0f - fr[0], b[1] ? fr[1] : 1.0f - fr[1], b[2] ? fr[2] : 1.0f - fr[2]};
          d[0] = fmaf((b[0] ? sc[0] : -sc[0]) * (w[1] * w[2]), ge, d[0]);
          d[1] = fmaf((b[1] ? sc[1] : -sc[1]) * (w[0] * w[2]), ge, d[1]);
          d[2] = fmaf((b[2] ? sc[2] : -sc[2]) * (w[0] * w[1]), ge, d[2]);
        }
      }
    }
    P.ws.dvc[s] = d[0];
    P.ws.dvc[S_cap + s] = d[1];
    P.ws.dvc[2 * S_cap + s] = d[2];
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_deform_bwd(const __grid_constant__ Plan P) {
  extern __shared__ float sm[];
  float* A = sm;                                                // staged weights
  float* fin = A + kDeformMaxHidden * kDeformMaxHidden;         // [n_feat][LD]
  float* hs = fin + kDeformMaxFeat * kBwdLD;                    // [n_hidden][H][LD]
  float* g0 = hs + kDeformMaxLayers * kDeformMaxHidden * kBwdLD; // [H][LD]
  float* g1 = g0 + kDeformMaxHidden * kBwdLD;                   // [H][LD]
  float* gsum = g1 + kDeformMaxHidden * kBwdLD;                 // [H]
  const int64_t S_cap = P.ws.S_cap;
  const int64_t S = P.ws.view_base[P.n_views];
  if (S > S_cap) return;
  const int64_t n_tiles = S / kBwdTS;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t s0 = t * kBwdTS;
    const ViewDev& V = P.v[view_of_slot(P, s0)];
    if (!V.has_deform || V.deform.tc) continue;
    const DeformDev& D = V.deform;
    const int H = D.hidden, n = D.n_hidden, n_in = D.n_feat + D.pose_dim;
    float* part = D.dw_scratch + (int64_t)blockIdx.x * D.n_w;
    auto h = [&](int l) { return hs + (int64_t)l * kDeformMaxHidden * kBwdLD; };
    // recompute the forward activations
    for (int e = threadIdx.x; e < D.n_feat * kBwdTS; e += kThreads) {
      const int k = e / kBwdTS, s = e - k * kBwdTS;
      fin[k * kBwdLD + s] = P.ws.feat_d[(int64_t)k * S_cap + s0 + s];
    }
    stage_t(D.weights, H, D.n_feat, n_in, 0, A);
    __syncthreads();
    tile_gemm<kBwdTS, kBwdLD>(A, H, D.n_feat, fin, h(0), D.pose_bias, true, nullptr);
    __syncthreads();
    for (int l = 1; l < n; ++l) {
      stage_t(D.weights + layer_offset(D, l), H, H, H, 0, A);
      __syncthreads();
      tile_gemm<kBwdTS, kBwdLD>(A, H, H, h(l - 1), h(l), nullptr, true, nullptr);
      __syncthreads();
    }
    // output layer: g_out = dL/d(delta v) = dL/dv_c
    for (int e = threadIdx.x; e < 3 * kBwdTS; e += kThreads) {
      const int a = e / kBwdTS, s = e - a * kBwdTS;
      g1[a * kBwdLD + s] = P.ws.dvc[(int64_t)a * S_cap + s0 + s];
    }
    __syncthreads();
    {
      float* po = part + layer_offset(D, n);
      for (int e = threadIdx.x; e < 3 * H; e += kThreads) {
        const int a = e / H, i = e - a * H;
        float acc = 0.0f;
        for (int s = 0; s < kBwdTS; ++s) acc = fmaf(g1[a * kBwdLD + s], h(n - 1)[i * kBwdLD + s], acc);
        po[e] += acc;
      }
    }
    stage_n(D.weights + layer_offset(D, n), H, 3, H, A);
    __syncthreads();
    tile_gemm<kBwdTS, kBwdLD>(A, H, 3, g1, g0, nullptr, false, h(n - 1));   // g_n
    __syncthreads();
    float* g = g0;
    float* gp = g1;
    for (int l = n - 1; l >= 1; --l) {
      accumulate_dw(g, h(l - 1), H, H, part + layer_offset(D, l), H);
      stage_n(D.weights + layer_offset(D, l), H, H, H, A);
      __syncthreads();
      tile_gemm<kBwdTS, kBwdLD>(A, H, H, g, gp, nullptr, false, h(l - 1));
      __syncthreads();
      float* tmp = g;
      g = gp;
      gp = tmp;
    }
    // first layer: feature columns, pose columns (rank one: (sum_s g) theta^T), dL/df
    accumulate_dw(g, fin, H, D.n_feat, part, n_in);
    for (int o = threadIdx.x; o < H; o += kThreads) {
      float acc = 0.0f;
      for (int s = 0; s < kBwdTS; ++s) acc += g[o * kBwdLD + s];
      gsum[o] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < H * D.pose_dim; e += kThreads) {
      const int o = e / D.pose_dim, k = e - o * D.pose_dim;
      part[(int64_t)o * n_in + D.n_feat + k] += gsum[o] * D.pose[k];
    }
    for (int e = threadIdx.x; e < H * D.n_feat; e += kThreads) {   // A[o][k] = W_1[o][k]
      const int o = e / D.n_feat, k = e - o * D.n_feat;
      A[e] = __ldg(D.weights + (int64_t)o * n_in + k);
    }
    __syncthreads();
    tile_gemm<kBwdTS, kBwdLD>(A, D.n_feat, H, g, gp, nullptr, false, nullptr);
    __syncthreads();
    for (int e = threadIdx.x; e < D.n_feat * kBwdTS; e += kThreads) {
      const int k = e / kBwdTS, s = e - k * kBwdTS;
      P.ws.dfeat_d[(int64_t)k * S_cap + s0 + s] = gp[k * kBwdLD + s];
    }
    __syncthreads();
  }
}

__global__ void k_deform_reduce(const float* __restrict__ parts, int n_parts, int64_t n_w, float* grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_w; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int p = 0; p < n_parts; ++p) acc += parts[(int64_t)p * n_w + i];
    grad[i] += acc;
  }
}

constexpr size_t kFwdSmem =
    sizeof(float) * ((size_t)kDeformMaxHidden * kDeformMaxHidden + kDeformMaxFeat * kFwdLD + 2 * kDeformMaxHidden * kFwdLD);
constexpr size_t kBwdSmem =
    sizeof(float) * ((size_t)kDeformMaxHidden * kDeformMaxHidden + kDeformMaxFeat * kBwdLD +
                     (size_t)kDeformMaxLayers * kDeformMaxHidden * kBwdLD + 2 * kDeformMaxHidden * kBwdLD +
                     kDeformMaxHidden);

}  // namespace

cudaError_t launch_deform_forward(const Plan& P, int num_sms, cudaStream_t s) {
  k_deform_bias<<<P.n_views, kThreads, 0, s>>>(P);
  bool simt = false, tc = false;
  for (int v = 0; v < P.n_views; ++v) {
    if (!P.v[v].has_deform) continue;
    (P.v[v].deform.tc ? tc : simt) = true;
  }
  cudaError_t e = cudaSuccess;
  if (simt) {
    e = cudaFuncSetAttribute(k_deform_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    k_deform_fwd<<<num_sms, kThreads, kFwdSmem, s>>>(P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && tc) e = launch_deform_forward_tc(P, num_sms, s);
  return e;
}

cudaError_t launch_encode_dx(const Plan& P, int num_sms, cudaStream_t s) {
  k_encode_dx<<<num_sms * 8, 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_deform_backward(const Plan& P, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_deform_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
  if (e != cudaSuccess) return e;
  k_deform_bwd<<<num_sms, kThreads, kBwdSmem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_deform_reduce(const DeformDev& D, int n_parts, cudaStream_t s) {
  k_deform_reduce<<<ceil_div(D.n_w, 256), 256, 0, s>>>(D.dw_scratch, n_parts, D.n_w, D.grad_weights);
  return cudaGetLastError();
}

}  // namespace invr
