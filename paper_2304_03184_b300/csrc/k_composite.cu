// Front-to-back volume rendering of every ray through every view (Sec. 3 "share
// volumetric rendering"; Sec. 4.3 depth-occlusion composition), and, for training, the
// Huber colour loss and the adjoint of the compositing.
//
//   alpha_j = 1 - exp(-sigma_j dt),  T_{j+1} = T_j (1 - alpha_j),
//   C = sum T_j alpha_j c_j,  A = sum T_j alpha_j,  D = sum T_j alpha_j t_j,
// over the occupied samples in order, stopping after the first with T_{j+1} < t_eps.
// Two views (human, object): the nearer by expected depth (D_h A_o <= D_o A_h, ties to
// the human) is laid over the farther: X = X_n + (1 - A_n) X_f for X in {C, A, D}; or,
// jointly per sample (k_composite_joint), densities added and colours mixed by density.
//
// Training adjoint per ray (k <= stop):
//   dC/dc_j = T_j alpha_j,   dC/dsigma_j = dt (T_{j+1} c_j - (C - sum_{k<=j} T_k alpha_k c_k))
// folded with sigma = exp(o_0) and c = sigmoid(z) into dL/do_0 and dL/dz per sample.
//
// Rendering: one thread per ray, samples read 4 at a time.  Training: one warp per 32 rays
// with segmented scans over their samples (k_composite_train).
#include "invr_internal.cuh"

namespace invr {

__device__ __forceinline__ bool ray_dt(const ViewDev& V, int64_t r, int n_samples, float& dt) {
  const int64_t n = V.n_rays;
  const float3 o = make_float3(__ldg(V.o + r), __ldg(V.o + n + r), __ldg(V.o + 2 * n + r));
  const float3 d = make_float3(__ldg(V.d + r), __ldg(V.d + n + r), __ldg(V.d + 2 * n + r));
  float tn;
  return ray_box(o, d, n_samples, tn, dt);
}

// Composite one ray of one view; res = (C.rgb, A, D); returns samples used.
__device__ __forceinline__ int composite(const Plan& P, int64_t g, float dt, float res[5]) {
  const int64_t S_cap = P.ws.S_cap;
  const int64_t first = P.ws.ray_first[g];
  const int cnt = P.ws.ray_count[g];
  float T = 1.0f;
  for (int c = 0; c < 5; ++c) res[c] = 0.0f;
  int used = cnt;
  // chunks of 4 samples: every load of a chunk is issued before its arithmetic, which runs
  // sample by sample in order (the same operations as a one-sample loop)
  for (int k = 0; k < cnt; k += 4) {
    float sg[4], cr[4], cg[4], cb[4], tj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t s = first + k + j;
      const bool in = k + j < cnt;
      sg[j] = in ? P.ws.out[s] : 0.0f;
      cr[j] = in ? P.ws.out[S_cap + s] : 0.0f;
      cg[j] = in ? P.ws.out[2 * S_cap + s] : 0.0f;
      cb[j] = in ? P.ws.out[3 * S_cap + s] : 0.0f;
      tj[j] = in ? P.ws.s_t[s] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (k + j >= cnt) return used;
      const float x = sg[j] * dt;
      const float alpha = -expm1f(-x);
      const float w = T * alpha;
      res[0] = fmaf(w, cr[j], res[0]);
      res[1] = fmaf(w, cg[j], res[1]);
      res[2] = fmaf(w, cb[j], res[2]);
      res[3] += w;
      res[4] = fmaf(w, tj[j], res[4]);
      T *= expf(-x);
      if (T < P.t_eps) return k + j + 1;
    }
  }
  return used;
}

__global__ void __launch_bounds__(256) k_composite_render(const __grid_constant__ Plan P, int64_t n_rays,
                                                          float* rgba, float* depth) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  if (P.ws.view_base[P.n_views] > P.ws.S_cap) return;
  float res[2][5];
  for (int v = 0; v < P.n_views; ++v) {
    const int64_t g = P.v[v].ray_begin + r;
    float dt = 0.0f;
    if (ray_dt(P.v[v], r, P.n_samples, dt)) {
      P.ws.ray_used[g] = composite(P, g, dt, res[v]);
    } else {
      for (int c = 0; c < 5; ++c) res[v][c] = 0.0f;
      P.ws.ray_used[g] = 0;
    }
  }
  float out[5];
  if (P.n_views == 1) {
    for (int c = 0; c < 5; ++c) out[c] = res[0][c];
  } else {
    const bool human_near = res[0][4] * res[1][3] <= res[1][4] * res[0][3];
    const float* n = res[human_near ? 0 : 1];
    const float* f = res[human_near ? 1 : 0];
    for (int c = 0; c < 5; ++c) out[c] = n[c] + (1.0f - n[3]) * f[c];
  }
  bool finite = true;
  for (int c = 0; c < 4; ++c) {
    rgba[c * n_rays + r] = out[c];
    finite &= isfinite(out[c]);
  }
  depth[r] = out[4];
  if (!(finite && isfinite(out[4]))) flag_status(P.status, kStatusNonFinite);
}

cudaError_t launch_composite_render(const Plan& P, int64_t n_rays, float* rgba, float* depth, cudaStream_t s) {
  if (n_rays > 0) k_composite_render<<<ceil_div(n_rays, 256), 256, 0, s>>>(P, n_rays, rgba, depth);
  return cudaGetLastError();
}

// Joint per-sample compositing of two views (human = view 0, object = view 1) of the same
// rays: both are sampled at the same t_j, so the two compacted sample lists of a ray merge
// by t; at a shared t_j the densities add and the colours mix in proportion to density,
// and the mixture is composited front to back with early termination.
__global__ void __launch_bounds__(256) k_composite_joint(const __grid_constant__ Plan P, int64_t n_rays,
                                                         float* rgba, float* depth) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  if (P.ws.view_base[P.n_views] > P.ws.S_cap) return;
  const int64_t S_cap = P.ws.S_cap;
  float out[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float dt = 0.0f;
  if (ray_dt(P.v[0], r, P.n_samples, dt)) {
    const int64_t g0 = P.v[0].ray_begin + r, g1 = P.v[1].ray_begin + r;
    int64_t i = P.ws.ray_first[g0], k = P.ws.ray_first[g1];
    const int64_t i_end = i + P.ws.ray_count[g0], k_end = k + P.ws.ray_count[g1];
    float T = 1.0f;
    while (i < i_end || k < k_end) {
      const float ti = i < i_end ? P.ws.s_t[i] : INFINITY;
      const float tk = k < k_end ? P.ws.s_t[k] : INFINITY;
      const float t = fminf(ti, tk);
      float sig = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
      if (ti == t) {
        const float si = P.ws.out[i];
        sig += si;
        cr = fmaf(si, P.ws.out[S_cap + i], cr);
        cg = fmaf(si, P.ws.out[2 * S_cap + i], cg);
        cb = fmaf(si, P.ws.out[3 * S_cap + i], cb);
        ++i;
      }
      if (tk == t) {
        const float sk = P.ws.out[k];
        sig += sk;
        cr = fmaf(sk, P.ws.out[S_cap + k], cr);
        cg = fmaf(sk, P.ws.out[2 * S_cap + k], cg);
        cb = fmaf(sk, P.ws.out[3 * S_cap + k], cb);
        ++k;
      }
      const float inv = sig > 0.0f ? 1.0f / sig : 0.0f;
      const float x = sig * dt;
      const float w = T * -expm1f(-x);
      out[0] = fmaf(w, cr * inv, out[0]);
      out[1] = fmaf(w, cg * inv, out[1]);
      out[2] = fmaf(w, cb * inv, out[2]);
      out[3] += w;
      out[4] = fmaf(w, t, out[4]);
      T *= expf(-x);
      if (T < P.t_eps) break;
    }
  }
  bool finite = true;
  for (int c = 0; c < 4; ++c) {
    rgba[c * n_rays + r] = out[c];
    finite &= isfinite(out[c]);
  }
  depth[r] = out[4];
  if (!(finite && isfinite(out[4]))) flag_status(P.status, kStatusNonFinite);
}

cudaError_t launch_composite_joint(const Plan& P, int64_t n_rays, float* rgba, float* depth, cudaStream_t s) {
  if (n_rays > 0) k_composite_joint<<<ceil_div(n_rays, 256), 256, 0, s>>>(P, n_rays, rgba, depth);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ training
__device__ __forceinline__ float huber(float x, float delta) {
  const float ax = fabsf(x);
  return ax <= delta ? 0.5f * x * x : delta * (ax - 0.5f * delta);
}

__device__ __forceinline__ float huber_grad(float x, float delta) {
  return fabsf(x) <= delta ? x : copysignf(delta, x);
}

// Training compositing, loss and adjoint: one warp per 32 consecutive rays.  The rays' occupied
// samples are contiguous slots (in ray order; padding between views has ray id -1), so the warp
// walks them 32 at a time, one sample per lane, and every per-ray sum is a segmented scan over
// the lanes (segments = runs of equal ray id): the optical depth S_j = sum_{k<j} x_k with
// x_k = sigma_k dt gives T_j = exp(-S_j) (the product of the exp(-x_k), in another rounding
// order), and the prefixes of T_j alpha_j c_j and T_j alpha_j t_j give the adjoint.  A ray lane
// keeps its ray's running sums between chunks.  Pass 1 accumulates C, A, D; the ray lanes then
// take the loss; pass 2 recomputes the same scans and writes dL/do_0, dL/dz per sample.  Loads
// and stores are coalesced and every lane of a chunk has a sample, where one thread per ray
// left 7.8 of 32 lanes active (rays of a warp differ in length).
__device__ __forceinline__ float seg_scan(float v, int lane, int start) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= start) v += y;
  }
  return v;
}

// Two warps (64 rays) per block: a block holds its slot until its slowest warp ends, and rays
// drawn in random order give the warps of a block very different sample counts (0.350 ms per
// batched step against 0.398 with 8 warps per block and 0.39 with one).
constexpr int kCompWarps = 2;

__global__ void __launch_bounds__(32 * kCompWarps) k_composite_train(const __grid_constant__ Plan P, float* loss_part) {
  __shared__ float red[kCompWarps];
  __shared__ float seg[kCompWarps][32][8];  // per warp, per ray of the group: this chunk's segment totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t S_cap = P.ws.S_cap;
  const int64_t g0 = (int64_t)blockIdx.x * (32 * kCompWarps) + wid * 32;
  const int64_t g = g0 + lane;  // this lane's ray
  const bool ray_ok = P.ws.view_base[P.n_views] <= S_cap && g < P.total_rays;
  float loss = 0.0f;
  // ---- ray lane set-up
  int v = 0;
  int64_t r = 0;
  float dt = 0.0f;
  int first = 0, cnt = 0;
  if (ray_ok) {
    v = view_of_ray(P, g);
    r = g - P.v[v].ray_begin;
    if (ray_dt(P.v[v], r, P.n_samples, dt)) {
      first = P.ws.ray_first[g];
      cnt = P.ws.ray_count[g];
    }
  }
  seg[wid][lane][7] = 0.0f;  // no segment total pending
  __syncwarp();
  const int lo = __reduce_min_sync(FULL, cnt > 0 ? (unsigned)first : 0x7FFFFFFFu);
  const int hi = (int)__reduce_max_sync(FULL, cnt > 0 ? (unsigned)(first + cnt) : 0u);
  // one sample per lane of a chunk: its ray (local lane), the segment it belongs to
  auto sample = [&](int base, int& lr, float& sg, float& c0, float& c1, float& c2, float& tt, int& start,
                    unsigned& heads) {
    const int s = base + lane;
    const int key = s < hi ? P.ws.s_ray[s] : -1;
    lr = key >= 0 ? (int)(key - g0) : -1;
    sg = c0 = c1 = c2 = tt = 0.0f;
    if (lr >= 0) {
      sg = P.ws.out[s];
      c0 = P.ws.out[S_cap + s];
      c1 = P.ws.out[2 * S_cap + s];
      c2 = P.ws.out[3 * S_cap + s];
      tt = P.ws.s_t[s];
    }
    const int prev = __shfl_up_sync(FULL, key, 1);
    heads = __ballot_sync(FULL, lane == 0 || prev != key);
    start = 31 - __clz(heads & (FULL >> (31 - lane)));
  };
  // ---- pass 1: C, A, D per ray
  float xs = 0.0f, res[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, nused = 0.0f;
  for (int base = lo; base < hi; base += 32) {
    int lr, start;
    unsigned heads;
    float sg, c0, c1, c2, tt;
    sample(base, lr, sg, c0, c1, c2, tt, start, heads);
    const int src = lr >= 0 ? lr : 0;
    const float dts = __shfl_sync(FULL, dt, src), carry = __shfl_sync(FULL, xs, src);
    const float x = lr >= 0 ? sg * dts : 0.0f;
    const float incl = seg_scan(x, lane, start);
    const float up = __shfl_up_sync(FULL, incl, 1);
    const float excl = lane > start ? up : 0.0f;
    const float T = expf(-(carry + excl));
    const bool used = lr >= 0 && T >= P.t_eps;
    const float w = used ? T * -expm1f(-x) : 0.0f;
    float q[6] = {w * c0, w * c1, w * c2, w, w * tt, used ? 1.0f : 0.0f};
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = seg_scan(q[k], lane, start);
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && lr >= 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) seg[wid][lr][k] = q[k];
      seg[wid][lr][6] = incl;
      seg[wid][lr][7] = 1.0f;
    }
    __syncwarp();
    if (seg[wid][lane][7] != 0.0f) {
      for (int k = 0; k < 5; ++k) res[k] += seg[wid][lane][k];
      nused += seg[wid][lane][5];
      xs += seg[wid][lane][6];
      seg[wid][lane][7] = 0.0f;
    }
    __syncwarp();
  }
  // ---- ray lane: loss and dL/dC, dL/dD
  float dC[3] = {0.f, 0.f, 0.f}, dD = 0.0f;
  if (ray_ok) {
    const ViewDev& V = P.v[v];
    P.ws.ray_used[g] = (int)nused;
    bool finite = true;
    float e[3];
    for (int c = 0; c < 3; ++c) {
      e[c] = res[c] - __ldg(V.target + c * V.n_rays + r);
      finite &= isfinite(res[c]);
    }
    if (P.loss_kind == kLossHuber) {
      for (int c = 0; c < 3; ++c) {
        loss += huber(e[c], P.huber_delta);
        dC[c] = huber_grad(e[c], P.huber_delta) * P.loss_norm;
      }
    } else {
      // the paper's losses: M ||e||_2 + w M |D_hat - D| (sum over rays, loss_norm = 1)
      const float M = V.mask ? __ldg(V.mask + r) : 1.0f;
      const float n = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      const float inv = n > 0.0f ? M / n : 0.0f;
      for (int c = 0; c < 3; ++c) dC[c] = e[c] * inv;
      const float ed = res[4] - __ldg(V.depth_target + r);
      dD = P.depth_weight * M * (ed > 0.0f ? 1.0f : (ed < 0.0f ? -1.0f : 0.0f));
      loss += M * n + P.depth_weight * M * fabsf(ed);
      finite &= isfinite(res[4]);
    }
    if (!finite) flag_status(P.status, kStatusNonFinite);
    if (V.rgba_out) {
      for (int c = 0; c < 4; ++c) V.rgba_out[c * V.n_rays + r] = res[c];
    }
    if (V.depth_out) V.depth_out[r] = res[4];
  }
  // ---- pass 2: the adjoint, the same scans again
  float xs2 = 0.0f, pre[4] = {0.f, 0.f, 0.f, 0.f};
  for (int base = lo; base < hi; base += 32) {
    int lr, start;
    unsigned heads;
    float sg, c0, c1, c2, tt;
    sample(base, lr, sg, c0, c1, c2, tt, start, heads);
    const int src = lr >= 0 ? lr : 0;
    const float dts = __shfl_sync(FULL, dt, src), carry = __shfl_sync(FULL, xs2, src);
    const float x = lr >= 0 ? sg * dts : 0.0f;
    const float incl = seg_scan(x, lane, start);
    const float up = __shfl_up_sync(FULL, incl, 1);
    const float excl = lane > start ? up : 0.0f;
    const float T = expf(-(carry + excl));
    const float Tn = expf(-(carry + incl));
    const bool used = lr >= 0 && T >= P.t_eps;
    const float w = used ? T * -expm1f(-x) : 0.0f;
    float q[4] = {w * c0, w * c1, w * c2, w * tt};
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = seg_scan(q[k], lane, start);
    float rc[4], dc[4], pc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rc[k] = __shfl_sync(FULL, k < 3 ? res[k] : res[4], src);
      dc[k] = __shfl_sync(FULL, k < 3 ? dC[k] : dD, src);
      pc[k] = __shfl_sync(FULL, pre[k], src);
    }
    if (lr >= 0) {
      const int s = base + lane;
      float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
      if (used) {
        const float col[4] = {c0, c1, c2, tt};
        float dsig = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) dsig = fmaf(dc[k], Tn * col[k] - (rc[k] - (pc[k] + q[k])), dsig);
        d0 = dsig * dts * sg;
        d1 = dc[0] * w * c0 * (1.0f - c0);
        d2 = dc[1] * w * c1 * (1.0f - c1);
        d3 = dc[2] * w * c2 * (1.0f - c2);
      }
      P.ws.dout[s] = d0;
      P.ws.dout[S_cap + s] = d1;
      P.ws.dout[2 * S_cap + s] = d2;
      P.ws.dout[3 * S_cap + s] = d3;
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && lr >= 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) seg[wid][lr][k] = q[k];
      seg[wid][lr][6] = incl;
      seg[wid][lr][7] = 1.0f;
    }
    __syncwarp();
    if (seg[wid][lane][7] != 0.0f) {
      for (int k = 0; k < 4; ++k) pre[k] += seg[wid][lane][k];
      xs2 += seg[wid][lane][6];
      seg[wid][lane][7] = 0.0f;
    }
    __syncwarp();
  }
  // deterministic block sum of the per-ray loss terms
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) red[wid] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int k = 0; k < kCompWarps; ++k) t += red[k];
    loss_part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_loss_finalize(const float* part, int n, float norm, float* loss) {
  __shared__ float red[32];
  float t = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < 32; ++w) s += red[w];
    *loss = s * norm;
  }
}

cudaError_t launch_composite_train(const Plan& P, float* loss, cudaStream_t s) {
  const int blocks = ceil_div(P.total_rays, 32 * kCompWarps);
  k_composite_train<<<blocks, 32 * kCompWarps, 0, s>>>(P, P.ws.loss_part);
  k_loss_finalize<<<1, 1024, 0, s>>>(P.ws.loss_part, blocks, P.loss_norm, loss);
  return cudaGetLastError();
}

}  // namespace invr
