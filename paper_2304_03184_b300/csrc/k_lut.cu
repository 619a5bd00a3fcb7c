// Look-up-table neighbour search of the human warp (Sec. 4.2, "On-the-fly Radiance
// Fields"): the approximate O(1) replacement of the K-nearest-node query.
//
//  * Canonical KNN field, built once per graph: for each of G^3 voxels over [-1,1]^3 the
//    K canonical nodes x_i nearest to the voxel centre (exact, same key and tie rule as
//    the live search, candidates from a 128^3 grid over the canonical nodes).
//  * Live index field, built per frame: every canonical voxel centre is carried to live
//    space by the forward warp of Eq. 2 (the blend of its own K nodes' motions) and its
//    index is stored in the live voxel it lands in; where several land in one voxel the
//    smallest index stays (atomicMin), voxels carried outside [-1,1]^3 are dropped and
//    live voxels that receive none are holes (the warp then uses the exact search).
//
// The integer results are decided by single-precision recipes with explicitly rounded
// operations (no contraction), so any implementation of the same recipe builds the same
// tables.  The weights' exponential is Cody-Waite range reduction (x = n ln2 + r, ln2
// split in a short high part and a low part) with the degree-6 Taylor polynomial of e^r
// by Horner's rule, scaled by 2^n; 0 where n < -125.
//
// Bound: the live build is FP32 ALU work (~150 operations per voxel) plus one 4-byte
// atomicMin per voxel into a G^3 x 4 B table (512 MiB at G = 512); the canonical build
// runs once.
#include "knn.cuh"

namespace invr {

__device__ __forceinline__ float lut_exp(float x) {
  const float n = rintf(__fmul_rn(x, 1.44269504f));
  if (n < -125.0f) return 0.0f;
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(n, 0.693145752f)), __fmul_rn(n, 1.42860682e-06f));
  float p = 1.38888889e-03f;
  p = __fadd_rn(__fmul_rn(p, r), 8.33333333e-03f);
  p = __fadd_rn(__fmul_rn(p, r), 4.16666667e-02f);
  p = __fadd_rn(__fmul_rn(p, r), 1.66666667e-01f);
  p = __fadd_rn(__fmul_rn(p, r), 0.5f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  return __fmul_rn(p, __int_as_float(((int)n + 127) << 23));
}

// voxel centre along one axis: (i + 1/2) (2/G) - 1
__device__ __forceinline__ float lut_centre(int i, int G) {
  return __fsub_rn(__fmul_rn(__fadd_rn((float)i, 0.5f), __fdiv_rn(2.0f, (float)G)), 1.0f);
}

// voxel of one coordinate, -1 outside [0, G)
__device__ __forceinline__ int lut_cell(float x, int G) {
  const float f = floorf(__fmul_rn(__fmul_rn(__fadd_rn(x, 1.0f), 0.5f), (float)G));
  return (f >= 0.0f && f < (float)G) ? (int)f : -1;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z)),
                   __fmul_rn(a.w, b.w));
}

__device__ __forceinline__ float cross_c(float a1, float a2, float b1, float b2) {  // a1 b2 - a2 b1
  return __fsub_rn(__fmul_rn(a1, b2), __fmul_rn(a2, b1));
}

// Forward warp (Eq. 2) of canonical point c by its K canonical neighbours ids (ascending
// by canonical key).  Quaternions are stored (w, x, y, z) in the (x, y, z, w) slots.
template <int K>
__device__ __forceinline__ float3 lut_forward(const float4* __restrict__ x_canon, const float4* __restrict__ dq,
                                              float inv_r2, const int (&ids)[K], float3 c) {
  float keys[K];
#pragma unroll
  for (int k = 0; k < K; ++k) keys[k] = knn_key(c, __ldg(x_canon + ids[k]));
  const float4 ref = __ldg(dq + 2 * ids[0]);
  float4 br = make_float4(0.f, 0.f, 0.f, 0.f), bd = br;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float4 r = __ldg(dq + 2 * ids[k]);
    const float4 du = __ldg(dq + 2 * ids[k] + 1);
    float w = lut_exp(__fmul_rn(__fsub_rn(keys[0], keys[k]), inv_r2));
    if (dot4(r, ref) < 0.0f) w = -w;
    br.x = __fadd_rn(br.x, __fmul_rn(w, r.x));
    br.y = __fadd_rn(br.y, __fmul_rn(w, r.y));
    br.z = __fadd_rn(br.z, __fmul_rn(w, r.z));
    br.w = __fadd_rn(br.w, __fmul_rn(w, r.w));
    bd.x = __fadd_rn(bd.x, __fmul_rn(w, du.x));
    bd.y = __fadd_rn(bd.y, __fmul_rn(w, du.y));
    bd.z = __fadd_rn(bd.z, __fmul_rn(w, du.z));
    bd.w = __fadd_rn(bd.w, __fmul_rn(w, du.w));
  }
  const float nr = __fsqrt_rn(dot4(br, br));
  const float4 qr = make_float4(__fdiv_rn(br.x, nr), __fdiv_rn(br.y, nr), __fdiv_rn(br.z, nr), __fdiv_rn(br.w, nr));
  const float4 dn = make_float4(__fdiv_rn(bd.x, nr), __fdiv_rn(bd.y, nr), __fdiv_rn(bd.z, nr), __fdiv_rn(bd.w, nr));
  const float dt = dot4(qr, dn);
  const float sd = __fsub_rn(dn.x, __fmul_rn(dt, qr.x));
  const float v0 = __fsub_rn(dn.y, __fmul_rn(dt, qr.y));
  const float v1 = __fsub_rn(dn.z, __fmul_rn(dt, qr.z));
  const float v2 = __fsub_rn(dn.w, __fmul_rn(dt, qr.w));
  const float w = qr.x, u0 = qr.y, u1 = qr.z, u2 = qr.w;
  // t = 2 (w v - s u - v x u)
  const float vxu0 = cross_c(v1, v2, u1, u2), vxu1 = cross_c(v2, v0, u2, u0), vxu2 = cross_c(v0, v1, u0, u1);
  const float t0 = __fmul_rn(2.0f, __fsub_rn(__fsub_rn(__fmul_rn(w, v0), __fmul_rn(sd, u0)), vxu0));
  const float t1 = __fmul_rn(2.0f, __fsub_rn(__fsub_rn(__fmul_rn(w, v1), __fmul_rn(sd, u1)), vxu1));
  const float t2 = __fmul_rn(2.0f, __fsub_rn(__fsub_rn(__fmul_rn(w, v2), __fmul_rn(sd, u2)), vxu2));
  // R(q_r) c = c + w tt + u x tt, tt = 2 (u x c)
  const float tt0 = __fmul_rn(2.0f, cross_c(u1, u2, c.y, c.z));
  const float tt1 = __fmul_rn(2.0f, cross_c(u2, u0, c.z, c.x));
  const float tt2 = __fmul_rn(2.0f, cross_c(u0, u1, c.x, c.y));
  const float ut0 = cross_c(u1, u2, tt1, tt2), ut1 = cross_c(u2, u0, tt2, tt0), ut2 = cross_c(u0, u1, tt0, tt1);
  return make_float3(__fadd_rn(__fadd_rn(__fadd_rn(c.x, __fmul_rn(w, tt0)), ut0), t0),
                     __fadd_rn(__fadd_rn(__fadd_rn(c.y, __fmul_rn(w, tt1)), ut1), t1),
                     __fadd_rn(__fadd_rn(__fadd_rn(c.z, __fmul_rn(w, tt2)), ut2), t2));
}

template <int K>
__global__ void __launch_bounds__(256) k_lut_canon(const __grid_constant__ WarpDev W, int G, uint16_t* canon) {
  const int64_t n = (int64_t)G * G * G;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float3 c = make_float3(lut_centre((int)(v % G), G), lut_centre((int)((v / G) % G), G),
                                 lut_centre((int)(v / ((int64_t)G * G)), G));
    float keys[K];
    int ids[K];
    knn_select<K>(W, c, keys, ids);
#pragma unroll
    for (int k = 0; k < K; ++k) canon[v * K + k] = (uint16_t)ids[k];
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_lut_live(const float4* __restrict__ x_canon, const float4* __restrict__ dq,
                                                  float inv_r2, int G, const uint16_t* __restrict__ canon,
                                                  uint32_t* live) {
  const int64_t n = (int64_t)G * G * G;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float3 c = make_float3(lut_centre((int)(k % G), G), lut_centre((int)((k / G) % G), G),
                                 lut_centre((int)(k / ((int64_t)G * G)), G));
    int ids[K];
#pragma unroll
    for (int j = 0; j < K; ++j) ids[j] = __ldg(canon + k * K + j);
    const float3 q = lut_forward<K>(x_canon, dq, inv_r2, ids, c);
    const int cx = lut_cell(q.x, G), cy = lut_cell(q.y, G), cz = lut_cell(q.z, G);
    if (cx < 0 || cy < 0 || cz < 0) continue;
    atomicMin(live + (cx + (int64_t)G * (cy + (int64_t)G * cz)), (uint32_t)k);
  }
}

__global__ void k_pack_points(const float* __restrict__ x, int n, float4* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float4(x[i], x[n + i], x[2 * n + i], 0.0f);
}

cudaError_t launch_pack_points(const float* x_soa, int n, float4* out, cudaStream_t s) {
  k_pack_points<<<ceil_div(n, 256), 256, 0, s>>>(x_soa, n, out);
  return cudaGetLastError();
}

template <int K>
static void canon_k(const WarpDev& W, int G, uint16_t* canon, int grid, cudaStream_t s) {
  k_lut_canon<K><<<grid, 256, 0, s>>>(W, G, canon);
}

template <int K>
static void live_k(const float4* x, const float4* dq, float inv_r2, int G, const uint16_t* canon, uint32_t* live,
                   int grid, cudaStream_t s) {
  k_lut_live<K><<<grid, 256, 0, s>>>(x, dq, inv_r2, G, canon, live);
}

cudaError_t launch_lut_canon(const float4* x_canon, int n, int K, const uint32_t* cand, const uint32_t* cand_head,
                             int cap, int G, uint16_t* canon, int num_sms, cudaStream_t s) {
  WarpDev W{};
  W.mode = 1;
  W.x_live = x_canon;  // the search runs over the canonical nodes
  W.cand = cand;
  W.cand_head = cand_head;
  W.cap = cap;
  W.n_nodes = n;
  W.K = K;
  const int grid = num_sms * 8;
  switch (K) {
    case 1: canon_k<1>(W, G, canon, grid, s); break;
    case 2: canon_k<2>(W, G, canon, grid, s); break;
    case 3: canon_k<3>(W, G, canon, grid, s); break;
    case 4: canon_k<4>(W, G, canon, grid, s); break;
    case 5: canon_k<5>(W, G, canon, grid, s); break;
    case 6: canon_k<6>(W, G, canon, grid, s); break;
    case 7: canon_k<7>(W, G, canon, grid, s); break;
    default: canon_k<8>(W, G, canon, grid, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_lut_live(const float4* x_canon, const float4* dq, int n, int K, float inv_r2, int G,
                            const uint16_t* canon, uint32_t* live, int num_sms, cudaStream_t s) {
  (void)n;
  cudaError_t e = cudaMemsetAsync(live, 0xFF, (size_t)G * G * G * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const int grid = num_sms * 8;
  switch (K) {
    case 1: live_k<1>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 2: live_k<2>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 3: live_k<3>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 4: live_k<4>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 5: live_k<5>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 6: live_k<6>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    case 7: live_k<7>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
    default: live_k<8>(x_canon, dq, inv_r2, G, canon, live, grid, s); break;
  }
  return cudaGetLastError();
}

}  // namespace invr
