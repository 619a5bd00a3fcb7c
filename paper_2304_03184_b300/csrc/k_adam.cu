// Fused Adam over a field's parameters (hash tables then MLP weights, one contiguous
// buffer): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr m_hat / (sqrt(v_hat) + eps),
// with bias corrections from the device step counter, and the gradient zeroed for the next
// step.  Every parameter is updated every step (dense Adam).
//
// Bound: HBM streaming, 7 x 4 B per parameter (read p, g, m, v; write p, m, v) plus the
// gradient clear (4 B), float4-vectorised, grid sized to the SM count.
#include <algorithm>

#include "invr_internal.cuh"

namespace invr {

__device__ __forceinline__ void adam1(float& p, float& g, float& m, float& v, float b1, float b2, float c1, float c2,
                                      float lr, float eps) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  const float mh = m / c1, vh = v / c2;
  p -= lr * mh / (sqrtf(vh) + eps);
  g = 0.0f;
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, int64_t n, const int64_t* __restrict__ step,
                                              float lr, float b1, float b2, float eps) {
  const float t = (float)(*step);
  const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
  const int64_t n4 = n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float4* p4 = reinterpret_cast<float4*>(p);
  float4* g4 = reinterpret_cast<float4*>(g);
  float4* m4 = reinterpret_cast<float4*>(m);
  float4* v4 = reinterpret_cast<float4*>(v);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 P = p4[i], G = g4[i], M = m4[i], V = v4[i];
    adam1(P.x, G.x, M.x, V.x, b1, b2, c1, c2, lr, eps);
    adam1(P.y, G.y, M.y, V.y, b1, b2, c1, c2, lr, eps);
    adam1(P.z, G.z, M.z, V.z, b1, b2, c1, c2, lr, eps);
    adam1(P.w, G.w, M.w, V.w, b1, b2, c1, c2, lr, eps);
    p4[i] = P;
    g4[i] = G;
    m4[i] = M;
    v4[i] = V;
  }
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    adam1(p[i], g[i], m[i], v[i], b1, b2, c1, c2, lr, eps);
}

__global__ void k_step_increment(int64_t* step) { *step += 1; }

cudaError_t launch_adam(float* params, const float* grads_in, float* grads_zero, float* m, float* v, int64_t n,
                        const int64_t* step_dev, float lr, float b1, float b2, float eps, cudaStream_t s) {
  (void)grads_in;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n4 = (n + 3) / 4;
  const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, (int64_t)sms * 8);
  if (n > 0) k_adam<<<blocks, 256, 0, s>>>(params, grads_zero, m, v, n, step_dev, lr, b1, b2, eps);
  return cudaGetLastError();
}

cudaError_t launch_step_increment(int64_t* step_dev, cudaStream_t s) {
  k_step_increment<<<1, 1, 0, s>>>(step_dev);
  return cudaGetLastError();
}

}  // namespace invr
