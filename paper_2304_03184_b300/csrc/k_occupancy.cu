// Density-driven maintenance of a view's 128^3 live-space occupancy bitfield: the density at
// every cell centre, evaluated through the view's warp, encoding and MLPs (the per-point
// kernels), updates an exponentially decaying maximum, and the bitfield marks the cells
// whose density exceeds a threshold.  The paper takes the occupied space as given; this
// keeps it current as the fields train and the poses change.
//
//   density[c] = max(decay * density[c], sigma(centre_c)),  bit_c = density[c] > threshold
//
// Cell c = x + 128 (y + 128 z), centre (i + 1/2) 2/128 - 1 per axis; bit c & 31 of word c >> 5.
// Bound: the point queries (2 M cells); the update itself streams 12 B per cell.
#include "invr_internal.cuh"

namespace invr {

__global__ void __launch_bounds__(256) k_occ_centres(float* __restrict__ p, int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int ijk[3] = {(int)(c % kOccRes), (int)((c / kOccRes) % kOccRes), (int)(c / (kOccRes * kOccRes))};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    p[a * n + c] = __fsub_rn(__fmul_rn(__fadd_rn((float)ijk[a], 0.5f), 2.0f / kOccRes), 1.0f);
}

// One thread per cell; a warp covers the 32 cells of one bitfield word.
__global__ void __launch_bounds__(256) k_occ_update(const float* __restrict__ sigma, int64_t n, float decay,
                                                    float threshold, float* density, uint32_t* bits) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool on = false;
  if (c < n) {
    const float d = fmaxf(__fmul_rn(decay, density[c]), __ldg(sigma + c));
    density[c] = d;
    on = d > threshold;
  }
  const unsigned word = __ballot_sync(0xffffffffu, on);
  if ((threadIdx.x & 31) == 0 && c < n) bits[c >> 5] = word;
}

cudaError_t launch_occ_centres(float* p, int64_t n, cudaStream_t s) {
  k_occ_centres<<<ceil_div(n, 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_occ_update(const float* sigma, int64_t n, float decay, float threshold, float* density,
                              uint32_t* bits, cudaStream_t s) {
  k_occ_update<<<ceil_div(n, 256), 256, 0, s>>>(sigma, n, decay, threshold, density, bits);
  return cudaGetLastError();
}

}  // namespace invr
