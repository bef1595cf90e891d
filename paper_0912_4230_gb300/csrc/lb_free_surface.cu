// Free-surface set-up and totals (Section 3): initial cell types, liquid
// mass and liquid fraction; FP64 sum of the liquid mass; mass export.
#include "lb_kernels.cuh"
#include "lb_ops.h"

namespace lbgb {

namespace {

// flowchart step b: liquid m = rho0, interface m = lambda0 rho0 (lambda0 = 1/2
// when not given), empty m = 0; solid cells are typed empty and never updated
template <class Real>
__global__ void fs_init_kernel(unsigned N, const uint32_t *link, const uint8_t *type_in,
                               const float *rho0, const float *lambda0, uint8_t *type0,
                               uint8_t *type1, Real *mass, Real *lam) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n >= N) return;
  uint8_t t = type_in[n];
  Real l = Real(0);
  if (link[n] >> 31) {
    t = CELL_EMPTY;
  } else if (t == CELL_LIQUID) {
    l = Real(1);
  } else if (t == CELL_INTERFACE) {
    l = lambda0 ? Real(lambda0[n]) : Real(0.5);
  } else {
    t = CELL_EMPTY;
  }
  type0[n] = t;
  type1[n] = t;
  lam[n] = l;
  mass[n] = (link[n] >> 31) ? Real(0) : l * Real(rho0[n]);
}

template <class Real>
__global__ void __launch_bounds__(BLOCK) fs_totals_kernel(unsigned N, const uint32_t *link,
                                                          const Real *mass, double *partials) {
  __shared__ double sh[BLOCK];
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  sh[threadIdx.x] = (n < N && !(link[n] >> 31)) ? double(mass[n]) : 0.0;
  __syncthreads();
  for (int k = BLOCK / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * size_t(blockIdx.x)] = sh[0];
    partials[2 * size_t(blockIdx.x) + 1] = 0.0;
  }
}

template <class Real>
__global__ void to_double_kernel(unsigned N, const Real *src, double *dst) {
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  if (n < N) dst[n] = double(src[n]);
}

unsigned blocks_for(unsigned N) { return (N + BLOCK - 1) / BLOCK; }

}  // namespace

cudaError_t fs_init(unsigned N, const uint32_t *link, const uint8_t *type_in, const float *rho0,
                    const float *lambda0, uint8_t *type0, uint8_t *type1, void *mass, void *lam,
                    bool fp64, cudaStream_t s) {
  if (fp64)
    fs_init_kernel<double><<<blocks_for(N), BLOCK, 0, s>>>(N, link, type_in, rho0, lambda0, type0,
                                                           type1, static_cast<double *>(mass),
                                                           static_cast<double *>(lam));
  else
    fs_init_kernel<float><<<blocks_for(N), BLOCK, 0, s>>>(N, link, type_in, rho0, lambda0, type0,
                                                          type1, static_cast<float *>(mass),
                                                          static_cast<float *>(lam));
  return cudaGetLastError();
}

cudaError_t fs_totals(unsigned N, const uint32_t *link, const void *mass, double *partials,
                      bool fp64, cudaStream_t s) {
  if (fp64)
    fs_totals_kernel<double><<<blocks_for(N), BLOCK, 0, s>>>(N, link,
                                                             static_cast<const double *>(mass),
                                                             partials);
  else
    fs_totals_kernel<float><<<blocks_for(N), BLOCK, 0, s>>>(N, link,
                                                            static_cast<const float *>(mass),
                                                            partials);
  return cudaGetLastError();
}

cudaError_t to_double(unsigned N, const void *src, double *dst, bool fp64, cudaStream_t s) {
  if (fp64)
    to_double_kernel<double><<<blocks_for(N), BLOCK, 0, s>>>(N, static_cast<const double *>(src), dst);
  else
    to_double_kernel<float><<<blocks_for(N), BLOCK, 0, s>>>(N, static_cast<const float *>(src), dst);
  return cudaGetLastError();
}

}  // namespace lbgb
