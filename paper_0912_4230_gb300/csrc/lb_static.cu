// FP64 mass and solute totals of caller-owned FP32 populations, computed
// without allocating any device memory.
//
// lb_reduce sums a context's populations through per-block partial sums held
// in memory the context allocated. Callers that cannot allocate device memory
// at the point where they need the totals — for example code whose device
// memory is entirely reserved up front by a framework's pool, or a loop that
// must not pay the device-wide synchronisation of cudaMalloc/cudaFree — use
// lb_totals_noalloc instead: the same per-block kernel and fixed-order finish,
// with the partial sums kept in a fixed-size array that lives in the library
// image itself (allocated when the library is loaded on a device and held
// until the process exits).
#include <mutex>
#include <string>

#include "../../include/lb.h"
#include "lb_kernels.cuh"
#include "lb_ops.h"

namespace {

using namespace lbgb;


// Largest lattice accepted: 2^24 cells (256^3), i.e. 65536 blocks of 256
// cells. The array holds two partial sums per block and the two totals:
// (2 * 65536 + 2) doubles = 1 MiB + 16 bytes per device.
constexpr long long kMaxCells = 1LL << 24;
constexpr unsigned kMaxBlocks = unsigned(kMaxCells / BLOCK);
constexpr unsigned kScratchDoubles = 2 * kMaxBlocks + 2;

// Device storage of the partial sums. In host code this name is only a
// host-side stand-in for the symbol, never a device address: kernels receive
// the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) double g_totals_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// the message is read back by lb_last_error(NULL) on the calling thread
int set_error(int code, const std::string &msg) {
  set_noctx_error(msg.c_str());
  return code;
}

// Device address of the scratch array on the current device, looked up once
// per device.
int scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(LB_EUNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (e != cudaSuccess || !p)
      return set_error(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return LB_OK;
}

// Per-block FP64 sums of the fluid mass (sum of f over non-solid cells, from
// the f_q - w_q storage, every value widened to FP64 before it is added) and
// the solute (sum of h), with a byte mask for solid cells.
__global__ void __launch_bounds__(BLOCK) noalloc_totals_kernel(const float *f, const float *h,
                                                               const uint8_t *solid, unsigned N,
                                                               double *partials) {
  __shared__ double sh[BLOCK][2];
  const unsigned n = blockIdx.x * BLOCK + threadIdx.x;
  double m = 0.0, s = 0.0;
  if (n < N && !(solid && solid[n])) {
    for (int q = 0; q < Q; ++q) m += StoreF32::to_f(f[size_t(q) * N + n], q);
    if (h)
      for (int q = 0; q < Q; ++q) s += StoreF32::to_h(h[size_t(q) * N + n], q);
  }
  sh[threadIdx.x][0] = m;
  sh[threadIdx.x][1] = s;
  __syncthreads();
  for (int k = BLOCK / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      sh[threadIdx.x][0] += sh[threadIdx.x + k][0];
      sh[threadIdx.x][1] += sh[threadIdx.x + k][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * size_t(blockIdx.x)] = sh[0][0];
    partials[2 * size_t(blockIdx.x) + 1] = sh[0][1];
  }
}

}  // namespace

extern "C" int lb_totals_noalloc(const float *f, const float *h, const uint8_t *solid,
                                 int64_t n_cells, double *out, void *stream) {
  if (!f || !out) return set_error(LB_EINVAL, "f and out are required");
  if (n_cells <= 0) return set_error(LB_EINVAL, "n_cells must be positive");
  if (n_cells > kMaxCells)
    return set_error(LB_EINVAL, "n_cells above the 16777216-cell limit of lb_totals_noalloc");
  double *scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != LB_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned N = unsigned(n_cells);
  const unsigned nblk = (N + BLOCK - 1) / BLOCK;
  // every block overwrites its own two partials and the finish overwrites the
  // totals, so nothing has to be cleared between calls
  noalloc_totals_kernel<<<nblk, BLOCK, 0, s>>>(f, h, solid, N, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    finish_sum_kernel<2><<<1, FINISH_THREADS, 0, s>>>(scratch, nblk, scratch + 2 * kMaxBlocks);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + 2 * kMaxBlocks, 2 * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(LB_ECUDA, std::string("lb_totals_noalloc: ") + cudaGetErrorString(e));
  return LB_OK;
}
