// lbm_field_mass_noalloc: the FP64 per-component mass reduction for callers
// that cannot allocate device memory. Its scratch (one partial sum per block
// and component) lives in a file-scope __device__ array instead of a
// caller-provided workspace; see include/lbm.h for the contract.
#include <mutex>

#include "lbm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;
constexpr int64_t NA_BLOCK_NODES = (int64_t)NA_THREADS * NA_PER_THREAD;  // 4096 nodes per block
constexpr int NA_MAX_BLOCKS = 16384;                                     // 2 x 16384 doubles = 256 KiB
constexpr int64_t NA_MAX_NODES = NA_BLOCK_NODES * NA_MAX_BLOCKS;         // 67,108,864 = 8192^2
constexpr int NA_MAX_DEVICES = 64;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) double g_mass_partials[2 * NA_MAX_BLOCKS];

// Device address of g_mass_partials per device, looked up once.
std::mutex g_lock;
double* g_addr[NA_MAX_DEVICES] = {};

// Block b sums the fluid nodes of [b * 4096, (b + 1) * 4096) in a fixed
// order: each thread its 16 nodes (stride 256), then a shuffle tree per
// warp, then the 8 warp sums in warp order.
__global__ void __launch_bounds__(NA_THREADS)
    k_field_mass_partial(const double* __restrict__ rA, const double* __restrict__ rB,
                         const uint8_t* __restrict__ mask, int64_t n, double* __restrict__ partial) {
  __shared__ double red[2][NA_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * NA_BLOCK_NODES;
  double a = 0.0, b = 0.0;
  for (int j = 0; j < NA_PER_THREAD; ++j) {
    const int64_t k = base + (int64_t)j * NA_THREADS + threadIdx.x;
    if (k < n && (mask == nullptr || mask[k] == 0)) {
      a += rA[k];
      b += rB[k];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    partial[2 * blockIdx.x] = sa;
    partial[2 * blockIdx.x + 1] = sb;
  }
}

// One warp per component adds the partials of this call in a fixed order.
__global__ void k_field_mass_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  const int s = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (s >= 2) return;
  double v = 0.0;
  for (int blk = lane; blk < nblocks; blk += 32) v += partial[2 * blk + s];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[s] = v;
}

// Set-up, once per device with that device current: the host-side name of a
// __device__ array is not a device address, so ask the runtime for it.
lbm_status partials_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || p == nullptr) return LBM_ERR_CUDA;
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_field_mass_noalloc(const double* d_rhoA, const double* d_rhoB, const uint8_t* d_mask,
                                             int32_t nx, int32_t ny, double* d_out, void* cuda_stream) {
  if (!d_rhoA || !d_rhoB || !d_out || nx < 1 || ny < 1) return LBM_ERR_ARG;
  const int64_t n = (int64_t)nx * ny;
  if (n > NA_MAX_NODES) return LBM_ERR_ARG;  // more blocks than the static scratch holds
  double* partial = nullptr;
  lbm_status s = partials_address(&partial);
  if (s) return s;
  const int nblocks = (int)((n + NA_BLOCK_NODES - 1) / NA_BLOCK_NODES);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_field_mass_partial<<<nblocks, NA_THREADS, 0, st>>>(d_rhoA, d_rhoB, d_mask, n, partial);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  k_field_mass_final<<<1, 64, 0, st>>>(partial, nblocks, d_out);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}
