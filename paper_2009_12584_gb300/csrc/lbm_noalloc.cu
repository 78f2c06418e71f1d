// lbm_field_mass_noalloc: the FP64 per-component mass reduction for callers
// that cannot allocate device memory. Its scratch (one partial sum per block
// and component) lives in a file-scope __device__ array instead of a
// caller-provided workspace; see include/lbm.h for the contract.
#include <cuda.h>  // CUcontext; the two driver calls are resolved through the runtime, not linked

#include <mutex>

#include "lbm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;
constexpr int64_t NA_BLOCK_NODES = (int64_t)NA_THREADS * NA_PER_THREAD;  // 4096 nodes per block
constexpr int NA_MAX_BLOCKS = 16384;                                     // 2 x 16384 doubles = 256 KiB
constexpr int64_t NA_MAX_NODES = NA_BLOCK_NODES * NA_MAX_BLOCKS;         // 67,108,864 = 8192^2
constexpr int NA_MAX_CONTEXTS = 64;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) double g_mass_partials[2 * NA_MAX_BLOCKS];

// Device address of g_mass_partials per CUDA context, looked up once in
// each. Contexts are told apart by the driver's context identifier, which
// is unique for the life of the process: a context destroyed (for instance
// by cudaDeviceReset) and created again gets a new identifier and a new
// lookup, so no stale address is ever used.
struct AddrEntry {
  unsigned long long ctx_id;
  double* addr;
};
std::mutex g_lock;
AddrEntry g_addr[NA_MAX_CONTEXTS] = {};
int g_next = 0;
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

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

// Identifier of the calling thread's current context (0 if none is current
// yet). Call with g_lock held.
lbm_status current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&g_ctx_current, 12000, cudaEnableDefault,
                                         &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&g_ctx_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      g_ctx_current = nullptr;
      g_ctx_id = nullptr;
      return LBM_ERR_CUDA;
    }
  }
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) return LBM_ERR_CUDA;
  *id = 0;
  if (ctx && g_ctx_id(ctx, id) != CUDA_SUCCESS) return LBM_ERR_CUDA;
  return LBM_OK;
}

// Set-up, once per context (so once per device for the runtime's primary
// contexts), with that context current: the host-side name of a __device__
// array is not a device address, so ask the runtime for it.
lbm_status partials_address(double** out) {
  std::lock_guard<std::mutex> guard(g_lock);
  unsigned long long id = 0;
  lbm_status s = current_context_id(&id);
  if (s) return s;
  if (id != 0)
    for (const AddrEntry& e : g_addr)
      if (e.ctx_id == id && e.addr) {
        *out = e.addr;
        return LBM_OK;
      }
  // the lookup makes the device's primary context current if none was
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || p == nullptr) return LBM_ERR_CUDA;
  if (id == 0 && ((s = current_context_id(&id)) || id == 0)) return s ? s : LBM_ERR_CUDA;
  g_addr[g_next] = AddrEntry{id, (double*)p};
  g_next = (g_next + 1) % NA_MAX_CONTEXTS;
  *out = (double*)p;
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
  // an error left by earlier work is the caller's: report it without clearing it
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ERR_CUDA;
  k_field_mass_partial<<<nblocks, NA_THREADS, 0, st>>>(d_rhoA, d_rhoB, d_mask, n, partial);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  k_field_mass_final<<<1, 64, 0, st>>>(partial, nblocks, d_out);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}
