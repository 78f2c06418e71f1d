// Tiled single-pass step with the tile's inputs staged by the Tensor Memory
// Accelerator (TMA): FP32 storage, the same per-tile lists, node arithmetic
// and results (bit for bit) as k_tile.
//
// k_tile pulls every population of every listed node with its own load and
// waits for them (list entry -> pulls -> update is a chain of dependent
// global round trips per node). Here persistent CTAs (TMA_MINB per SM) walk
// a work list of the tiles that own fluid nodes (items blockIdx.x,
// + gridDim.x, ...) and, while a CTA updates one tile, the TMA copies its
// next tile's inputs into the other stage of a ring of TMA_NBUF buffers: the
// nine population planes and the density plane over the (TILE_W + 4) x
// (TILE_H + 4) window that the tile and its one-node ring pull from (nine
// 3-D boxes and one 2-D box) and the tile's list entries (one 1-D bulk copy;
// the lists are padded to 16-byte boundaries). No per-node address
// arithmetic for the loads, no registers held by loads in flight, no
// dependent global load before a tile's update. An mbarrier per buffer
// counts the bytes in; the wait on it is bounded (TMA_WAIT_NS). One thread
// per region slot; f*(t+1) is written over the consumed window. Stores, the
// ring, phase 2 and the periodic images are those of k_tile.
#pragma once

#include <cuda.h>  // CUtensorMap

#include "lbm_tiled.cuh"

namespace lbm {

constexpr int TMA_WW = TILE_W + 4;                  // window columns (pairs): x0 - 2 ... x0 + TILE_W + 1
constexpr int TMA_WH = TILE_H + 4;                  // window rows
constexpr int TMA_BOX_X = 2 * TMA_WW;               // floats per window row (component pairs)
constexpr int TMA_PLANE_BYTES = TMA_BOX_X * TMA_WH * 4;
constexpr int TMA_SLOT_BYTES = (TMA_PLANE_BYTES + 127) / 128 * 128;  // 128-byte aligned destinations
constexpr int TMA_ENTRY_BYTES = (TILE_RS + 7) / 8 * 16;  // a tile's list, padded to 8 entries
// nine population planes, the density plane and the entries, 128-byte aligned
constexpr int TMA_BUF_BYTES = (10 * TMA_SLOT_BYTES + TMA_ENTRY_BYTES + 127) / 128 * 128;
#ifndef LBM_TMA_THREADS
#define LBM_TMA_THREADS 0  // 0: one thread per region slot, rounded up to a warp
#endif
#ifndef LBM_TMA_NBUF
#define LBM_TMA_NBUF 2
#endif
#ifndef LBM_TMA_MINB
#define LBM_TMA_MINB 2
#endif
constexpr int TMA_THREADS = LBM_TMA_THREADS > 0 ? LBM_TMA_THREADS : (TILE_RS + 31) / 32 * 32;
constexpr int TMA_NBUF = LBM_TMA_NBUF;  // copy stages per CTA (tiles in flight: NBUF - 1 ahead)
constexpr int TMA_MINB = LBM_TMA_MINB;  // CTAs per SM (registers and shared memory must allow it)
// One node per thread, and f*(t+1) of the region written over the consumed
// window: the schedule exists for tile shapes whose region fits both (else
// LBM_KERNEL_TMA runs the tiled schedule).
constexpr bool TMA_AVAILABLE = TILE_RS <= TMA_THREADS && 9 * TILE_RS * 8 <= 10 * TMA_SLOT_BYTES;
// Nanoseconds (of the global timer) a CTA waits for a tile's copies before
// it gives up and reports them: far above any copy's latency, short enough
// to return control to the host within about a second.
constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;
static_assert(TMA_BOX_X <= 256 && TMA_WH <= 256, "TMA box dimensions are at most 256");
static_assert((TMA_BOX_X * 4) % 16 == 0, "the box's inner extent must be a multiple of 16 bytes");
static_assert(TILE_W % 2 == 0, "window x starts must be 16-byte aligned: 4 * 2 * (x0 - 2 + LP) % 16 == 0");

template <typename T>
constexpr size_t tma_smem() {
  return TMA_NBUF * (size_t)TMA_BUF_BYTES + 128;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase with the given parity to complete; false once
// TMA_WAIT_NS have passed (the timer is read every 256 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (unsigned long long r = 0;; ++r) {  // 64-bit: never wraps to 0
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((r & 255ull) == 0) {
      const unsigned long long t = global_ns();
      if (r == 0)
        t0 = t;
      else if (t - t0 > TMA_WAIT_NS)
        return false;
    }
  }
}

// One TMA box of a rank-3 tensor (x, y, plane) into shared memory, counted
// on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// A contiguous 16-byte-aligned run of global memory into shared memory,
// counted on bar (bytes: a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The TMA schedule's work list: the tiles with owned nodes in tile order,
// as (tile, first entry, listed nodes, owned nodes), and their number in
// *n_work. One CTA of 1024 threads, fixed-order scan (deterministic).
static __global__ void __launch_bounds__(1024)
    k_tile_work(const int2* __restrict__ cnt, const int* __restrict__ offsets, int n_tiles, int4* __restrict__ work,
                int* __restrict__ n_work) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n_tiles; base += 1024) {
    const int t = base + threadIdx.x;
    const int2 c = t < n_tiles ? cnt[t] : make_int2(0, 0);
    const bool keep = c.x > 0;
    const unsigned ball = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_sums[wid] = __popc(ball);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      before += w < wid ? warp_sums[w] : 0;
      all += warp_sums[w];
    }
    if (keep) work[carry + before + __popc(ball & ((1u << lane) - 1u))] = make_int4(t, offsets[t], c.y, c.x);
    __syncthreads();
    if (threadIdx.x == 0) carry += all;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_work = carry;
}

// Issue the copies of work item w (tile's window and entries) into buffer
// `buf` (one thread).
// extra_tx: bytes the barrier expects beyond what the copies deliver (0;
// the test of the bounded wait sets it so that the wait runs out).
__device__ __forceinline__ void tma_issue(unsigned char* buf, uint64_t* bar, const CUtensorMap* mapf,
                                          const CUtensorMap* mapP, const uint16_t* __restrict__ entries, int4 w,
                                          int ntx, uint32_t extra_tx) {
  const int tile = w.x;
  const int x0 = (tile % ntx) * TILE_W, y0 = (tile / ntx) * TILE_H;
  // padded coordinates of the window's first pair: column x0 - 2 + LP (its
  // first float, times 4 bytes, is 16-byte aligned: TILE_W is even), row
  // y0 - 2 + GH
  const int xf = 2 * (x0 - 2 + LP), yw = y0 - 2 + GH;
  const uint32_t ebytes = (uint32_t)((w.z + 7) & ~7) * 2;  // the list, padded to 16 bytes
  // order the generic-proxy reads of this buffer (three tiles back) before
  // the copies' writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, 10u * TMA_PLANE_BYTES + ebytes + extra_tx);
#pragma unroll
  for (int i = 0; i < 9; ++i) tma_load_3d(buf + i * TMA_SLOT_BYTES, mapf, xf, yw, i, bar);
  tma_load_2d(buf + 9 * TMA_SLOT_BYTES, mapP, xf, yw, bar);
  bulk_load(buf + 10 * TMA_SLOT_BYTES, entries + w.y, ebytes, bar);
}


// Persistent CTAs walk the work list with a stride of the grid, TMA_MINB per
// SM; the copies of each CTA's next TMA_NBUF - 1 tiles are in flight while it
// updates the current one. One thread per listed node (TILE_RS <= threads):
// phase 1 reads the window and keeps f*(t+1) in registers, the CTA waits for
// every read of the window, writes f*(t+1) over it ([9][TILE_RS] pairs at
// the buffer's start; the entry list after the planes stays), waits again,
// and phase 2 sums rho(t+1) of the owned nodes from there.
// err: set to 1 when a copy was not seen to complete within the bound (the
// CTA then stops). The host reads it at its next synchronising call.
// extra_tx: see tma_issue (0 in operation).
static __global__ void __launch_bounds__(TMA_THREADS, TMA_MINB)
    k_tile_tma(const __grid_constant__ CUtensorMap mapf, const __grid_constant__ CUtensorMap mapP,
               float* __restrict__ fo, float* __restrict__ Po, const uint16_t* __restrict__ flags,
               const uint16_t* __restrict__ entries, const int4* __restrict__ work, int n_work, Geo g, int ntx,
               PhysK<float> ph, int* __restrict__ err, uint32_t extra_tx) {
  if constexpr (!TMA_AVAILABLE) {
    return;  // never launched (the host runs the tiled schedule instead)
  } else {
  using V = float2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t bar[TMA_NBUF];
  const float zr[2][9] = {};  // storage references: zero for 4-byte populations
  const int G = gridDim.x;
  int4 wnext = make_int4(-1, 0, 0, 0);  // thread 0: the work item TMA_NBUF - 1 ahead of the current one
  if (threadIdx.x == 0) {
    for (int b = 0; b < TMA_NBUF; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < TMA_NBUF - 1; ++k) {
      const int wk = blockIdx.x + k * G;
      if (wk < n_work)
        tma_issue(base + k * TMA_BUF_BYTES, &bar[k], &mapf, &mapP, entries, __ldg(work + wk), ntx, extra_tx);
    }
    const int w2 = blockIdx.x + (TMA_NBUF - 1) * G;
    if (w2 < n_work) wnext = __ldg(work + w2);
  }
  __syncthreads();
  const int t = threadIdx.x;
  for (int n = 0;; ++n) {
    const int wn = blockIdx.x + n * G;
    if (wn >= n_work) break;
    const int cur = n % TMA_NBUF;
    unsigned char* buf = base + cur * TMA_BUF_BYTES;
    if (t == 0) {
      // the item TMA_NBUF - 1 ahead into the buffer the previous iteration
      // freed (its closing barrier)
      const int wa = wn + (TMA_NBUF - 1) * G;
      if (wa < n_work) {
        const int ba = (n + TMA_NBUF - 1) % TMA_NBUF;
        tma_issue(base + ba * TMA_BUF_BYTES, &bar[ba], &mapf, &mapP, entries, wnext, ntx, extra_tx);
        if (wa + G < n_work) wnext = __ldg(work + wa + G);
      }
    }
    const int4 item = __ldg(work + wn);  // (tile, first entry, listed nodes, owned nodes)
    const bool ok = mbar_wait(&bar[cur], (uint32_t)((n / TMA_NBUF) & 1));
    if (__syncthreads_or(!ok)) {
      // a copy did not complete within the bound: report it and stop this
      // CTA after waiting (bounded) for the copies it has in flight
      if (t == 0) {
        atomicExch(err, 1);
        for (int k = n; k < n + TMA_NBUF; ++k)
          if (blockIdx.x + k * G < n_work) mbar_wait(&bar[k % TMA_NBUF], (uint32_t)((k / TMA_NBUF) & 1));
      }
      break;
    }
    const float* win = reinterpret_cast<const float*>(buf);
    const uint16_t* ent = reinterpret_cast<const uint16_t*>(buf + 10 * TMA_SLOT_BYTES);
    const int tile = item.x, n_all = item.z, n_own = item.w;
    const int x0 = (tile % ntx) * TILE_W, y0 = (tile / ntx) * TILE_H;
    const int korg = g.idx(x0 - 1, y0 - 1);  // padded index of region slot 0
    const bool valid = t < n_all;
    const uint16_t e = valid ? ent[t] : uint16_t(0);
    const bool warp_edge = __any_sync(0xffffffffu, (e & TE_SOLIDNB) != 0);
    const bool warp_border = __any_sync(0xffffffffu, (e & TE_BORDER) != 0);
    const int slot = e & TE_SLOT;
    const int row = slot / TILE_RW, col = slot - row * TILE_RW;
    const int k = korg + row * g.px + col;
    float fv[2][9];
    if (valid) {
      const uint16_t fl = warp_edge ? __ldg(flags + k) : uint16_t(0);
      // region slot (row, col) is window pair (row + 1, col + 1)
      const int wc = (row + 1) * TMA_BOX_X + 2 * (col + 1);
      float nbP[2][9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const V v = *reinterpret_cast<const V*>(win + i * (TMA_SLOT_BYTES / 4) + wc - cy_of(i) * TMA_BOX_X -
                                                2 * cx_of(i));
        fv[0][i] = v.x;
        fv[1][i] = v.y;
      }
      nbP[0][0] = nbP[1][0] = 0.0f;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const V v = *reinterpret_cast<const V*>(win + 9 * (TMA_SLOT_BYTES / 4) + wc + cy_of(i) * TMA_BOX_X +
                                                2 * cx_of(i));
        nbP[0][i] = v.x;
        nbP[1][i] = v.y;
      }
      float rho[2], u[2];
      march_update<float>(fv, nbP, fl, warp_edge, ph, rho, u);
      if (t < n_own) {
        if (!warp_border) {
#pragma unroll
          for (int i = 0; i < 9; ++i) Pop<float>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], 0.0f, 0.0f);
          if (warp_edge) store_bounced_near(fo, g, k, fl, fv, zr);
        } else {
          const int x = x0 - 1 + col, y = y0 - 1 + row;
          store_node(fo, g, x, y, k, fv, zr);
          store_bounced(fo, g, x, y, fl, fv, zr);
        }
      }
    }
    __syncthreads();  // every read of the window is done: f*(t+1) goes over it
    V* s = reinterpret_cast<V*>(buf);
    if (valid) {
#pragma unroll
      for (int i = 0; i < 9; ++i) s[i * TILE_RS + slot] = make_float2(fv[0][i], fv[1][i]);
    }
    __syncthreads();
    if (t < n_own) {
      const uint16_t fl = (e & TE_SOLIDNB) ? __ldg(flags + k) : uint16_t(0);
      float fn[2][9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const bool bounce = i != 0 && (fl & nb_bit(opp_of(i)));
        const V v = bounce ? s[opp_of(i) * TILE_RS + slot] : s[i * TILE_RS + slot - cx_of(i) - cy_of(i) * TILE_RW];
        fn[0][i] = v.x;
        fn[1][i] = v.y;
      }
      const float r0 = density(fn[0]), r1 = density(fn[1]);
      stP(Po, k, r0, r1);
      if (e & TE_BORDER) {
        const int x = x0 - 1 + col, y = y0 - 1 + row;
        for_ghost_images(g, x, y, [&](int kk) { stP(Po, kk, r0, r1); });
      }
    }
    // this thread's generic accesses to the buffer before the copies that
    // will overwrite it (issued after the barrier)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();  // the buffer is free
  }
  }
}

}  // namespace lbm
