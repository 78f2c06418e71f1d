// Geometry set-up kernels: per-node flags from the caller's mask (with
// periodic wrap or solid ghosts) and the deterministic compaction of the
// interface-solid list (solid nodes with a fluid D2Q9 neighbour, identified
// once per geometry, Sec. 3.2 of arXiv:2009.12584).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

// Solidity of logical node (x, y), which may lie outside the owned range.
__device__ __forceinline__ bool solid_at(const uint8_t* __restrict__ mask, const Geo& g, int x, int y) {
  if (x < 0 || x >= g.nx) {
    if (!g.per_x) return true;
    x = (x % g.nx + g.nx) % g.nx;
  }
  if (y < 0 || y >= g.ny) {
    if (!g.per_y) return true;
    y = (y % g.ny + g.ny) % g.ny;
  }
  return mask[(int64_t)y * g.nx + x] != 0;
}

// One thread per padded cell. Cells of the ghost layers get the flags of
// the node they image (periodic axes) or solid (walled axes), neighbour and
// interface bits included, because the single-pass kernel recomputes
// densities there. Padding beyond the ghost layers is solid. err[0] counts
// fluid nodes on a walled border.
static __global__ void k_flags(const uint8_t* __restrict__ mask, uint16_t* __restrict__ flags, Geo g,
                        int* __restrict__ err) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y;
  if (px >= g.px) return;
  const int x = px - LP, y = py - GH;
  const bool owned = x >= 0 && x < g.nx && y >= 0 && y < g.ny;
  const bool in_halo = x >= -GH && x < g.nx + GH;
  uint16_t fl = 0;
  if (!in_halo || solid_at(mask, g, x, y)) fl |= F_SOLID;
  if (in_halo) {
    bool any_fluid_nb = false;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      if (solid_at(mask, g, x + cx_of(i), y + cy_of(i))) {
        fl |= nb_bit(i);
      } else {
        any_fluid_nb = true;
      }
    }
    if ((fl & F_SOLID) && any_fluid_nb) fl |= F_IFACE;
    if (owned && !(fl & F_SOLID)) {
      const bool on_wall = (!g.per_x && (x == 0 || x == g.nx - 1)) || (!g.per_y && (y == 0 || y == g.ny - 1));
      if (on_wall) atomicAdd(err, 1);
    }
  }
  flags[(int64_t)py * g.px + px] = fl;
}

constexpr int SCAN_BLOCK = 256;

// Node classes compacted into index lists at set-up (padded indices, node
// order). IFACE: interface-solid nodes (Eq. 8 is evaluated there). FLUID:
// every fluid node, its entry tagged in the two top bits. BORDER_TAG: the
// node lies within GH + 1 of a periodic border, so that it or one of its
// D2Q9 neighbours has periodic images in the ghost layers. EDGE_TAG: the
// node has a solid neighbour or carries BORDER_TAG. A "bulk" node has
// neither tag. Node order is kept so that neighbouring nodes are updated
// together and every 32-byte sector is read and written whole. Padded
// indices stay below 2^30, which leaves the two top bits free.
enum { CLS_IFACE = 0, CLS_FLUID = 1 };
constexpr unsigned EDGE_TAG = 0x80000000u;
constexpr unsigned BORDER_TAG = 0x40000000u;
constexpr unsigned LIST_TAGS = EDGE_TAG | BORDER_TAG;

__device__ __forceinline__ bool near_border(const Geo& g, int x, int y) {
  return (g.per_x && (x <= GH || x >= g.nx - GH - 1)) || (g.per_y && (y <= GH || y >= g.ny - GH - 1));
}

__device__ __forceinline__ bool in_class(const uint16_t* __restrict__ flags, const Geo& g, int64_t n, int cls,
                                         int* k_out) {
  const int x = (int)(n % g.nx), y = (int)(n / g.nx);
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  if (cls == CLS_IFACE) {
    *k_out = k;
    return fl & F_IFACE;
  }
  const bool border = near_border(g, x, y);
  const bool edge = (fl & NB_ANY) || border;
  *k_out = (int)((unsigned)k | (edge ? EDGE_TAG : 0u) | (border ? BORDER_TAG : 0u));
  return !(fl & F_SOLID);
}

// Pass 1: nodes of class cls per block of SCAN_BLOCK owned nodes.
static __global__ void __launch_bounds__(SCAN_BLOCK) k_class_count(const uint16_t* __restrict__ flags, Geo g, int cls,
                                                            int* __restrict__ counts) {
  const int64_t n = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  const int64_t N = (int64_t)g.nx * g.ny;
  int k;
  const bool hit = n < N && in_class(flags, g, n, cls, &k);
  const int c = __syncthreads_count(hit);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Pass 2: exclusive scan of the per-block counts in one block (fixed order).
static __global__ void __launch_bounds__(1024) k_iface_scan(int* __restrict__ counts, int nblocks,
                                                     int* __restrict__ total) {
  __shared__ int carry;
  __shared__ int warp_sums[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nblocks ? counts[i] : 0;
    int x = v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const int incl = x + (wid ? warp_sums[wid - 1] : 0);
    if (i < nblocks) counts[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Pass 3: write the padded indices of the nodes of class cls in node order,
// starting at list[*base] (base may be null: start at 0).
static __global__ void __launch_bounds__(SCAN_BLOCK) k_class_write(const uint16_t* __restrict__ flags, Geo g, int cls,
                                                            const int* __restrict__ offsets,
                                                            const int* __restrict__ base, int capacity,
                                                            int* __restrict__ list) {
  __shared__ int warp_base[SCAN_BLOCK / 32];
  const int64_t n = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  const int64_t N = (int64_t)g.nx * g.ny;
  int k = 0;
  const bool hit = n < N && in_class(flags, g, n, cls, &k);
  const unsigned ball = __ballot_sync(0xffffffffu, hit);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_base[wid] = __popc(ball);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < SCAN_BLOCK / 32; ++w) {
      const int c = warp_base[w];
      warp_base[w] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (hit) {
    const int pos = (base ? *base : 0) + offsets[blockIdx.x] + warp_base[wid] + __popc(ball & ((1u << lane) - 1u));
    if (pos < capacity) list[pos] = k;
  }
}

// Fluid neighbours of each interface-solid cell within its 5 x 5 stencil:
// bit (dy + 2) * 5 + (dx + 2) is set when node (x + dx, y + dy) is fluid.
// Computed once per geometry; Eq. 8 then loads only the densities of fluid
// neighbours (both the D2Q25 and the D2Q9 average read this mask).
static __global__ void __launch_bounds__(128) k_iface_mask(const uint16_t* __restrict__ flags,
                                                           const int* __restrict__ list, int n, Geo g,
                                                           uint32_t* __restrict__ mask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = list[t];
  uint32_t m = 0;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      if (dx == 0 && dy == 0) continue;
      if (!(flags[k + dx + dy * g.px] & F_SOLID)) m |= 1u << ((dy + 2) * 5 + (dx + 2));
    }
  mask[t] = m;
}

}  // namespace lbm
