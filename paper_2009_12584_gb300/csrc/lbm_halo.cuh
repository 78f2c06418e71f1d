// Halo-tiled single-pass step: one kernel per time step and no density
// plane (4- and 8-byte storage).
//
// The step needs rho(t) at a fluid node's eight neighbours (Eq. 5) and,
// under the improved scheme, rho~(t) at its solid neighbours, which Eq. 8
// averages from rho(t) up to two nodes further out. Both are recomputed per
// tile from the populations themselves: one CTA takes a HALO_W x HALO_H
// tile and
//   phase A: pulls f_i(x) = f*_i(x - c_i, t) at every fluid node of the tile
//     and of the R rings around it (R = 3 for the D2Q25 average of Eq. 8,
//     2 for the D2Q9 average, 1 for the other schemes) and keeps
//     rho(t) = sum_i f_i (Eq. 3) in shared memory;
//   phase B (improved scheme only): evaluates Eq. 8 at the interface-solid
//     cells of the tile and its first ring from those densities;
//   phase C: each fluid node of the tile pulls its populations again (now
//     L1/L2 hits), takes rho or rho~ of its neighbours from shared memory,
//     evaluates Eqs. 5 and 7, u of Eq. 3 and the collision (Eqs. 1, 2, 4),
//     and stores f*(t+1) (with bounced slots and periodic images).
// The ring nodes cost nine pulls and a sum each, not a collision; the
// populations cross HBM once per step. Every value is computed with the
// arithmetic, in the order, of the two-pass schedule, so the schedules agree
// bit for bit.
//
// Fluid nodes are listed per tile at set-up: the tile's own nodes first, then
// the rings by distance, each in row order (16-bit entries: the slot in the
// (HALO_W + 2 HALO_R) x (HALO_H + 2 HALO_R) region and two tags). A per-tile
// bitmask of the region's fluid slots gives phase B the fluid neighbours of
// each solid cell.
#pragma once

#include "lbm.h"
#include "lbm_common.cuh"
#include "lbm_fused.cuh"
#include "lbm_geometry.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

#ifndef LBM_HALO_W
#define LBM_HALO_W 32
#endif
#ifndef LBM_HALO_H
#define LBM_HALO_H 14
#endif
// 128-thread CTAs, 8 per SM: on the 8192^2 porous medium 2.09 ms per step
// against 2.34 ms with 256 threads at 4 per SM (improved scheme; Martys-Chen
// 1.59 against 1.68 ms)
#ifndef LBM_HALO_THREADS
#define LBM_HALO_THREADS 128
#endif
#ifndef LBM_HALO_MINB
#define LBM_HALO_MINB 8
#endif
#ifndef LBM_HALO_AHEAD
#define LBM_HALO_AHEAD 512
#endif
constexpr int HALO_R = 3;  // widest halo: Eq. 8's D2Q25 reach (2) plus the force's (1)
constexpr int HALO_W = LBM_HALO_W, HALO_H = LBM_HALO_H;  // owned nodes per tile
constexpr int HALO_RW = HALO_W + 2 * HALO_R;  // region pitch
constexpr int HALO_RH = HALO_H + 2 * HALO_R;
constexpr int HALO_RS = HALO_RW * HALO_RH;    // region slots
constexpr int HALO_MW = (HALO_RS + 31) / 32;  // words of a tile's fluid bitmask
constexpr int HALO_THREADS = LBM_HALO_THREADS;
constexpr int HALO_MINB = LBM_HALO_MINB;      // CTAs per SM the registers must allow
constexpr int HALO_AHEAD = LBM_HALO_AHEAD;    // tiles between a CTA and the one whose entries it prefetches
constexpr int HALO_LIST_THREADS = 256;        // k_halo_lists
static_assert(HALO_RS <= 2048, "slots must fit the 11 slot bits of an entry");
static_assert(HALO_MW <= HALO_THREADS, "one thread per bitmask word");

constexpr uint16_t HE_SLOT = 0x07FFu;     // slot = row * HALO_RW + col in the region
constexpr uint16_t HE_SOLIDNB = 0x2000u;  // own node with a solid D2Q9 neighbour
constexpr uint16_t HE_BORDER = 0x4000u;   // own node within GH + 1 of a periodic border

inline int64_t halo_tile_count(const Geo& g) {
  return (int64_t)((g.nx + HALO_W - 1) / HALO_W) * ((g.ny + HALO_H - 1) / HALO_H);
}

// Rings a step needs for the installed wetting scheme.
inline int halo_reach(const Phys& ph) { return ph.bc == BC_VAVG ? (ph.avg9 ? 2 : 3) : 1; }

// Ring of region slot (col, row) of a tile with tw x th owned nodes: 0 for
// an owned slot, else its distance (max norm) from the owned rectangle; -1
// outside the region.
__device__ __forceinline__ int halo_ring(int col, int row, int tw, int th) {
  if (col > tw + 2 * HALO_R - 1 || row > th + 2 * HALO_R - 1) return -1;
  const int dc = col < HALO_R ? HALO_R - col : (col >= HALO_R + tw ? col - (HALO_R + tw - 1) : 0);
  const int dr = row < HALO_R ? HALO_R - row : (row >= HALO_R + th ? row - (HALO_R + th - 1) : 0);
  return max(dc, dr);
}

// Per-tile lists, two passes over the same deterministic order (four
// rounds: the owned nodes, then rings 1, 2, 3). Count pass (entries ==
// nullptr): totals[tile] = fluid nodes of the region, cnt[tile] = the
// cumulative counts after each round, fmask[tile] = the region's fluid
// bitmask. Write pass: the entries from offsets[tile] on.
static __global__ void __launch_bounds__(HALO_LIST_THREADS)
    k_halo_lists(const uint16_t* __restrict__ flags, Geo g, int ntx, const int* __restrict__ offsets,
                 int* __restrict__ totals, int4* __restrict__ cnt, uint32_t* __restrict__ fmask,
                 uint16_t* __restrict__ entries) {
  __shared__ int warp_cnt[HALO_LIST_THREADS / 32];
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * HALO_W, y0 = (tile / ntx) * HALO_H;
  const int tw = min(HALO_W, g.nx - x0), th = min(HALO_H, g.ny - y0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int base = 0;
  int cum[4];
  for (int round = 0; round < 4; ++round) {
    for (int c0 = 0; c0 < HALO_RS; c0 += HALO_LIST_THREADS) {
      const int slot = c0 + threadIdx.x;
      const int row = slot / HALO_RW, col = slot - row * HALO_RW;
      const int ring = slot < HALO_RS ? halo_ring(col, row, tw, th) : -1;
      bool fluid = false;
      uint16_t e = 0;
      if (ring >= 0) {
        const int x = x0 - HALO_R + col, y = y0 - HALO_R + row;
        const uint16_t fl = flags[g.idx(x, y)];
        fluid = !(fl & F_SOLID);
        e = (uint16_t)slot;
        if (ring == 0 && (fl & NB_ANY)) e |= HE_SOLIDNB;
        if (ring == 0 && near_border(g, x, y)) e |= HE_BORDER;
      }
      if (round == 0 && !entries) {
        const unsigned bits = __ballot_sync(0xffffffffu, fluid);
        const int word = (c0 >> 5) + wid;
        if (lane == 0 && word < HALO_MW) fmask[(int64_t)tile * HALO_MW + word] = bits;
      }
      const bool hit = fluid && ring == round;
      const unsigned ball = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) warp_cnt[wid] = __popc(ball);
      __syncthreads();
      int before = 0, all = 0;
      for (int w = 0; w < HALO_LIST_THREADS / 32; ++w) {
        const int v = warp_cnt[w];
        before += w < wid ? v : 0;
        all += v;
      }
      if (entries && hit) entries[offsets[tile] + base + before + __popc(ball & ((1u << lane) - 1u))] = e;
      base += all;
      __syncthreads();
    }
    cum[round] = base;
  }
  if (!entries && threadIdx.x == 0) {
    totals[tile] = base;
    cnt[tile] = make_int4(cum[0], cum[1], cum[2], cum[3]);
  }
}

// One CTA per tile. reach: the rings phase A covers (halo_reach).
template <typename T>
__global__ void __launch_bounds__(HALO_THREADS, HALO_MINB)
    k_halo(const T* __restrict__ f, T* __restrict__ fo, const uint16_t* __restrict__ flags,
           const uint16_t* __restrict__ entries, const int* __restrict__ offsets, const int4* __restrict__ cnt,
           const uint32_t* __restrict__ fmask, Geo g, int ntx, int reach, PhysK<typename Pop<T>::C> ph) {
  using C = typename Pop<T>::C;
  using V = typename CPair<C>::V;
  static_assert(!kDev<T>, "the halo schedule stores 4- and 8-byte populations");
  __shared__ V rho[HALO_RS];       // rho(t) at fluid slots, rho~(t) at interface-solid slots
  __shared__ uint32_t fm[HALO_MW];  // fluid slots of the region
  const int tile = blockIdx.x;
  const int4 cn = cnt[tile];
  const int n_own = cn.x;
  if (n_own == 0) return;  // the whole CTA: nothing owned, nothing to store
  const int n_a = reach <= 1 ? cn.y : (reach == 2 ? cn.z : cn.w);
  const int e0 = offsets[tile];
  // the entries are the first load of every node and its pulls depend on
  // them: ask L2 for those of the tile HALO_AHEAD launches later
  constexpr int ENTRY_LINES = (HALO_RS + 63) / 64;
  static_assert(ENTRY_LINES <= HALO_THREADS, "one thread per line");
  if (threadIdx.x < ENTRY_LINES && tile + HALO_AHEAD < (int)gridDim.x) {
    const int e1 = __ldg(offsets + tile + HALO_AHEAD);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(entries + e1 + threadIdx.x * 64));
  }
  const bool vavg = ph.bc == BC_VAVG;
  if (vavg && threadIdx.x < HALO_MW) fm[threadIdx.x] = __ldg(fmask + (int64_t)tile * HALO_MW + threadIdx.x);
  const int x0 = (tile % ntx) * HALO_W, y0 = (tile / ntx) * HALO_H;
  const int korg = g.idx(x0 - HALO_R, y0 - HALO_R);  // padded index of slot 0
  const C zr[2][9] = {};  // storage references: unused for 4- and 8-byte populations

  // phase A: rho(t) of the tile and its rings
  for (int t = threadIdx.x; t < n_a; t += HALO_THREADS) {
    const int slot = __ldg(entries + e0 + t) & HE_SLOT;
    const int row = slot / HALO_RW, col = slot - row * HALO_RW;
    const int k = korg + row * g.px + col;
    C fv[2][9];
    gather<T>(f, g, k, zr, fv);
    V v;
    v.x = density(fv[0]);
    v.y = density(fv[1]);
    rho[slot] = v;
  }
  __syncthreads();

  // phase B: Eq. 8 at the interface-solid cells of the tile and its first
  // ring (the solid neighbours of the owned nodes); it reads the densities
  // of fluid slots only and writes solid slots only
  if (vavg) {
    const int tw = min(HALO_W, g.nx - x0), th = min(HALO_H, g.ny - y0);
    const int cw = tw + 2, ch = th + 2;
    auto fluid = [&](int s) { return (fm[s >> 5] >> (s & 31)) & 1u; };
    for (int j = threadIdx.x; j < cw * ch; j += HALO_THREADS) {
      const int row = HALO_R - 1 + j / cw, col = HALO_R - 1 + j % cw;
      const int slot = row * HALO_RW + col;
      if (fluid(slot)) continue;
      uint32_t msk = 0;
      bool iface = false;
#pragma unroll
      for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
          if (dx == 0 && dy == 0) continue;
          if (fluid(slot + dx + dy * HALO_RW)) {
            msk |= 1u << ((dy + 2) * 5 + (dx + 2));
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) iface = true;
          }
        }
      if (!iface) continue;
      auto load = [&](int dx, int dy, C& a, C& b) {
        const V v = rho[slot + dx + dy * HALO_RW];
        a = v.x;
        b = v.y;
      };
      V v;
      if (ph.avg9)
        virtual_density_at<C, true>(msk, ph, load, v.x, v.y);
      else
        virtual_density_at<C, false>(msk, ph, load, v.x, v.y);
      rho[slot] = v;
    }
    __syncthreads();
  }

  // phase C: force, velocity, collision and stores of the owned nodes
  for (int b = 0; b < n_own; b += HALO_THREADS) {
    const int t = b + threadIdx.x;
    const bool valid = t < n_own;
    const uint16_t e = valid ? __ldg(entries + e0 + t) : uint16_t(0);
    const bool warp_edge = __any_sync(0xffffffffu, (e & HE_SOLIDNB) != 0);
    const bool warp_border = __any_sync(0xffffffffu, (e & HE_BORDER) != 0);
    if (!valid) continue;
    const int slot = e & HE_SLOT;
    const int row = slot / HALO_RW, col = slot - row * HALO_RW;
    const int k = korg + row * g.px + col;
    const uint16_t fl = warp_edge ? __ldg(flags + k) : uint16_t(0);
    C fv[2][9];
    gather<T>(f, g, k, zr, fv);
    C nbP[2][9];
    nbP[0][0] = nbP[1][0] = C(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const V v = rho[slot + cx_of(i) + cy_of(i) * HALO_RW];
      nbP[0][i] = v.x;
      nbP[1][i] = v.y;
    }
    C rh[2], uu[2];
    march_update<C>(fv, nbP, fl, warp_edge, ph, rh, uu);
    if (!warp_border) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Pop<T>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], C(0), C(0));
      if (warp_edge) store_bounced_near(fo, g, k, fl, fv, zr);
    } else {
      const int x = x0 - HALO_R + col, y = y0 - HALO_R + row;
      store_node(fo, g, x, y, k, fv, zr);
      store_bounced(fo, g, x, y, fl, fv, zr);
    }
  }
}

template <typename T>
inline lbm_status launch_halo(const Geo& g, const Phys& ph, const T* fin, T* fout, const uint16_t* flags,
                              const uint16_t* entries, const int* offsets, const int4* cnt, const uint32_t* fmask,
                              cudaStream_t stream) {
  if constexpr (kDev<T>) {
    return LBM_ERR_ARG;
  } else {
    const int ntx = (g.nx + HALO_W - 1) / HALO_W;
    const int64_t nt = halo_tile_count(g);
    k_halo<T><<<(unsigned)nt, HALO_THREADS, 0, stream>>>(fin, fout, flags, entries, offsets, cnt, fmask, g, ntx,
                                                         halo_reach(ph), kphys<typename Pop<T>::C>(ph));
    return LBM_OK;
  }
}

}  // namespace lbm
