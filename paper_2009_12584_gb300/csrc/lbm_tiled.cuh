// Tiled single-pass step: one kernel per time step (plus the interface-list
// pass of Eq. 8 under the improved scheme), on compacted per-tile lists.
//
// Same contract as k_march: step t reads rho(t) (rho~(t) at interface-solid
// cells) and f*(t), and writes f*(t+1) and rho(t+1) into the other buffers.
// The owned grid is cut into TILE_W x TILE_H tiles; one CTA takes one tile.
//   Phase 1: every fluid node of the tile and of the one-node ring around
//     it pulls f_i = f*_i(x - c_i, t), takes rho(t) of its neighbours from
//     the plane, evaluates Eqs. 5 and 7, u of Eq. 3 and the collision
//     (Eqs. 1, 2, 4), and keeps f*(t+1) in shared memory; the tile's own
//     nodes also store it to HBM (with bounced slots and periodic images).
//     Ring nodes are computed again by the neighbouring tiles that own them
//     (at their padded index, images included), with the same arithmetic.
//   Phase 2 (after one barrier): rho(t+1) (Eq. 3) of the tile's own fluid
//     nodes as the sum of f_i(x) = f*_i(x - c_i), or of the node's own
//     f*_opp(i) where x - c_i is solid (halfway bounce-back), out of shared
//     memory.
// Fluid nodes are listed per tile at set-up (own nodes first, then the
// ring, each in row order), so no lane works on a solid cell. A list entry
// is 16 bits: the node's slot in the (TILE_W + 2) x (TILE_H + 2) region of
// the tile and two tags.
#pragma once

#include "lbm.h"
#include "lbm_common.cuh"
#include "lbm_fused.cuh"
#include "lbm_geometry.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

#ifndef LBM_TILE_W
#define LBM_TILE_W 32
#endif
#ifndef LBM_TILE_H
#define LBM_TILE_H 14
#endif
#ifndef LBM_TILE_THREADS
#define LBM_TILE_THREADS 256
#endif
#ifndef LBM_TILE_MINB
#define LBM_TILE_MINB 4
#endif
#ifndef LBM_TILE_AHEAD
#define LBM_TILE_AHEAD 512
#endif
constexpr int TILE_W = LBM_TILE_W, TILE_H = LBM_TILE_H;  // owned nodes per tile
constexpr int TILE_RW = TILE_W + 2;         // region pitch (one ring node each side)
constexpr int TILE_RH = TILE_H + 2;
constexpr int TILE_RS = TILE_RW * TILE_RH;  // region slots
constexpr int TILE_THREADS = LBM_TILE_THREADS;  // k_tile
constexpr int TILE_MINB = LBM_TILE_MINB;    // k_tile CTAs per SM the registers must allow
constexpr int TILE_AHEAD = LBM_TILE_AHEAD;  // tiles between a CTA and the one whose entries it prefetches
constexpr int TILE_LIST_THREADS = 256;      // k_tile_lists
static_assert(TILE_RS <= 2048, "slots must fit the 11 slot bits of an entry");

constexpr uint16_t TE_SLOT = 0x07FFu;    // slot = row * TILE_RW + col in the region
constexpr uint16_t TE_SOLIDNB = 0x2000u; // the node has a solid D2Q9 neighbour
constexpr uint16_t TE_BORDER = 0x4000u;  // own node within GH + 1 of a periodic border

inline int64_t tile_count(const Geo& g) {
  return (int64_t)((g.nx + TILE_W - 1) / TILE_W) * ((g.ny + TILE_H - 1) / TILE_H);
}

// Per-tile lists, two passes over the same deterministic order. Count pass
// (entries == nullptr): counts[tile] = fluid nodes of the region rounded up
// to a multiple of 8 (so that every tile's list starts on a 16-byte
// boundary after the scan, for bulk copies), cnt[tile] = (fluid nodes owned
// by the tile, fluid nodes of the region). Write pass: entries from
// offsets[tile] on, the owned nodes first.
static __global__ void __launch_bounds__(TILE_LIST_THREADS) k_tile_lists(const uint16_t* __restrict__ flags, Geo g,
                                                                    int ntx, const int* __restrict__ offsets,
                                                                    int* __restrict__ counts,
                                                                    int2* __restrict__ cnt,
                                                                    uint16_t* __restrict__ entries) {
  __shared__ int warp_cnt[TILE_LIST_THREADS / 32];
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * TILE_W, y0 = (tile / ntx) * TILE_H;
  const int tw = min(TILE_W, g.nx - x0), th = min(TILE_H, g.ny - y0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int base = 0, n_own = 0;
  for (int round = 0; round < 2; ++round) {
    for (int c0 = 0; c0 < TILE_RS; c0 += TILE_LIST_THREADS) {
      const int slot = c0 + threadIdx.x;
      const int row = slot / TILE_RW, col = slot - row * TILE_RW;
      const bool in_region = slot < TILE_RS && col <= tw + 1 && row <= th + 1;
      const bool own = col >= 1 && col <= tw && row >= 1 && row <= th;
      bool hit = false;
      uint16_t e = 0;
      if (in_region && own == (round == 0)) {
        const int x = x0 - 1 + col, y = y0 - 1 + row;
        const uint16_t fl = flags[g.idx(x, y)];
        hit = !(fl & F_SOLID);
        e = (uint16_t)slot;
        if (fl & NB_ANY) e |= TE_SOLIDNB;
        if (own && near_border(g, x, y)) e |= TE_BORDER;
      }
      const unsigned ball = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) warp_cnt[wid] = __popc(ball);
      __syncthreads();
      int before = 0, all = 0;
      for (int w = 0; w < TILE_LIST_THREADS / 32; ++w) {
        const int v = warp_cnt[w];
        before += w < wid ? v : 0;
        all += v;
      }
      if (entries && hit) entries[offsets[tile] + base + before + __popc(ball & ((1u << lane) - 1u))] = e;
      base += all;
      __syncthreads();
    }
    if (round == 0) n_own = base;
  }
  if (!entries && threadIdx.x == 0) {
    counts[tile] = (base + 7) & ~7;
    cnt[tile] = make_int2(n_own, base);
  }
}

// One CTA per tile; dynamic shared memory holds f*(t+1) of the region as
// nine planes of component pairs, [9][TILE_RS]. 16-bit storage: Pref and
// Uref hold the densities and velocities the pulled populations were
// encoded with (their writers' rho(t - 1), 3 u(t - 1)), the node encodes
// what it stores with its own rho(t) and 3 u(t) (written to Uo), and shared
// memory keeps each value as the next step will decode it (encoded and
// decoded again), so that phase 2 sums exactly what the next step pulls,
// like the density pass. Pref, Uref and Uo are not used for 4- and 8-byte
// storage.
// The work of one CTA on tile `tile` of n_tiles (one simulation).
template <typename T>
__device__ __forceinline__ void tile_step(int tile, int n_tiles, const T* __restrict__ f, T* __restrict__ fo,
                                          const typename Pop<T>::C* __restrict__ P,
                                          const typename Pop<T>::C* __restrict__ Pref,
                                          const UPair* __restrict__ Uref, UPair* __restrict__ Uo,
                                          typename Pop<T>::C* __restrict__ Po, const uint16_t* __restrict__ flags,
                                          const uint16_t* __restrict__ entries, const int* __restrict__ offsets,
                                          const int2* __restrict__ cnt, const Geo& g, int ntx,
                                          const PhysK<typename Pop<T>::C>& ph) {
  using C = typename Pop<T>::C;
  using V = typename CPair<C>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s = reinterpret_cast<V*>(smem_raw);
  const int2 cn = cnt[tile];
  const int n_own = cn.x;
  if (n_own == 0) return;  // the whole CTA: nothing owned, nothing to store
  const int e0 = offsets[tile], n_all = cn.y;
  // The entries are the first load of every node and its pulls depend on
  // them: ask L2 for the entries of the tile TILE_AHEAD launches later (one
  // 128-byte line per 64 entries, enough lines for a full region).
  constexpr int ENTRY_LINES = (TILE_RS + 63) / 64;
  static_assert(ENTRY_LINES <= TILE_THREADS, "one thread per line");
  if (threadIdx.x < ENTRY_LINES && tile + TILE_AHEAD < n_tiles) {
    const int e1 = __ldg(offsets + tile + TILE_AHEAD);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(entries + e1 + threadIdx.x * 64));
  }
  const int x0 = (tile % ntx) * TILE_W, y0 = (tile / ntx) * TILE_H;
  const int korg = g.idx(x0 - 1, y0 - 1);  // padded index of slot 0
  for (int b = 0; b < n_all; b += TILE_THREADS) {
    const int t = b + threadIdx.x;
    const bool valid = t < n_all;
    const uint16_t e = valid ? __ldg(entries + e0 + t) : uint16_t(0);
    // the first round asks L2 for the pulls of the second round's node
    const bool pf = b == 0 && t + TILE_THREADS < n_all;
    const uint16_t e2 = pf ? __ldg(entries + e0 + t + TILE_THREADS) : uint16_t(0);
    const bool warp_edge = __any_sync(0xffffffffu, (e & TE_SOLIDNB) != 0);
    const bool warp_border = __any_sync(0xffffffffu, (e & TE_BORDER) != 0);
    if (!valid) continue;
    const int slot = e & TE_SLOT;
    const int row = slot / TILE_RW, col = slot - row * TILE_RW;
    const int k = korg + row * g.px + col;
    const uint16_t fl = warp_edge ? __ldg(flags + k) : uint16_t(0);
    C ref[2][9];  // storage references (zero for 4- and 8-byte populations)
    pull_refs<T>(Pref, Uref, g, k, fl, warp_edge, ref);
    C fv[2][9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
      Pop<T>::ld2(f, pslot(g, i, k - cx_of(i) - cy_of(i) * g.px), ref[0][i], ref[1][i], fv[0][i], fv[1][i]);
    C nbP[2][9];
    neighbour_P(P, g, k, nbP);
    if (pf) {
      const int s2 = e2 & TE_SLOT, r2 = s2 / TILE_RW;
      const int k2 = korg + r2 * g.px + (s2 - r2 * TILE_RW);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(f + pslot(g, i, k2 - cx_of(i) - cy_of(i) * g.px)));
    }
    C rho[2], u[2];
    march_update<C>(fv, nbP, fl, warp_edge, ph, rho, u);
    UVal U{};
    if constexpr (kDev<T>) {
      if (Uo) {
        // momentum of each component's post-collision populations
        float2 jx, jy;
        momentum(fv[0], jx.x, jy.x);
        momentum(fv[1], jx.y, jy.y);
        const UPair up = u_pack(jx, jy, make_float2(rho[0], rho[1]));
        U = u_unpack(up);
        if (t < n_own) {
          Uo[k] = up;
          if (e & TE_BORDER)
            for_ghost_images(g, x0 - 1 + col, y0 - 1 + row, [&](int kk) { Uo[kk] = up; });
        }
      }
    }
    write_refs<T>(rho, Uo != nullptr, U, ref);
    if (t < n_own) {
      if (!warp_border) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Pop<T>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], ref[0][i], ref[1][i]);
        if (warp_edge) store_bounced_near(fo, g, k, fl, fv, ref);
      } else {
        const int x = x0 - 1 + col, y = y0 - 1 + row;
        store_node(fo, g, x, y, k, fv, ref);
        store_bounced(fo, g, x, y, fl, fv, ref);
      }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      V v;
      v.x = Pop<T>::dec(Pop<T>::enc(fv[0][i], ref[0][i]), ref[0][i]);
      v.y = Pop<T>::dec(Pop<T>::enc(fv[1][i], ref[1][i]), ref[1][i]);
      s[i * TILE_RS + slot] = v;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_own; t += TILE_THREADS) {
    const uint16_t e = __ldg(entries + e0 + t);
    const int slot = e & TE_SLOT;
    const int row = slot / TILE_RW, col = slot - row * TILE_RW;
    const int k = korg + row * g.px + col;
    const uint16_t fl = (e & TE_SOLIDNB) ? __ldg(flags + k) : uint16_t(0);
    C fn[2][9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const bool bounce = i != 0 && (fl & nb_bit(opp_of(i)));
      const V v = bounce ? s[opp_of(i) * TILE_RS + slot] : s[i * TILE_RS + slot - cx_of(i) - cy_of(i) * TILE_RW];
      fn[0][i] = v.x;
      fn[1][i] = v.y;
    }
    const C r0 = density(fn[0]), r1 = density(fn[1]);
    stP(Po, k, r0, r1);
    if (e & TE_BORDER) {
      const int x = x0 - 1 + col, y = y0 - 1 + row;
      for_ghost_images(g, x, y, [&](int kk) { stP(Po, kk, r0, r1); });
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(TILE_THREADS, TILE_MINB)
    k_tile(const T* __restrict__ f, T* __restrict__ fo, const typename Pop<T>::C* __restrict__ P,
           const typename Pop<T>::C* __restrict__ Pref, const UPair* __restrict__ Uref,
           UPair* __restrict__ Uo, typename Pop<T>::C* __restrict__ Po,
           const uint16_t* __restrict__ flags,
           const uint16_t* __restrict__ entries, const int* __restrict__ offsets, const int2* __restrict__ cnt,
           Geo g, int ntx, PhysK<typename Pop<T>::C> ph) {
  tile_step<T>(blockIdx.x, gridDim.x, f, fo, P, Pref, Uref, Uo, Po, flags, entries, offsets, cnt, g, ntx, ph);
}

template <typename T>
constexpr size_t tile_smem() {
  return (size_t)9 * TILE_RS * sizeof(typename CPair<typename Pop<T>::C>::V);
}

// Launch one tiled step. *smem_set records, per context (one device), that
// the kernel's dynamic shared memory limit has been raised.
template <typename T>
inline lbm_status launch_tiled(const Geo& g, const Phys& ph, const T* fin, T* fout, const typename Pop<T>::C* P,
                               const typename Pop<T>::C* Pref, const UPair* Uref, UPair* Uo,
                               typename Pop<T>::C* Po, const uint16_t* flags,
                               const uint16_t* entries, const int* offsets, const int2* cnt, bool* smem_set,
                               cudaStream_t stream) {
  constexpr size_t SMEM = tile_smem<T>();
  auto kern = k_tile<T>;
  if (SMEM > 48 * 1024 && !*smem_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess)
      return LBM_ERR_CUDA;
    *smem_set = true;
  }
  const int ntx = (g.nx + TILE_W - 1) / TILE_W;
  const int64_t nt = tile_count(g);
  kern<<<(unsigned)nt, TILE_THREADS, SMEM, stream>>>(fin, fout, P, Pref, Uref, Uo, Po, flags, entries, offsets, cnt, g, ntx,
                                                     kphys<typename Pop<T>::C>(ph));
  return LBM_OK;
}

}  // namespace lbm
