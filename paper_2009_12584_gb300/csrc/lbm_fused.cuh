// Single-pass step: one kernel per time step (plus the interface-list pass
// of Eq. 8 under the improved scheme).
//
// The density plane is double-buffered: step t reads rho(t) (rho~(t) at
// interface-solid cells, written by k_virtual_density just before) and the
// populations f*(t), and writes f*(t+1) together with rho(t+1), so the
// populations cross HBM once per step. Work is split into independent warps:
// a warp owns a strip of MARCH_OWN = 30 columns and a segment of rows, and
// marches up the rows with lane l at column x0 - 1 + l (the two outer lanes
// compute the neighbour strips' border columns again). Per row y it
//   - pulls f_i(x) = f*_i(x - c_i, t) from global memory (halfway
//     bounce-back is folded into the state, see store_bounced),
//   - takes rho(t) of the node's neighbours from the three rows of the
//     density plane it keeps in registers (x +- 1 by warp shuffles),
//   - evaluates Eqs. 5 and 7, u of Eq. 3 and the collision (Eqs. 1, 2, 4),
//     stores f*(t+1) of its owned columns and keeps the row in a 4-row ring
//     in shared memory,
//   - and sums rho(t+1) (Eq. 3) of row y - 1 out of the ring.
// It also computes one row below and above its segment without storing
// them. Only __syncwarp orders the ring; no barrier spans warps.
#pragma once

#include "lbm.h"
#include "lbm_common.cuh"
#include "lbm_pair.cuh"

namespace lbm {

constexpr int MARCH_OWN = 30;   // owned columns per warp
constexpr int MARCH_RING = 4;   // rows of f*(t+1) kept per warp: y - 3 ... y
constexpr int MARCH_WARPS = 4;  // warps per CTA

template <typename T>
struct MarchCfg {
  static constexpr size_t WARP_ELEMS = (size_t)MARCH_RING * 18 * 32;
  static constexpr size_t SMEM = MARCH_WARPS * WARP_ELEMS * sizeof(T);
};

// Force, velocity and collision of one fluid node in place (fv: f on entry,
// f* on exit; nbP: density plane at x + c_i; rho: the node's densities on
// exit; u: the velocity of Eq. 3). The FP32 compute type runs the paired
// path of the two-pass kernel (same arithmetic, same results).
template <typename C>
__device__ __forceinline__ void march_update(C fv[2][9], const C nbP[2][9], uint16_t fl, bool general,
                                             const PhysK<C>& ph, C rho_out[2], C u_out[2]) {
  if constexpr (sizeof(C) == 4) {
    float2 fp[9], q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fp[i] = f2(fv[0][i], fv[1][i]);
      q[i] = f2(nbP[0][i], nbP[1][i]);
    }
    const float2 r = general ? update_pair<true>(fp, q, fl, ph, u_out[0], u_out[1])
                             : update_pair<false>(fp, q, fl, ph, u_out[0], u_out[1]);
    rho_out[0] = r.x;
    rho_out[1] = r.y;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fv[0][i] = fp[i].x;
      fv[1][i] = fp[i].y;
    }
  } else {
    const C rho[2] = {density(fv[0]), density(fv[1])};
    rho_out[0] = rho[0];
    rho_out[1] = rho[1];
    C F[2][2];
    interaction_force<C, true>(ph, fl, rho, nbP, F);
    C jxA, jyA, jxB, jyB;
    momentum(fv[0], jxA, jyA);
    momentum(fv[1], jxB, jyB);
    const C inv = C(1) / (rho[0] + rho[1]);
    const C ux = ((jxA + jxB) + C(0.5) * (F[0][0] + F[1][0])) * inv;
    const C uy = ((jyA + jyB) + C(0.5) * (F[0][1] + F[1][1])) * inv;
    collide(fv, rho, ux, uy, F, ph.omega, ph.kF);
    u_out[0] = ux;
    u_out[1] = uy;
  }
}

// Neighbour value along x from the lane's own column value: lanes 1 ... 31
// take it from the lane to the left (dx = -1) or right (dx = +1); the outer
// lanes use the value they loaded for the column beyond the warp.
template <typename C>
__device__ __forceinline__ C lane_nb(C own, C outer, int lane, int dx) {
  const C v = dx < 0 ? __shfl_up_sync(0xffffffffu, own, 1) : __shfl_down_sync(0xffffffffu, own, 1);
  return (dx < 0 ? lane == 0 : lane == 31) ? outer : v;
}

template <typename T>
__global__ void __launch_bounds__(MARCH_WARPS * 32, 4)
    k_march(const T* __restrict__ f, T* __restrict__ fo, const typename Pop<T>::C* __restrict__ P,
            typename Pop<T>::C* __restrict__ Po, const uint16_t* __restrict__ flags, Geo g,
            PhysK<typename Pop<T>::C> ph, int H) {
  using C = typename Pop<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* ring = (T*)smem_raw + (size_t)wib * MarchCfg<T>::WARP_ELEMS;  // [MARCH_RING][18][32]
  const int xs = (blockIdx.x * MARCH_WARPS + wib) * MARCH_OWN;
  if (xs >= g.nx) return;  // the whole warp
  const int xc = xs - 1 + lane;
  // columns up to nx + 1 are read (ghost layers); up to nx are computed
  // (column nx is the image of column 0 on a periodic axis, solid otherwise)
  const bool reads = xc <= g.nx + 1;
  const bool computable = xc <= g.nx;
  const bool own = lane >= 1 && lane <= MARCH_OWN && xc < g.nx;
  const int xo = lane == 0 ? xc - 1 : xc + 1;  // the outer lanes' extra column
  const bool outer = (lane == 0 || lane == 31) && reads;
  const int y0 = blockIdx.y * H, y_end = min(g.ny, y0 + H);
  C ref[2][9];  // storage references: unused for 4- and 8-byte populations
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 9; ++i) ref[s][i] = C(0);

  // Software pipeline: while row y is computed, the pulled populations of
  // row y + 1 and the flags and density-plane values of row y + 2 are in
  // flight. Density plane rows y - 1 ... y + 2 of this column (p*) and of
  // the outer lanes' extra column (o*), both components.
  C pm[2] = {0, 0}, p0[2] = {0, 0}, pp[2] = {0, 0}, pq[2] = {0, 0};
  C om[2] = {0, 0}, o0[2] = {0, 0}, op[2] = {0, 0}, oq[2] = {0, 0};
  auto load_row = [&](int y, C p[2], C o[2]) {
    if (reads) {
      const int k = g.idx(xc, y);
      ldP(P, k, p[0], p[1]);
    }
    if (outer) {
      const int k = g.idx(xo, y);
      ldP(P, k, o[0], o[1]);
    }
  };
  auto load_flags = [&](int y) -> uint16_t { return reads ? __ldg(flags + g.idx(xc, y)) : F_SOLID; };
  auto pull = [&](int y, uint16_t fl, C fv[2][9]) {
    if (computable && !(fl & F_SOLID)) {
      const int k = g.idx(xc, y);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        Pop<T>::ld2(f, pslot(g, i, k - cx_of(i) - cy_of(i) * g.px), ref[0][i], ref[1][i], fv[0][i], fv[1][i]);
    }
  };
  load_row(y0 - 2, p0, o0);
  load_row(y0 - 1, pp, op);
  load_row(y0, pq, oq);
  uint16_t fl_cur = load_flags(y0 - 1), fl_next = load_flags(y0);
  C fv_next[2][9];
  pull(y0 - 1, fl_cur, fv_next);
  uint16_t fl_prev = F_SOLID;
  for (int y = y0 - 1; y <= y_end; ++y) {
    C fv[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
      for (int i = 0; i < 9; ++i) fv[s][i] = fv_next[s][i];
      pm[s] = p0[s]; p0[s] = pp[s]; pp[s] = pq[s];
      om[s] = o0[s]; o0[s] = op[s]; op[s] = oq[s];
    }
    const uint16_t fl = fl_cur;
    // issue the loads of the rows ahead (all within the ghost layers)
    const uint16_t fl_nn = load_flags(y + 2);
    load_row(y + 2, pq, oq);
    if (y < y_end) pull(y + 1, fl_next, fv_next);
    fl_cur = fl_next;
    fl_next = fl_nn;
    const int k = g.idx(xc, y);
    const bool fluid = computable && !(fl & F_SOLID);
    const bool general = __any_sync(0xffffffffu, fluid && (fl & NB_ANY));
    // density plane at the eight neighbours: rows from registers, x +- 1
    // from the neighbouring lanes (every lane takes part in the shuffles)
    C nbP[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C wm = lane_nb(pm[s], om[s], lane, -1), w0 = lane_nb(p0[s], o0[s], lane, -1),
              wp = lane_nb(pp[s], op[s], lane, -1);
      const C em = lane_nb(pm[s], om[s], lane, +1), e0 = lane_nb(p0[s], o0[s], lane, +1),
              ep = lane_nb(pp[s], op[s], lane, +1);
      nbP[s][0] = 0;
      nbP[s][1] = e0; nbP[s][2] = pp[s]; nbP[s][3] = w0; nbP[s][4] = pm[s];
      nbP[s][5] = ep; nbP[s][6] = wp; nbP[s][7] = wm; nbP[s][8] = em;
    }
    T* rrow = ring + (size_t)((y + MARCH_RING) % MARCH_RING) * 18 * 32 + lane;
    if (fluid) {
      C rho_unused[2];
      C u_unused[2];
      march_update<C>(fv, nbP, fl, general, ph, rho_unused, u_unused);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) rrow[(s * 9 + i) * 32] = Pop<T>::enc(fv[s][i], ref[s][i]);
      if (own && y >= y0 && y < y_end) {
        if (near_border(g, xc, y)) {
          store_node(fo, g, xc, y, k, fv, ref);
          store_bounced(fo, g, xc, y, fl, fv, ref);
        } else {
#pragma unroll
          for (int i = 0; i < 9; ++i)
            Pop<T>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], ref[0][i], ref[1][i]);
          if (fl & NB_ANY) store_bounced_near(fo, g, k, fl, fv, ref);
        }
      }
    }
    __syncwarp();
    // rho(t+1) of row r = y - 1 from the ring (rows r - 1 ... r + 1, lanes
    // l - 1 ... l + 1): f_i(x) = f*_i(x - c_i), or the node's own f*_opp(i)
    // where x - c_i is solid (halfway bounce-back)
    const int r = y - 1;
    if (own && r >= y0 && r < y_end && !(fl_prev & F_SOLID)) {
      const T* b0 = ring + (size_t)((r + MARCH_RING) % MARCH_RING) * 18 * 32 + lane;
      const T* bm = ring + (size_t)((r - 1 + MARCH_RING) % MARCH_RING) * 18 * 32 + lane;
      const T* bp = ring + (size_t)((r + 1 + MARCH_RING) % MARCH_RING) * 18 * 32 + lane;
      C fn[2][9];
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int o = opp_of(i);
          const bool bounce = (i != 0) && (fl_prev & nb_bit(o));
          const T* rb = cy_of(i) > 0 ? bm : (cy_of(i) < 0 ? bp : b0);  // row of x - c_i
          const T raw = bounce ? b0[(s * 9 + o) * 32] : rb[(s * 9 + i) * 32 - cx_of(i)];
          fn[s][i] = Pop<T>::dec(raw, ref[s][i]);
        }
      stP_ghosts(Po, g, xc, r, density(fn[0]), density(fn[1]));
    }
    fl_prev = fl;
  }
}

// The marching kernel keeps 4- and 8-byte populations only (16-bit storage
// needs the encoding references of the step before, which its
// double-buffered density plane no longer holds; the tiled schedule keeps a
// third plane for them).
template <typename T>
inline bool fused_supported(const Geo&, const Phys&) {
  return sizeof(T) >= 4;
}

template <typename T>
// *smem_set records, per context (one device), that the kernel's dynamic
// shared memory limit has been raised (FP64 needs 72 KB).
inline lbm_status launch_fused(const Geo& g, const Phys& ph, const T* fin, T* fout, const typename Pop<T>::C* P,
                               typename Pop<T>::C* Po, const uint16_t* flags, int num_sms, bool* smem_set,
                               cudaStream_t stream) {
  using Cfg = MarchCfg<T>;
  auto kern = k_march<T>;
  if (Cfg::SMEM > 48 * 1024 && !*smem_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess)
      return LBM_ERR_CUDA;
    *smem_set = true;
  }
  const int nstrips = (g.nx + MARCH_OWN - 1) / MARCH_OWN;
  const int gx = (nstrips + MARCH_WARPS - 1) / MARCH_WARPS;
  int per_sm = (int)((220 * 1024) / (Cfg::SMEM + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  const int target = 3 * num_sms * per_sm;  // about three waves of CTAs
  int nseg = (target + gx - 1) / gx;
  int H = (g.ny + nseg - 1) / nseg;
  if (H < 8) H = 8;
  nseg = (g.ny + H - 1) / H;
  kern<<<dim3(gx, nseg), MARCH_WARPS * 32, Cfg::SMEM, stream>>>(fin, fout, P, Po, flags, g,
                                                                kphys<typename Pop<T>::C>(ph), H);
  return LBM_OK;
}

}  // namespace lbm
