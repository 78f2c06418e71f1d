// Kernels of the two-pass schedule and the auxiliary kernels (geometry,
// initialisation, moments, populations, mass). The stored state between
// steps is the post-collision population f*_i(x) at its source node; a step
// pulls f_i(x) = f*_i(x - c_i), the post-streaming distribution of Eq. 1,
// then collides it in place. Halfway bounce-back (Sec. 2) is folded into
// the state: slot i of a solid node x - c_i holds f*_opp(i)(x), written by x
// (store_bounced), so the pull needs no test.
#pragma once

#include "lbm_common.cuh"
#include "lbm_geometry.cuh"
#include "lbm_pair.cuh"

namespace lbm {

// Pull the post-streaming populations of both components at padded index k.
template <typename T, typename C = typename Pop<T>::C>
__device__ __forceinline__ void gather(const T* __restrict__ f, const Geo& g, int k, const C ref[2][9],
                                       C out[2][9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i)
    Pop<T>::ld2(f, pslot(g, i, k - cx_of(i) - cy_of(i) * g.px), ref[0][i], ref[1][i], out[0][i], out[1][i]);
}

// The list entry is the first load of every node and the pulls depend on
// it. A CTA asks L2 for the list lines of the CTA LIST_AHEAD launches after
// it (one 128-byte line per 32 entries), so that CTA finds them there.
constexpr int LIST_AHEAD = 1024;
template <int NT>
__device__ __forceinline__ void prefetch_list_ahead(const int* __restrict__ list, int n) {
  if (threadIdx.x < NT / 32) {
    const int64_t t = ((int64_t)blockIdx.x + LIST_AHEAD) * NT + threadIdx.x * 32;
    if (t < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(list + t));
  }
}

// Encoding references of 16-bit storage. A 2-byte population travelling
// along c_d is stored as its deviation from a reference its writer and its
// reader both know, taken from the node that wrote it when it collided:
//  - by default w_d rho^s of the writer (density plane Pref): the deviation
//    is the velocity and non-equilibrium part, a few percent of f;
//  - with velocity references (lbm_params.velocity_refs), w_d rho^s
//    (1 + c_d . U^s) with U^s = 3 j*^s / rho^s, j*^s the momentum of the
//    populations the writer stored (post-collision), rounded to FP16 and
//    kept with the writer's rho^s in a velocity plane Uref (one 16-byte
//    element per node): the reference then carries the first moment of
//    what was written (the equilibrium's velocity term and the Guo source's
//    first-order term), and the deviation only the rest.
// The 11 (FP16) or 8 (BF16) significand bits go to what varies. For 4- and
// 8-byte storage the references are zero and the planes are not read.
template <typename T>
constexpr bool kDev = sizeof(T) == 2;

// Element of a velocity plane (16 bytes, one load): the writer's rho^A and
// rho^B in FP32 (the densities it encoded with) and its U^A, U^B as two
// FP16 pairs.
using UPair = uint4;
struct UVal {
  float2 v[2];  // U^A, U^B
  float r[2];   // rho^A, rho^B
};
__device__ __forceinline__ UVal u_unpack(UPair p) {
  UVal u;
  u.r[0] = __uint_as_float(p.x);
  u.r[1] = __uint_as_float(p.y);
  u.v[0] = __half22float2(*reinterpret_cast<const __half2*>(&p.z));
  u.v[1] = __half22float2(*reinterpret_cast<const __half2*>(&p.w));
  return u;
}
// The element of a writer with densities rho and momenta (jx, jy)
// (component A in .x, B in .y): U^s = 3 j^s / rho^s rounded to FP16.
__device__ __forceinline__ UPair u_pack(float2 jx, float2 jy, float2 rho) {
  const float ia = rho.x > 0.0f ? 3.0f / rho.x : 0.0f, ib = rho.y > 0.0f ? 3.0f / rho.y : 0.0f;
  const __half2 a = __floats2half2_rn(jx.x * ia, jy.x * ia);
  const __half2 b = __floats2half2_rn(jx.y * ib, jy.y * ib);
  UPair p;
  p.x = __float_as_uint(rho.x);
  p.y = __float_as_uint(rho.y);
  p.z = *reinterpret_cast<const unsigned*>(&a);
  p.w = *reinterpret_cast<const unsigned*>(&b);
  return p;
}

// c_d . U as a fixed sequence of FP32 operations; for -c_d it gives the
// exact negation (round to nearest is symmetric).
__device__ __forceinline__ float cdot(int d, float2 U) {
  const int cx = cx_of(d), cy = cy_of(d);
  float v = cx > 0 ? U.x : (cx < 0 ? -U.x : 0.0f);
  if (cy > 0) v = cx != 0 ? v + U.y : U.y;
  if (cy < 0) v = cx != 0 ? v - U.y : -U.y;
  return v;
}

// w_i rho (1 + cu), one rounding for w_i rho and one for the fused rest.
__device__ __forceinline__ float ref_of(int i, float rho, float cu) {
  const float wr = w_of<float>(i) * rho;
  return fmaf(wr, cu, wr);
}

// References of the 18 populations pulled at padded index k: the writer of
// slot i is x - c_i (direction i), or x itself when x - c_i is solid (its
// bounced slot, which holds the value it sent along -c_i). check: whether fl
// may hold solid neighbours. Uref: the velocity plane, or null.
template <typename T, typename C>
__device__ __forceinline__ void pull_refs(const C* __restrict__ Pref, const UPair* __restrict__ Uref, const Geo& g,
                                          int k, uint16_t fl, bool check, C ref[2][9]) {
  if constexpr (kDev<T>) {
    if (Uref) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const bool self = i == 0 || (check && (fl & nb_bit(opp_of(i))));
        const int m = self ? k : k - cx_of(i) - cy_of(i) * g.px;
        const UVal u = u_unpack(__ldg(Uref + m));  // the writer's densities and velocities
        const bool back = self && i != 0;          // the value was sent along -c_i
        const float ca = cdot(i, u.v[0]), cb = cdot(i, u.v[1]);
        ref[0][i] = ref_of(i, u.r[0], back ? -ca : ca);
        ref[1][i] = ref_of(i, u.r[1], back ? -cb : cb);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const bool self = i == 0 || (check && (fl & nb_bit(opp_of(i))));
        const int m = self ? k : k - cx_of(i) - cy_of(i) * g.px;
        C a, b;
        ldP(Pref, m, a, b);
        ref[0][i] = w_of<C>(i) * a;
        ref[1][i] = w_of<C>(i) * b;
      }
    }
  } else {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) ref[s][i] = C(0);
  }
}

// References for what a node writes, given its own rho and (with velocity
// references, vref) its U as stored: ref[s][i] for its slot i (direction
// i). Its bounced slot i holds the value sent along -c_i, whose reference
// is ref[s][opp(i)].
template <typename T, typename C>
__device__ __forceinline__ void write_refs(const C rho[2], bool vref, const UVal& U, C ref[2][9]) {
  if constexpr (kDev<T>) {
    if (vref) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) ref[s][i] = ref_of(i, rho[s], cdot(i, U.v[s]));
    } else {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) ref[s][i] = w_of<C>(i) * rho[s];
    }
  } else {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) ref[s][i] = C(0);
  }
}

// ---- K1: densities --------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_density(const T* __restrict__ f, typename Pop<T>::C* __restrict__ P,
                                                 const typename Pop<T>::C* __restrict__ Pref,
                                                 const UPair* __restrict__ Uref,
                                                 const uint16_t* __restrict__ flags, Geo g,
                                                 PhysK<typename Pop<T>::C> ph) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  if (fl & F_SOLID) return;
  C ref[2][9];
  pull_refs<T>(Pref, Uref, g, k, fl, true, ref);
  C fv[2][9];
  gather<T>(f, g, k, ref, fv);
  stP_ghosts(P, g, x, y, density(fv[0]), density(fv[1]));
}

// Read the density plane at the 8 neighbours of padded index k.
template <typename C>
__device__ __forceinline__ void neighbour_P(const C* __restrict__ P, const Geo& g, int k, C nbP[2][9]) {
  nbP[0][0] = nbP[1][0] = 0;
#pragma unroll
  for (int i = 1; i < 9; ++i) ldP(P, k + cx_of(i) + cy_of(i) * g.px, nbP[0][i], nbP[1][i]);
}

// Owned coordinates of padded index k.
__device__ __forceinline__ void coords(const Geo& g, int k, int& x, int& y) {
  y = k / g.px - GH;
  x = k - (y + GH) * g.px - LP;
}

// ---- K1 over the fluid-node list (node order, edge nodes tagged) ---------
template <typename T>
__device__ __forceinline__ void density_node(const T* __restrict__ f, typename Pop<T>::C* __restrict__ P,
                                             const typename Pop<T>::C* __restrict__ Pref,
                                             const UPair* __restrict__ Uref,
                                             const uint16_t* __restrict__ flags, const int* __restrict__ list, int t,
                                             const Geo& g) {
  using C = typename Pop<T>::C;
  const unsigned e = (unsigned)__ldg(list + t);
  const int k = (int)(e & ~LIST_TAGS);
  C ref[2][9];
  if constexpr (kDev<T>) {
    const bool edge = e & EDGE_TAG;
    pull_refs<T>(Pref, Uref, g, k, edge ? __ldg(flags + k) : uint16_t(0), edge, ref);
  } else {
    pull_refs<T>(Pref, Uref, g, k, 0, false, ref);
  }
  C fv[2][9];
  gather<T>(f, g, k, ref, fv);
  const C r0 = density(fv[0]), r1 = density(fv[1]);
  stP(P, k, r0, r1);
  if (e & BORDER_TAG) {  // may have periodic images
    int x, y;
    coords(g, k, x, y);
    for_ghost_images(g, x, y, [&](int kk) {
      stP(P, kk, r0, r1);
    });
  }
}

// VR: whether the velocity planes may be read (16-bit storage with velocity
// references); without it Uref is never touched and the kernel carries no
// code for it, and 32 registers give 8 CTAs per SM.
template <typename T, bool VR = false>
__global__ void __launch_bounds__(256, VR ? 1 : 8) k_density_list(const T* __restrict__ f, typename Pop<T>::C* __restrict__ P,
                                                      const typename Pop<T>::C* __restrict__ Pref,
                                                      const UPair* __restrict__ Uref,
                                                      const uint16_t* __restrict__ flags,
                                                      const int* __restrict__ list, int nfluid, Geo g,
                                                      PhysK<typename Pop<T>::C> ph) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nfluid) density_node<T>(f, P, Pref, VR ? Uref : nullptr, flags, list, t, g);
}

// The update of collide_node for the FP32 compute type, with the two
// components as float2 pairs (lbm_pair.cuh). Same paths, same stores.
template <typename T>
__device__ __forceinline__ void collide_node_pair(const T* __restrict__ f, T* __restrict__ fo,
                                                  const float* __restrict__ P, const float* __restrict__ Pref,
                                                  const UPair* __restrict__ Uref, UPair* __restrict__ Uo,
                                                  const uint16_t* __restrict__ flags, unsigned e, bool warp_edge,
                                                  bool warp_border, const Geo& g, const PhysK<float>& ph) {
  const int k = (int)(e & ~LIST_TAGS);
  const uint16_t fl = warp_edge ? __ldg(flags + k) : uint16_t(0);
  float ref[2][9];
  pull_refs<T>(Pref, Uref, g, k, fl, warp_edge, ref);
  float2 fp[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    Pop<T>::ld2(f, pslot(g, i, k - cx_of(i) - cy_of(i) * g.px), ref[0][i], ref[1][i], fp[i].x, fp[i].y);
  }
  float2 q[9];
  q[0] = f2(0.0f);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int m = k + cx_of(i) + cy_of(i) * g.px;
    q[i] = __ldg(reinterpret_cast<const float2*>(P) + m);
  }
  float ux, uy;
  const float2 rho = warp_edge ? update_pair<true>(fp, q, fl, ph, ux, uy) : update_pair<false>(fp, q, fl, ph, ux, uy);
  const float rr[2] = {rho.x, rho.y};
  UVal U{};
  if constexpr (kDev<T>) {
    if (Uo) {
      // momentum of each component's post-collision populations
      const float2 d57 = sub2(fp[5], fp[7]), d86 = sub2(fp[8], fp[6]);
      const float2 jx = add2(sub2(fp[1], fp[3]), add2(d57, d86));
      const float2 jy = add2(sub2(fp[2], fp[4]), sub2(d57, d86));
      const UPair up = u_pack(jx, jy, rho);
      U = u_unpack(up);
      Uo[k] = up;
      if (warp_border) {
        int x, y;
        coords(g, k, x, y);
        for_ghost_images(g, x, y, [&](int kk) { Uo[kk] = up; });
      }
    }
  }
  write_refs<T>(rr, Uo != nullptr, U, ref);
  if (!warp_border) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Pop<T>::st2(fo, pslot(g, i, k), fp[i].x, fp[i].y, ref[0][i], ref[1][i]);
    }
    if (warp_edge) {
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        if (!(fl & nb_bit(opp_of(i)))) continue;
        const int ks = k - cx_of(i) - cy_of(i) * g.px;
        Pop<T>::st2(fo, pslot(g, i, ks), fp[opp_of(i)].x, fp[opp_of(i)].y, ref[0][opp_of(i)], ref[1][opp_of(i)]);
      }
    }
  } else {
    float fv[2][9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fv[0][i] = fp[i].x;
      fv[1][i] = fp[i].y;
    }
    int x, y;
    coords(g, k, x, y);
    store_node(fo, g, x, y, k, fv, ref);
    store_bounced(fo, g, x, y, fl, fv, ref);
  }
}

// ---- K3 over the fluid-node list ------------------------------------------
// 128-thread CTAs, 8 per SM at 64 registers: a CTA's slot frees sooner than
// with 256 threads when its warps finish at different times.
constexpr int COLLIDE_THREADS = 128;

// Three paths, chosen per warp so that a warp never splits between them: a
// warp whose 32 nodes are all bulk (eight fluid neighbours, away from
// periodic borders) loads no flags and has no adhesion and no bounce-back;
// a warp with wall nodes but none near a periodic border stores bounced
// slots at k - c_i; any other warp takes the general path with periodic
// images. All lanes of the warp must call this (t >= nfluid marks an idle
// lane).
template <typename T>
__device__ __forceinline__ void collide_node(const T* __restrict__ f, T* __restrict__ fo,
                                             const typename Pop<T>::C* __restrict__ P,
                                             const typename Pop<T>::C* __restrict__ Pref,
                                             const UPair* __restrict__ Uref, UPair* __restrict__ Uo,
                                             const uint16_t* __restrict__ flags, const int* __restrict__ list,
                                             int t, int nfluid, const Geo& g,
                                             const PhysK<typename Pop<T>::C>& ph) {
  using C = typename Pop<T>::C;
  const bool valid = t < nfluid;
  const unsigned e = valid ? (unsigned)__ldg(list + t) : 0u;
  const bool warp_edge = __any_sync(0xffffffffu, (e & EDGE_TAG) != 0u);
  const bool warp_border = __any_sync(0xffffffffu, (e & BORDER_TAG) != 0u);
  if (!valid) return;
  if constexpr (sizeof(C) == 4) {
    collide_node_pair<T>(f, fo, P, Pref, Uref, Uo, flags, e, warp_edge, warp_border, g, ph);
    return;
  } else {
  const int k = (int)(e & ~LIST_TAGS);
  const uint16_t fl = warp_edge ? __ldg(flags + k) : uint16_t(0);
  C ref[2][9];
  pull_refs<T>(Pref, Uref, g, k, fl, warp_edge, ref);
  C fv[2][9];
  gather<T>(f, g, k, ref, fv);
  const C rho[2] = {density(fv[0]), density(fv[1])};
  C nbP[2][9];
  neighbour_P(P, g, k, nbP);
  C F[2][2];
  if (!warp_edge) {
    interaction_force<C, true>(ph, 0, rho, nbP, F);
  } else {
    interaction_force<C, false>(ph, fl, rho, nbP, F);
  }
  C jxA, jyA, jxB, jyB;
  momentum(fv[0], jxA, jyA);
  momentum(fv[1], jxB, jyB);
  const C inv = C(1) / (rho[0] + rho[1]);
  const C ux = ((jxA + jxB) + C(0.5) * (F[0][0] + F[1][0])) * inv;
  const C uy = ((jyA + jyB) + C(0.5) * (F[0][1] + F[1][1])) * inv;
  collide(fv, rho, ux, uy, F, ph.omega, ph.kF);
  write_refs<T>(rho, false, UVal{}, ref);  // the FP64 compute type stores 8-byte populations
  if (!warp_border) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Pop<T>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], ref[0][i], ref[1][i]);
    if (warp_edge) store_bounced_near(fo, g, k, fl, fv, ref);
  } else {
    int x, y;
    coords(g, k, x, y);
    store_node(fo, g, x, y, k, fv, ref);
    store_bounced(fo, g, x, y, fl, fv, ref);
  }
  }
}

// VR as for k_density_list (Uref and Uo untouched without it).
template <typename T, bool VR = false>
__global__ void __launch_bounds__(COLLIDE_THREADS, 8) k_collide_list(const T* __restrict__ f, T* __restrict__ fo,
                                                         const typename Pop<T>::C* __restrict__ P,
                                                         const typename Pop<T>::C* __restrict__ Pref,
                                                         const UPair* __restrict__ Uref,
                                                         UPair* __restrict__ Uo,
                                                         const uint16_t* __restrict__ flags,
                                                         const int* __restrict__ list, int nfluid, Geo g,
                                                         PhysK<typename Pop<T>::C> ph) {
  prefetch_list_ahead<COLLIDE_THREADS>(list, nfluid);
  collide_node<T>(f, fo, P, Pref, VR ? Uref : nullptr, VR ? Uo : nullptr, flags, list,
                  blockIdx.x * blockDim.x + threadIdx.x, nfluid, g, ph);
}

// ---- K2: virtual solid density of Eq. 8 over the interface-solid list -----
// The fluid neighbours come from the per-cell mask built with the geometry
// (k_iface_mask); the densities of all of them are loaded in one round trip
// before the sums. The 5 x 5 stencil reads around scattered cells use up
// whole 128-byte lines, so these loads ask L2 for 128-byte fetches whatever
// the context's fetch granularity (the pulls of the other passes run best
// with 32-byte fetches).
template <typename C>
__device__ __forceinline__ void ldP_line(const C* __restrict__ P, int64_t k, C& a, C& b) {
  if constexpr (sizeof(C) == 4)
    asm("ld.global.nc.L2::128B.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(P + 2 * k));
  else
    asm("ld.global.nc.L2::128B.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(P + 2 * k));
}

// Eq. 8 at one interface-solid cell: msk holds its fluid neighbours (bit
// (dy + 2) * 5 + (dx + 2)), load(dx, dy, a, b) fetches the densities of
// neighbour (dx, dy); the sums run in a fixed order, so every caller (the
// plane-based pass and the shared-memory pass of the halo schedule) gets
// the same bits.
template <typename C, bool AVG9, typename Load>
__device__ __forceinline__ void virtual_density_at(uint32_t msk, const PhysK<C>& ph, Load&& load, C& v0, C& v1) {
  constexpr int REACH = AVG9 ? 1 : 2;
  constexpr int NB = (2 * REACH + 1) * (2 * REACH + 1);
  C p0[NB], p1[NB];
#pragma unroll
  for (int dy = -REACH; dy <= REACH; ++dy)
#pragma unroll
    for (int dx = -REACH; dx <= REACH; ++dx) {
      const int j = (dy + REACH) * (2 * REACH + 1) + (dx + REACH);
      p0[j] = p1[j] = C(0);
      if ((msk >> ((dy + 2) * 5 + (dx + 2))) & 1u) load(dx, dy, p0[j], p1[j]);
    }
  C num0 = 0, num1 = 0, den = 0;
#pragma unroll
  for (int dy = -REACH; dy <= REACH; ++dy)
#pragma unroll
    for (int dx = -REACH; dx <= REACH; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const int j = (dy + REACH) * (2 * REACH + 1) + (dx + REACH);
      const bool fluid = (msk >> ((dy + 2) * 5 + (dx + 2))) & 1u;
      const int r2 = dx * dx + dy * dy;
      const C w = AVG9 ? (r2 == 1 ? C(1) / C(9) : C(1) / C(36))
                       : (r2 == 1   ? C(4) / C(21)
                          : r2 == 2 ? C(4) / C(45)
                          : r2 == 4 ? C(1) / C(60)
                          : r2 == 5 ? C(2) / C(315)
                                    : C(1) / C(5040));  // D2Q25 weights printed after Eq. 8
      num0 += fluid ? w * p0[j] : C(0);
      num1 += fluid ? w * p1[j] : C(0);
      den += fluid ? w : C(0);
    }
  v0 = ph.chi[0] * num0 / den;
  v1 = ph.chi[1] * num1 / den;
}

template <typename C, bool AVG9>
__device__ __forceinline__ void virtual_density(const C* __restrict__ P, uint32_t msk, const Geo& g, int k,
                                                const PhysK<C>& ph, C& v0, C& v1) {
  virtual_density_at<C, AVG9>(msk, ph, [&](int dx, int dy, C& a, C& b) { ldP_line(P, k + dx + dy * g.px, a, b); },
                              v0, v1);
}

template <typename C>
__device__ __forceinline__ void virtual_density_node(C* __restrict__ P, const uint32_t* __restrict__ mask,
                                                     const int* __restrict__ list, int t, const Geo& g,
                                                     const PhysK<C>& ph) {
  const int k = list[t];
  const uint32_t msk = mask[t];
  C v0, v1;
  if (ph.avg9)
    virtual_density<C, true>(P, msk, g, k, ph, v0, v1);
  else
    virtual_density<C, false>(P, msk, g, k, ph, v0, v1);
  int x, y;
  coords(g, k, x, y);
  stP_ghosts(P, g, x, y, v0, v1);
}

template <typename C>
__global__ void __launch_bounds__(128) k_virtual_density(C* __restrict__ P, const uint32_t* __restrict__ mask,
                                                         const int* __restrict__ list, int n, Geo g,
                                                         PhysK<C> ph) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) virtual_density_node<C>(P, mask, list, t, g, ph);
}


// ---- Evaluation of the current state: moments or forces -----------------
// MODE 1: write the moments (rho^A, rho^B, u of Eq. 3). MODE 2: write the
// forces (Eq. 5 + Eq. 7). The populations are not changed. O: the type of
// the output arrays (double, or float for the FP32 host interface).
template <typename T, int MODE, typename O = double>
__global__ void __launch_bounds__(128) k_collide(const T* __restrict__ f, const typename Pop<T>::C* __restrict__ P,
                                                 const typename Pop<T>::C* __restrict__ Pref,
                                                 const UPair* __restrict__ Uref,
                                                 const uint16_t* __restrict__ flags, Geo g,
                                                 PhysK<typename Pop<T>::C> ph, O* __restrict__ out) {
  static_assert(MODE == 1 || MODE == 2, "evaluation modes only");
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  const int64_t n = (int64_t)y * g.nx + x;
  const int64_t N = (int64_t)g.nx * g.ny;
  if (fl & F_SOLID) {
    out[n] = 0; out[N + n] = 0; out[2 * N + n] = 0; out[3 * N + n] = 0;
    return;
  }
  C ref[2][9];
  pull_refs<T>(Pref, Uref, g, k, fl, true, ref);
  C fv[2][9];
  gather<T>(f, g, k, ref, fv);
  C rho[2] = {density(fv[0]), density(fv[1])};
  C nbP[2][9];
  neighbour_P(P, g, k, nbP);
  C F[2][2];
  interaction_force(ph, fl, rho, nbP, F);
  C jxA, jyA, jxB, jyB;
  momentum(fv[0], jxA, jyA);
  momentum(fv[1], jxB, jyB);
  const C inv = C(1) / (rho[0] + rho[1]);
  const C ux = ((jxA + jxB) + C(0.5) * (F[0][0] + F[1][0])) * inv;
  const C uy = ((jyA + jyB) + C(0.5) * (F[0][1] + F[1][1])) * inv;
  if (MODE == 1) {
    out[n] = O(rho[0]);
    out[N + n] = O(rho[1]);
    out[2 * N + n] = O(ux);
    out[3 * N + n] = O(uy);
  } else {
    out[n] = O(F[0][0]);
    out[N + n] = O(F[0][1]);
    out[2 * N + n] = O(F[1][0]);
    out[3 * N + n] = O(F[1][1]);
  }
}

// Widen n floats to doubles (separate arrays).
static __global__ void k_widen(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

// ---- post-streaming populations out / in ---------------------------------
template <typename T>
__global__ void k_get_populations(const T* __restrict__ f, const typename Pop<T>::C* __restrict__ Pref,
                                  const UPair* __restrict__ Uref,
                                  const uint16_t* __restrict__ flags, Geo g,
                                  PhysK<typename Pop<T>::C> ph, double* __restrict__ out) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  const int64_t n = (int64_t)y * g.nx + x, N = (int64_t)g.nx * g.ny;
  C fv[2][9];
  if (fl & F_SOLID) {
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 9; ++i) fv[s][i] = 0;
  } else {
    C ref[2][9];
    pull_refs<T>(Pref, Uref, g, k, fl, true, ref);
    gather<T>(f, g, k, ref, fv);
  }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 9; ++i) out[(s * 9 + i) * N + n] = fv[s][i];
}

// Wrapped compact index of (x, y) for caller arrays [ny][nx].
// Compact index of node (x, y) with x in [-1, nx] and y in [-1, ny],
// wrapped once (a D2Q9 neighbour of an owned node).
__device__ __forceinline__ int64_t wrap_compact(const Geo& g, int x, int y) {
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  return (int64_t)y * g.nx + x;
}

// State from post-streaming populations O: the stored f*_j(y) is the value
// that streaming delivers to (y + c_j, j), or to (y, opp(j)) when y + c_j
// is solid; and slot i of a solid node x - c_i holds O_i(x) (the bounced
// value x receives). SRC 0: O is read from fin [2][9][ny][nx]. SRC 1: O is
// the equilibrium of Eq. 2 of the rho/u arrays.
// The node's own post-streaming density (to Pref) and 3 u (to Uo, 16-bit
// storage only; u = the momentum of the received populations over their
// density) are the encoding references of everything the node stores here.
template <typename T, int SRC>
__global__ void k_set_state(T* __restrict__ f, typename Pop<T>::C* __restrict__ Pref, UPair* __restrict__ Uo,
                            const uint16_t* __restrict__ flags, Geo g, PhysK<typename Pop<T>::C> ph,
                            const double* __restrict__ fin, const double* __restrict__ rA,
                            const double* __restrict__ rB, const double* __restrict__ ux,
                            const double* __restrict__ uy) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  if (fl & F_SOLID) return;
  const int64_t N = (int64_t)g.nx * g.ny;
  // Eq. 2 is evaluated in the compute type: FP32 for 4- and 2-byte storage,
  // FP64 for FP64 storage. The caller's FP64 fields of a node are converted
  // once (FP64 instructions, conversions included, run at a small fraction
  // of the FP32 rate on this GPU).
  struct Node { C r[2], vx, vy; };
  auto node = [&](int64_t m) {
    Node v;
    v.r[0] = C(rA[m]);
    v.r[1] = C(rB[m]);
    v.vx = ux ? C(ux[m]) : C(0);
    v.vy = uy ? C(uy[m]) : C(0);
    return v;
  };
  auto feq = [&](const Node& v, int s, int j) -> C {
    const C cu = C(cx_of(j)) * v.vx + C(cy_of(j)) * v.vy;
    return v.r[s] * w_of<C>(j) * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * (v.vx * v.vx + v.vy * v.vy));
  };
  const int64_t n = (int64_t)y * g.nx + x;
  Node own{};
  if (SRC == 1) own = node(n);
  // O at node m (whose converted fields are v when SRC == 1), component s,
  // direction j
  auto O = [&](int64_t m, const Node& v, int s, int j) -> C {
    if (SRC == 0) return C(fin[(s * 9 + j) * N + m]);
    return feq(v, s, j);
  };
  C rho0[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    C r = C(0);
    for (int j = 0; j < 9; ++j) r += O(n, own, s, j);
    rho0[s] = r;
  }
  stP_ghosts(Pref, g, x, y, rho0[0], rho0[1]);
  UVal U{};
  if constexpr (kDev<T>) {
    if (Uo) {
      // momentum of each component's received populations
      float j[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
      for (int s = 0; s < 2; ++s)
        for (int jd = 1; jd < 9; ++jd) {
          const C o = O(n, own, s, jd);
          j[s][0] += float(cx_of(jd)) * o;
          j[s][1] += float(cy_of(jd)) * o;
        }
      const UPair up = u_pack(make_float2(j[0][0], j[1][0]), make_float2(j[0][1], j[1][1]),
                              make_float2(rho0[0], rho0[1]));
      U = u_unpack(up);
      put_with_ghosts(Uo, g, x, y, up);
    }
  }
  C ref[2][9];
  write_refs<T>(rho0, Uo != nullptr, U, ref);
  C fv[2][9];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const bool bounce = (j != 0) && (fl & nb_bit(j));
    const int64_t m = bounce ? n : wrap_compact(g, x + cx_of(j), y + cy_of(j));
    Node nb{};
    if (SRC == 1 && !bounce) nb = node(m);
#pragma unroll
    for (int s = 0; s < 2; ++s) fv[s][j] = C(bounce ? O(n, own, s, opp_of(j)) : O(m, nb, s, j));
  }
  store_node(f, g, x, y, k, fv, ref);
  // the bounced slots: store_bounced writes fv[s][opp(i)] into slot i, so
  // pass it the received values O_i(x) in the opposite slots
  if (fl & NB_ANY) {
    C rv[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) rv[s][opp_of(i)] = C(O(n, own, s, i));
    store_bounced(f, g, x, y, fl, rv, ref);
  }
}

// ---- FP64 mass: per-block partial sums, then one fixed-order final sum ----
template <typename T>
__global__ void __launch_bounds__(256) k_mass_partial(const T* __restrict__ f,
                                                      const typename Pop<T>::C* __restrict__ Pref,
                                                      const UPair* __restrict__ Uref,
                                                      const uint16_t* __restrict__ flags, Geo g,
                                                      PhysK<typename Pop<T>::C> ph, double* __restrict__ partial) {
  using C = typename Pop<T>::C;
  __shared__ double red[2][256 / 32];
  double acc[2] = {0.0, 0.0};
  const int64_t N = (int64_t)g.nx * g.ny;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(n / g.nx), x = (int)(n % g.nx);
    const int k = g.idx(x, y);
    if (flags[k] & F_SOLID) continue;
    // a node's own slots were written by the node itself
    C rw[2] = {C(0), C(0)};
    UVal U{};
    if (kDev<T>) {
      if (Uref) {
        U = u_unpack(Uref[k]);
        rw[0] = U.r[0];
        rw[1] = U.r[1];
      } else {
        ldP(Pref, k, rw[0], rw[1]);
      }
    }
    C ref[2][9];
    write_refs<T>(rw, Uref != nullptr, U, ref);
    double r[2] = {0.0, 0.0};
    for (int i = 0; i < 9; ++i) {
      C a, b;
      Pop<T>::ld2(f, pslot(g, i, k), ref[0][i], ref[1][i], a, b);
      r[0] += (double)a;
      r[1] += (double)b;
    }
    acc[0] += r[0];
    acc[1] += r[1];
  }
  for (int s = 0; s < 2; ++s) {
    double v = acc[s];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[s][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[s][w];
      partial[2 * blockIdx.x + s] = v;
    }
  }
}

static __global__ void k_mass_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  // one warp per component, fixed lane/stride order, then a fixed shuffle tree
  const int s = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (s >= 2) return;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += partial[2 * b + s];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[s] = v;
}

}  // namespace lbm
