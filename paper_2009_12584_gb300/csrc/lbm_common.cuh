// Shared device-side definitions of the GB300 lattice-Boltzmann library:
// D2Q9 tables, the padded grid geometry, population storage formats and the
// per-node physics of one time step (Eqs. 2-5, 7 of arXiv:2009.12584).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (Sec. 2): 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
// constexpr functions so that fully unrolled loops fold them to immediates.
__host__ __device__ constexpr int cx_of(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename C>
__host__ __device__ constexpr C w_of(int i) {
  return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// Ghost layer width around the owned nx * ny nodes. Periodic axes hold
// copies of the opposite border there; walled axes hold solid cells. Four
// layers cover the widest stencil of the step (Eq. 8's D2Q25 reach of 2 plus
// the force's reach of 1, plus one for streaming).
constexpr int GH = 4;
// Columns of padding left of column 0: more than the ghost layers so that
// column 0 starts on a 128-byte boundary for 4-byte types (aligned stores of
// whole rows); the columns beyond the ghost layers count as solid.
constexpr int LP = 32;

// Per-node flag bits (uint16): bit 0 the node is solid; bit i (1..8) the
// neighbour x + c_i is solid; bit 9 interface-solid (a solid node with a
// fluid D2Q9 neighbour).
constexpr uint16_t F_SOLID = 1u;
constexpr uint16_t F_IFACE = 1u << 9;
constexpr uint16_t NB_ANY = 0x1FEu;  // any of the eight neighbours solid
__host__ __device__ constexpr uint16_t nb_bit(int i) { return uint16_t(1u << i); }

struct Geo {
  int nx, ny;      // owned nodes
  int px, py;      // padded pitch and rows
  int64_t plane;   // px * py
  int per_x, per_y;
  __host__ __device__ int idx(int x, int y) const { return (y + GH) * px + (x + LP); }
};

// Call fn(k) for every padded index k that holds a periodic image of owned
// node (x, y) (up to three: one per periodic axis plus the corner). A node
// may have images on both sides of an axis when that axis is shorter than
// twice the ghost width.
template <typename Fn>
__device__ __forceinline__ void for_ghost_images(const Geo& g, int x, int y, Fn&& fn) {
  const bool xa = g.per_x && x < GH, xb = g.per_x && x >= g.nx - GH;
  const bool ya = g.per_y && y < GH, yb = g.per_y && y >= g.ny - GH;
  if (!(xa | xb | ya | yb)) return;
  const int x1 = x + g.nx, x2 = x - g.nx, y1 = y + g.ny, y2 = y - g.ny;
  if (xa) fn(g.idx(x1, y));
  if (xb) fn(g.idx(x2, y));
  if (ya) {
    fn(g.idx(x, y1));
    if (xa) fn(g.idx(x1, y1));
    if (xb) fn(g.idx(x2, y1));
  }
  if (yb) {
    fn(g.idx(x, y2));
    if (xa) fn(g.idx(x1, y2));
    if (xb) fn(g.idx(x2, y2));
  }
}

// Store v at owned node (x, y) of a plane and at its periodic images.
template <typename V>
__device__ __forceinline__ void put_with_ghosts(V* plane, const Geo& g, int x, int y, V v) {
  plane[g.idx(x, y)] = v;
  for_ghost_images(g, x, y, [&](int k) { plane[k] = v; });
}

// ---------------------------------------------------------------------------
// Density planes (rho, rho~ at interface-solid cells, and the encoding
// references of 16-bit storage) hold (component A, component B) pairs: the
// value of component s at padded index k is element 2 k + s.
template <typename C>
struct CPair;
template <>
struct CPair<float> {
  using V = float2;
};
template <>
struct CPair<double> {
  using V = double2;
};

template <typename C>
__device__ __forceinline__ void ldP(const C* __restrict__ P, int64_t k, C& a, C& b) {
  const typename CPair<C>::V v = __ldg(reinterpret_cast<const typename CPair<C>::V*>(P) + k);
  a = v.x;
  b = v.y;
}
template <typename C>
__device__ __forceinline__ void stP(C* __restrict__ P, int64_t k, C a, C b) {
  typename CPair<C>::V v;
  v.x = a;
  v.y = b;
  reinterpret_cast<typename CPair<C>::V*>(P)[k] = v;
}
// Store the pair at owned node (x, y) and at its periodic images.
template <typename C>
__device__ __forceinline__ void stP_ghosts(C* __restrict__ P, const Geo& g, int x, int y, C a, C b) {
  stP(P, g.idx(x, y), a, b);
  for_ghost_images(g, x, y, [&](int k) { stP(P, k, a, b); });
}

// ---------------------------------------------------------------------------
// Population storage. FP32/FP64 store f itself. FP16/BF16 store the
// deviation of f from a reference its writer and reader both know (see
// pull_refs), which keeps the rest-state part exact and spends the 11/8
// significand bits on what varies.
//
// Layout: nine planes of component pairs. The populations of components A
// and B for direction i at padded index k are adjacent, at element
// pslot(g, i, k) + s, so that one vector access (8 bytes for FP32) moves
// both and each plane streams as a single sequence.
__host__ __device__ __forceinline__ int64_t pslot(const Geo& g, int i, int64_t k) {
  return ((int64_t)i * g.plane + k) * 2;
}

template <typename T>
struct Pop;
template <>
struct Pop<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float* p, int64_t k, float) { return p[k]; }
  static __device__ __forceinline__ void st(float* p, int64_t k, float v, float) { p[k] = v; }
  static __device__ __forceinline__ float enc(float v, float) { return v; }
  static __device__ __forceinline__ float dec(float v, float) { return v; }
  static __device__ __forceinline__ void ld2(const float* p, int64_t j, float, float, float& a, float& b) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p + j));
    a = v.x;
    b = v.y;
  }
  static __device__ __forceinline__ void st2(float* p, int64_t j, float a, float b, float, float) {
    *reinterpret_cast<float2*>(p + j) = make_float2(a, b);
  }
};
template <>
struct Pop<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double* p, int64_t k, double) { return p[k]; }
  static __device__ __forceinline__ void st(double* p, int64_t k, double v, double) { p[k] = v; }
  static __device__ __forceinline__ double enc(double v, double) { return v; }
  static __device__ __forceinline__ double dec(double v, double) { return v; }
  static __device__ __forceinline__ void ld2(const double* p, int64_t j, double, double, double& a, double& b) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p + j));
    a = v.x;
    b = v.y;
  }
  static __device__ __forceinline__ void st2(double* p, int64_t j, double a, double b, double, double) {
    *reinterpret_cast<double2*>(p + j) = make_double2(a, b);
  }
};
// FP16 keeps the deviation times 2^12 (exact: a power of two), so that the
// small deviations left by the references stay out of FP16's subnormal range
// (below 2^-14), where precision would be absolute instead of relative;
// deviations up to 16 in magnitude fit.
// The difference from and the sum with the reference are explicitly rounded
// operations (__fsub_rn, __fadd_rn), which the compiler never fuses with the
// multiply that formed the reference (w_i rho): every kernel encodes and
// decodes with the same roundings, whatever it inlined around them.
constexpr float HALF_SCALE = 4096.0f, HALF_UNSCALE = 1.0f / 4096.0f;
template <>
struct Pop<__half> {
  using C = float;
  static __device__ __forceinline__ float ld(const __half* p, int64_t k, float ref) {
    return fmaf(__half2float(p[k]), HALF_UNSCALE, ref);
  }
  static __device__ __forceinline__ void st(__half* p, int64_t k, float v, float ref) {
    p[k] = __float2half_rn(__fsub_rn(v, ref) * HALF_SCALE);
  }
  static __device__ __forceinline__ __half enc(float v, float ref) { return __float2half_rn(__fsub_rn(v, ref) * HALF_SCALE); }
  static __device__ __forceinline__ float dec(__half v, float ref) { return fmaf(__half2float(v), HALF_UNSCALE, ref); }
  static __device__ __forceinline__ void ld2(const __half* p, int64_t j, float ra, float rb, float& a, float& b) {
    const __half2 v = __ldg(reinterpret_cast<const __half2*>(p + j));
    a = fmaf(__low2float(v), HALF_UNSCALE, ra);
    b = fmaf(__high2float(v), HALF_UNSCALE, rb);
  }
  static __device__ __forceinline__ void st2(__half* p, int64_t j, float a, float b, float ra, float rb) {
    *reinterpret_cast<__half2*>(p + j) = __floats2half2_rn(__fsub_rn(a, ra) * HALF_SCALE, __fsub_rn(b, rb) * HALF_SCALE);
  }
};
template <>
struct Pop<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t k, float ref) {
    return __fadd_rn(__bfloat162float(p[k]), ref);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, int64_t k, float v, float ref) {
    p[k] = __float2bfloat16_rn(__fsub_rn(v, ref));
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(float v, float ref) { return __float2bfloat16_rn(__fsub_rn(v, ref)); }
  static __device__ __forceinline__ float dec(__nv_bfloat16 v, float ref) { return __fadd_rn(__bfloat162float(v), ref); }
  static __device__ __forceinline__ void ld2(const __nv_bfloat16* p, int64_t j, float ra, float rb, float& a,
                                             float& b) {
    const __nv_bfloat162 v = __ldg(reinterpret_cast<const __nv_bfloat162*>(p + j));
    a = __fadd_rn(__low2float(v), ra);
    b = __fadd_rn(__high2float(v), rb);
  }
  static __device__ __forceinline__ void st2(__nv_bfloat16* p, int64_t j, float a, float b, float ra, float rb) {
    *reinterpret_cast<__nv_bfloat162*>(p + j) = __floats2bfloat162_rn(__fsub_rn(a, ra), __fsub_rn(b, rb));
  }
};

// ---------------------------------------------------------------------------
// Per-step constants.
enum { BC_MC = 0, BC_LLKC = 1, BC_VAVG = 2, BC_CONST = 3 };

struct Phys {
  double omega[2];   // 1 / tau
  double kF[2];      // 1 - 1 / (2 tau), the Guo prefactor of Eq. 4
  double G_AB;       // Eq. 5
  double G_s[2];     // Eq. 7
  double chi[2];     // Eq. 8
  double rho_s[2];   // constant solid densities
  double rho_ref[2]; // FP16/BF16 storage reference densities
  int bc, pairing, avg9;
  // Eq. 7 with the improved scheme's virtual densities, cross pairing and
  // G_As = G_Bs = G_AB: the solid neighbours then enter exactly like fluid
  // ones (the density plane holds rho~ there), so every node can take the
  // one-sum formula of a node without solid neighbours
  int uniform;
};

// The same constants in the arithmetic type of a kernel, converted once on
// the host (an FP32 kernel then does no FP64 conversions).
template <typename C>
struct PhysK {
  C omega[2], kF[2], G_AB, G_s[2], chi[2], rho_s[2], rho_ref[2];
  int bc, pairing, avg9, uniform;
};

template <typename C>
inline PhysK<C> kphys(const Phys& p) {
  PhysK<C> k;
  for (int s = 0; s < 2; ++s) {
    k.omega[s] = C(p.omega[s]);
    k.kF[s] = C(p.kF[s]);
    k.G_s[s] = C(p.G_s[s]);
    k.chi[s] = C(p.chi[s]);
    k.rho_s[s] = C(p.rho_s[s]);
    k.rho_ref[s] = C(p.rho_ref[s]);
  }
  k.G_AB = C(p.G_AB);
  k.bc = p.bc;
  k.pairing = p.pairing;
  k.avg9 = p.avg9;
  k.uniform = p.uniform;
  return k;
}

// sum_i w_i c_i q_i over the eight moving directions, as paired
// differences (q[0] unused).
template <typename C>
__device__ __forceinline__ void weighted_sum(const C q[9], C& sx, C& sy) {
  sx = (q[1] - q[3]) * C(1.0 / 9.0) + ((q[5] - q[7]) + (q[8] - q[6])) * C(1.0 / 36.0);
  sy = (q[2] - q[4]) * C(1.0 / 9.0) + ((q[5] - q[7]) + (q[6] - q[8])) * C(1.0 / 36.0);
}

// Interaction force on both components at a fluid node (Eq. 5 restricted to
// fluid neighbours plus Eq. 7). nbP[s][i] is the value of the density plane
// of component s at x + c_i (the density at fluid nodes, rho~ at interface-
// solid nodes under the improved scheme); fl holds the neighbour bits.
// Values at solid neighbours are only used under the improved scheme.
// BULK_FAST: take the short path when no neighbour is solid (callers that
// know their whole warp is bulk pass fl = 0; others pass false so that a
// warp does not split between the two paths). The general path splits the
// neighbour values by select into a fluid and a solid part and sums each
// with the bulk formula. With ph.uniform (see Phys) every node takes the
// short path.
template <typename C, bool BULK_FAST = true>
__device__ __forceinline__ void interaction_force(const PhysK<C>& ph, uint16_t fl, const C rho[2],
                                                  const C nbP[2][9], C F[2][2]) {
  const C G = ph.G_AB;
  if ((BULK_FAST && !(fl & NB_ANY)) || ph.uniform) {
    // bulk node: every neighbour is fluid, Eq. 5 over all eight
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C ax, ay;
      weighted_sum(nbP[1 - s], ax, ay);
      F[s][0] = -rho[s] * (G * ax);
      F[s][1] = -rho[s] * (G * ay);
    }
    return;
  }
  C ax[2], ay[2];                    // fluid-weighted sums per component
  C sx[2] = {0, 0}, sy[2] = {0, 0};  // solid-weighted sums (improved scheme)
  C qf[9], qs[9], b[9];
  qf[0] = qs[0] = b[0] = C(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const bool solid = fl & nb_bit(i);
      qf[i] = solid ? C(0) : nbP[s][i];
      qs[i] = solid ? nbP[s][i] : C(0);
    }
    weighted_sum(qf, ax[s], ay[s]);
    if (ph.bc == BC_VAVG) weighted_sum(qs, sx[s], sy[s]);
  }
#pragma unroll
  for (int i = 1; i < 9; ++i) b[i] = (fl & nb_bit(i)) ? C(1) : C(0);
  C vx, vy;  // sum_i w_i phi(x + c_i) c_i
  weighted_sum(b, vx, vy);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int o = 1 - s;
    // the component whose solid pseudopotential enters Eq. 7 (selects only
    // between compile-time indices so the arrays stay in registers)
    const bool self = ph.pairing != 0;
    const C rho_c = self ? rho[s] : rho[o];
    const C sx_c = self ? sx[s] : sx[o], sy_c = self ? sy[s] : sy[o];
    const C rs_c = self ? ph.rho_s[s] : ph.rho_s[o];
    C bx, by;
    if (ph.bc == BC_MC) {
      bx = vx;
      by = vy;
    } else if (ph.bc == BC_LLKC) {
      bx = rho_c * vx;
      by = rho_c * vy;
    } else if (ph.bc == BC_VAVG) {
      bx = sx_c;
      by = sy_c;
    } else {
      bx = rs_c * vx;
      by = rs_c * vy;
    }
    const C Gs = ph.G_s[s];
    F[s][0] = -rho[s] * (G * ax[o] + Gs * bx);
    F[s][1] = -rho[s] * (G * ay[o] + Gs * by);
  }
}

// Momentum sum_i f_i c_i of one component, as paired differences.
template <typename C>
__device__ __forceinline__ void momentum(const C f[9], C& jx, C& jy) {
  jx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
  jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
}

// rho = sum_i f_i (Eq. 3) as a balanced tree. The collision does not rely
// on rho being correctly rounded: it conserves mass through the rest
// population (see collide).
template <typename C>
__device__ __forceinline__ C density(const C f[9]) {
  return ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
}

// rho / 9 with one rounding: the product with the two-term split of 1/9.
// Multiplying by the rounded 1/9 alone makes every weight w_i too large by
// the same 7.5e-9 (FP32), so sum_i f^eq_i = rho (1 + 7.5e-9) and each
// collision would add that much mass at every node.
template <typename C>
__device__ __forceinline__ C rho_over_9(C rho);
template <>
__device__ __forceinline__ float rho_over_9<float>(float rho) {
  constexpr float HI = (float)(1.0 / 9.0);               // fl(1/9)
  constexpr float LO = (float)(1.0 / 9.0 - (double)HI);  // 1/9 - fl(1/9)
  return fmaf(rho, HI, rho * LO);
}
template <>
__device__ __forceinline__ double rho_over_9<double>(double rho) {
  return rho / 9.0;
}

// BGK relaxation towards Eq. 2 plus the Guo source of Eq. 4, in place:
//   f_i <- f_i + Delta_i,  Delta_i = omega (f^eq_i - f_i) + S_i,
// with f^eq_i - f_i evaluated as (rho w_i - f_i) + rho w_i p_i, where p_i =
// 3 c.u + 4.5 (c.u)^2 - 1.5 u^2 is the small part of Eq. 2's bracket, so the
// O(1) part of the bracket is never rounded, and S_i of Eq. 4 written as
// w_i (1 - 1/(2 tau)) [3 c.F - 3 u.F + 9 (c.u)(c.F)]. The moving populations
// take their increments and the rest population takes minus their sum:
// exactly what the method gives (sum_i Delta_i = 0 by Eqs. 2 and 4), and in
// floating point the mass of each component changes only by the rounding
// of the nine final additions, whatever the rounding of rho.
template <typename C>
__device__ __forceinline__ void collide(C f[2][9], const C rho[2], C ux, C uy, const C F[2][2],
                                        const C omega[2], const C kF[2]) {
  const C usq15 = C(1.5) * (ux * ux + uy * uy);
  C r9[2], r36[2], k9[2], k36[2], uF3[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    r9[s] = rho_over_9(rho[s]);
    r36[s] = C(0.25) * r9[s];  // exact
    k9[s] = kF[s] * C(1.0 / 9.0);
    k36[s] = kF[s] * C(1.0 / 36.0);
    uF3[s] = C(3) * (ux * F[s][0] + uy * F[s][1]);
  }
  C acc[2] = {0, 0};
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const C cu = C(cx_of(i)) * ux + C(cy_of(i)) * uy;
    const C p = cu * (C(3) + C(4.5) * cu) - usq15;
    const C cu9 = C(9) * cu;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C cF = C(cx_of(i)) * F[s][0] + C(cy_of(i)) * F[s][1];
      const C src = (i <= 4 ? k9[s] : k36[s]) * ((C(3) * cF - uF3[s]) + cu9 * cF);
      const C ri = i <= 4 ? r9[s] : r36[s];
      const C d = (ri - f[s][i]) + ri * p;
      const C delta = omega[s] * d + src;
      acc[s] += delta;
      f[s][i] = f[s][i] + delta;
    }
  }
  f[0][0] = f[0][0] - acc[0];
  f[1][0] = f[1][0] - acc[1];
}

// Halfway bounce-back done by the writer. When the upstream node x - c_i of
// fluid node x is solid, what x receives along c_i at the next step is its
// own post-collision f*_opp(i) (Sec. 2); it is stored in slot i of that solid
// node (and its periodic images), which no other node writes, so that every
// pull reads f*_i(x - c_i) without a test. ref[s][d] is the encoding
// reference of the node's value along c_d, so slot i takes ref[s][opp(i)].
template <typename T, typename C>
__device__ __forceinline__ void store_bounced(T* __restrict__ fo, const Geo& g, int x, int y, uint16_t fl,
                                              const C fv[2][9], const C ref[2][9]) {
  if (!(fl & NB_ANY)) return;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (!(fl & nb_bit(opp_of(i)))) continue;
    int sx = x - cx_of(i), sy = y - cy_of(i);
    if (g.per_x) sx = (sx + g.nx) % g.nx;
    if (g.per_y) sy = (sy + g.ny) % g.ny;
    const int ks = g.idx(sx, sy);
    const C a = fv[0][opp_of(i)], b = fv[1][opp_of(i)], ra = ref[0][opp_of(i)], rb = ref[1][opp_of(i)];
    Pop<T>::st2(fo, pslot(g, i, ks), a, b, ra, rb);
    for_ghost_images(g, sx, sy, [&](int kk) { Pop<T>::st2(fo, pslot(g, i, kk), a, b, ra, rb); });
  }
}

// store_bounced for a node that is not within GH + 1 of a periodic border:
// its solid neighbours are owned nodes without images, at padded index
// k - c_i.
template <typename T, typename C>
__device__ __forceinline__ void store_bounced_near(T* __restrict__ fo, const Geo& g, int k, uint16_t fl,
                                                   const C fv[2][9], const C ref[2][9]) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (!(fl & nb_bit(opp_of(i)))) continue;
    const int ks = k - cx_of(i) - cy_of(i) * g.px;
    Pop<T>::st2(fo, pslot(g, i, ks), fv[0][opp_of(i)], fv[1][opp_of(i)], ref[0][opp_of(i)], ref[1][opp_of(i)]);
  }
}

// Store the 18 post-collision populations of owned node (x, y) at padded
// index k, and at its periodic images.
template <typename T, typename C>
__device__ __forceinline__ void store_node(T* __restrict__ fo, const Geo& g, int x, int y, int k,
                                           const C fv[2][9], const C ref[2][9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) Pop<T>::st2(fo, pslot(g, i, k), fv[0][i], fv[1][i], ref[0][i], ref[1][i]);
  const bool img = (g.per_x && (x < GH || x >= g.nx - GH)) || (g.per_y && (y < GH || y >= g.ny - GH));
  if (img) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const C a = fv[0][i], b = fv[1][i], ra = ref[0][i], rb = ref[1][i];
      for_ghost_images(g, x, y, [&](int kk) { Pop<T>::st2(fo, pslot(g, i, kk), a, b, ra, rb); });
    }
  }
}

}  // namespace lbm
