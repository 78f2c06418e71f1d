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

// Per-node flag bits (uint16): bit 0 the node is solid; bit i (1..8) the
// neighbour x + c_i is solid; bit 9 interface-solid (a solid node with a
// fluid D2Q9 neighbour).
constexpr uint16_t F_SOLID = 1u;
constexpr uint16_t F_IFACE = 1u << 9;
__host__ __device__ constexpr uint16_t nb_bit(int i) { return uint16_t(1u << i); }

struct Geo {
  int nx, ny;      // owned nodes
  int px, py;      // padded pitch and rows
  int64_t plane;   // px * py
  int per_x, per_y;
  __host__ __device__ int idx(int x, int y) const { return (y + GH) * px + (x + GH); }
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
// Population storage. FP32/FP64 store f itself. FP16/BF16 store the
// deviation f - w_i rho_ref^sigma, which keeps the rest-state part exact and
// spends the 11/8 significand bits on what varies.
template <typename T>
struct Pop;
template <>
struct Pop<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float* p, int64_t k, float) { return p[k]; }
  static __device__ __forceinline__ void st(float* p, int64_t k, float v, float) { p[k] = v; }
};
template <>
struct Pop<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double* p, int64_t k, double) { return p[k]; }
  static __device__ __forceinline__ void st(double* p, int64_t k, double v, double) { p[k] = v; }
};
template <>
struct Pop<__half> {
  using C = float;
  static __device__ __forceinline__ float ld(const __half* p, int64_t k, float ref) {
    return __half2float(p[k]) + ref;
  }
  static __device__ __forceinline__ void st(__half* p, int64_t k, float v, float ref) {
    p[k] = __float2half_rn(v - ref);
  }
};
template <>
struct Pop<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t k, float ref) {
    return __bfloat162float(p[k]) + ref;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, int64_t k, float v, float ref) {
    p[k] = __float2bfloat16_rn(v - ref);
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
};

// Interaction force on both components at a fluid node (Eq. 5 restricted to
// fluid neighbours plus Eq. 7). nbP[s][i] is the value of the density plane
// of component s at x + c_i (the density at fluid nodes, rho~ at interface-
// solid nodes under the improved scheme); fl holds the neighbour bits.
template <typename C>
__device__ __forceinline__ void interaction_force(const Phys& ph, uint16_t fl, const C rho[2],
                                                  const C nbP[2][9], C F[2][2]) {
  C ax[2] = {0, 0}, ay[2] = {0, 0};  // fluid-weighted sums per component
  C sx[2] = {0, 0}, sy[2] = {0, 0};  // solid-weighted sums (improved scheme)
  C vx = 0, vy = 0;                  // sum_i w_i phi_i c_i
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const C w = w_of<C>(i);
    const bool solid = fl & nb_bit(i);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C wv = w * nbP[s][i];
      if (!solid) {
        if (cx_of(i)) ax[s] += cx_of(i) > 0 ? wv : -wv;
        if (cy_of(i)) ay[s] += cy_of(i) > 0 ? wv : -wv;
      } else {
        if (cx_of(i)) sx[s] += cx_of(i) > 0 ? wv : -wv;
        if (cy_of(i)) sy[s] += cy_of(i) > 0 ? wv : -wv;
      }
    }
    if (solid) {
      if (cx_of(i)) vx += cx_of(i) > 0 ? w : -w;
      if (cy_of(i)) vy += cy_of(i) > 0 ? w : -w;
    }
  }
  const C G = C(ph.G_AB);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int o = 1 - s;
    // the component whose solid pseudopotential enters Eq. 7 (selects only
    // between compile-time indices so the arrays stay in registers)
    const bool self = ph.pairing != 0;
    const C rho_c = self ? rho[s] : rho[o];
    const C sx_c = self ? sx[s] : sx[o], sy_c = self ? sy[s] : sy[o];
    const C rs_c = C(self ? ph.rho_s[s] : ph.rho_s[o]);
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
    const C Gs = C(ph.G_s[s]);
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

// Knuth's branch-free two-sum: s + e == a + b exactly.
template <typename C>
__device__ __forceinline__ C two_sum(C a, C b, C& e) {
  const C s = a + b;
  const C bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

// rho = sum_i f_i (Eq. 3). In FP32 the sum is compensated so that rho is
// (in practice) correctly rounded: the collision conserves mass to within
// the rounding of rho, and an uncompensated sum leaves a bias that builds up
// over thousands of steps.
template <typename C>
__device__ __forceinline__ C density(const C f[9]) {
  C e, err = 0;
  C s = two_sum(f[0], f[1], e);
  err += e;
#pragma unroll
  for (int i = 2; i < 9; ++i) {
    s = two_sum(s, f[i], e);
    err += e;
  }
  return s + err;
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
//   f_i <- f_i + omega (f^eq_i - f_i) + S_i,
// with f^eq_i - f_i evaluated as (rho w_i - f_i) + rho w_i p_i, where p_i =
// 3 c.u + 4.5 (c.u)^2 - 1.5 u^2 is the small part of Eq. 2's bracket. Each
// population then takes one rounding at its own magnitude (the final add),
// and the O(1) part of the bracket is never rounded.
template <typename C>
__device__ __forceinline__ void collide(C f[2][9], const C rho[2], C ux, C uy, const C F[2][2],
                                        const C omega[2], const C kF[2]) {
  const C usq15 = C(1.5) * (ux * ux + uy * uy);
  const C r9[2] = {rho_over_9(rho[0]), rho_over_9(rho[1])};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const C cu = C(cx_of(i)) * ux + C(cy_of(i)) * uy;
    const C k = i == 0 ? C(4) : (i <= 4 ? C(1) : C(0.25));  // w_i * 9, exact
    const C p = C(3) * cu + C(4.5) * cu * cu - usq15;
    const C w = w_of<C>(i);
    // w_i [3 (c_i - u) + 9 (c_i . u) c_i]; a common scale error of the weights cancels in sum_i S_i
    const C ex = w * (C(3) * (C(cx_of(i)) - ux) + C(9) * cu * C(cx_of(i)));
    const C ey = w * (C(3) * (C(cy_of(i)) - uy) + C(9) * cu * C(cy_of(i)));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C ri = k * r9[s];
      const C d = (ri - f[s][i]) + ri * p;
      const C src = kF[s] * (ex * F[s][0] + ey * F[s][1]);
      f[s][i] = f[s][i] + (omega[s] * d + src);
    }
  }
}

}  // namespace lbm
