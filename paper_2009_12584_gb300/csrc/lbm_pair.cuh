// The fluid-node update of the two-pass schedule for the FP32 compute type
// (FP32, FP16 and BF16 storage) with the two components carried as one
// float2 pair (A in .x, B in .y). Components A and B go through the same
// arithmetic with their own rho, F, tau (Eqs. 1-5, 7 of arXiv:2009.12584),
// so each pair of scalar operations becomes one paired FP32 instruction
// (add/mul/fma .f32x2 of sm_100-family GPUs), each lane rounded as its
// scalar operation.
#pragma once

#include "lbm_common.cuh"
#include "lbm_geometry.cuh"

namespace lbm {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 sel2(bool p, float2 a, float2 b) { return p ? a : b; }

// sum_i w_i c_i q_i over the eight moving directions for both components.
__device__ __forceinline__ void weighted_sum2(const float2 q[9], float2& sx, float2& sy) {
  const float2 d57 = sub2(q[5], q[7]), d86 = sub2(q[8], q[6]);
  sx = fma2(sub2(q[1], q[3]), f2(1.0f / 9.0f), mul2(add2(d57, d86), f2(1.0f / 36.0f)));
  sy = fma2(sub2(q[2], q[4]), f2(1.0f / 9.0f), mul2(sub2(d57, d86), f2(1.0f / 36.0f)));
}

// Eq. 5 (fluid neighbours) plus Eq. 7 for both components. q[i]: the
// density plane (rho, or rho~ at interface-solid nodes) at x + c_i. With
// ph.uniform (the improved scheme with G_As = G_Bs = G_AB and Eq. 7's cross
// pairing) both sums are one weighted sum over the plane, the bulk formula.
template <bool GENERAL>
__device__ __forceinline__ void interaction_force2(const PhysK<float>& ph, uint16_t fl, float2 rho,
                                                   const float2 q[9], float2& Fx, float2& Fy) {
  const float2 G = f2(ph.G_AB);
  if (!GENERAL || ph.uniform) {
    float2 ax, ay;
    weighted_sum2(q, ax, ay);
    // component s feels the other component's density
    Fx = mul2(neg2(rho), mul2(G, swap2(ax)));
    Fy = mul2(neg2(rho), mul2(G, swap2(ay)));
    return;
  }
  float2 qf[9], qs[9];
  float b[9];
  qf[0] = qs[0] = f2(0.0f);
  b[0] = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const bool solid = fl & nb_bit(i);
    qf[i] = sel2(solid, f2(0.0f), q[i]);
    qs[i] = sel2(solid, q[i], f2(0.0f));
    b[i] = solid ? 1.0f : 0.0f;
  }
  float2 ax, ay;
  weighted_sum2(qf, ax, ay);
  float vx, vy;  // sum_i w_i phi(x + c_i) c_i
  weighted_sum(b, vx, vy);
  // the component whose solid pseudopotential enters Eq. 7: the other one
  // (cross pairing) or the same one (self pairing)
  const bool self = ph.pairing != 0;
  float2 bx, by;
  if (ph.bc == BC_MC) {
    bx = f2(vx);
    by = f2(vy);
  } else if (ph.bc == BC_LLKC) {
    const float2 rc = self ? rho : swap2(rho);
    bx = mul2(rc, f2(vx));
    by = mul2(rc, f2(vy));
  } else if (ph.bc == BC_VAVG) {
    float2 sx, sy;
    weighted_sum2(qs, sx, sy);
    bx = self ? sx : swap2(sx);
    by = self ? sy : swap2(sy);
  } else {
    const float2 rs = self ? f2(ph.rho_s[0], ph.rho_s[1]) : f2(ph.rho_s[1], ph.rho_s[0]);
    bx = mul2(rs, f2(vx));
    by = mul2(rs, f2(vy));
  }
  const float2 Gs = f2(ph.G_s[0], ph.G_s[1]);
  const float2 nrho = neg2(rho);
  Fx = mul2(nrho, fma2(G, swap2(ax), mul2(Gs, bx)));
  Fy = mul2(nrho, fma2(G, swap2(ay), mul2(Gs, by)));
}

// rho / 9 with one rounding per component (the two-term split of 1/9).
__device__ __forceinline__ float2 rho_over_9_2(float2 rho) {
  constexpr float HI = (float)(1.0 / 9.0);
  constexpr float LO = (float)(1.0 / 9.0 - (double)HI);
  return fma2(rho, f2(HI), mul2(rho, f2(LO)));
}

// BGK towards Eq. 2 plus the Guo source of Eq. 4, in the form of collide()
// in lbm_common.cuh: moving populations take Delta_i = omega (f^eq_i - f_i)
// + S_i with f^eq_i - f_i = (rho w_i - f_i) + rho w_i p_i, and the rest
// population takes minus their sum (mass conserved per node).
__device__ __forceinline__ void collide2(float2 f[9], float2 rho, float ux, float uy, float2 Fx, float2 Fy,
                                         const PhysK<float>& ph) {
  const float usq15 = 1.5f * (ux * ux + uy * uy);
  const float2 r9 = rho_over_9_2(rho);
  const float2 r36 = mul2(f2(0.25f), r9);  // exact
  const float2 om = f2(ph.omega[0], ph.omega[1]);
  const float2 k9 = mul2(f2(ph.kF[0], ph.kF[1]), f2(1.0f / 9.0f));
  const float2 k36 = mul2(f2(ph.kF[0], ph.kF[1]), f2(1.0f / 36.0f));
  const float2 uF3 = mul2(f2(3.0f), fma2(f2(ux), Fx, mul2(f2(uy), Fy)));
  float2 acc = f2(0.0f);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const float cu = float(cx_of(i)) * ux + float(cy_of(i)) * uy;
    const float p = cu * (3.0f + 4.5f * cu) - usq15;
    const float cu9 = 9.0f * cu;
    // c_i . F for both components (c_i components are -1, 0, 1)
    float2 cF;
    if (cx_of(i) == 0)
      cF = cy_of(i) > 0 ? Fy : neg2(Fy);
    else if (cy_of(i) == 0)
      cF = cx_of(i) > 0 ? Fx : neg2(Fx);
    else {
      const float2 a = cx_of(i) > 0 ? Fx : neg2(Fx);
      cF = cy_of(i) > 0 ? add2(a, Fy) : sub2(a, Fy);
    }
    const float2 src = mul2(i <= 4 ? k9 : k36, fma2(f2(cu9), cF, sub2(mul2(f2(3.0f), cF), uF3)));
    const float2 ri = i <= 4 ? r9 : r36;
    const float2 d = fma2(ri, f2(p), sub2(ri, f[i]));
    const float2 delta = fma2(om, d, src);
    acc = add2(acc, delta);
    f[i] = add2(f[i], delta);
  }
  f[0] = sub2(f[0], acc);
}

// Force, velocity and collision of one fluid node (Eqs. 1-5, 7): fp holds
// the pulled populations f_i of both components on entry and f*_i on exit;
// q[i] the density plane at x + c_i. GENERAL: the node may have solid
// neighbours (fl holds the neighbour bits); a node without any gets the
// same result on either path. Returns rho of both components and, in
// ux_out, uy_out, the velocity u of Eq. 3 the collision used.
template <bool GENERAL>
__device__ __forceinline__ float2 update_pair(float2 fp[9], const float2 q[9], uint16_t fl,
                                              const PhysK<float>& ph, float& ux_out, float& uy_out) {
  const float2 rho = add2(add2(add2(fp[0], add2(fp[1], fp[3])), add2(fp[2], fp[4])),
                          add2(add2(fp[5], fp[7]), add2(fp[6], fp[8])));
  float2 Fx, Fy;
  interaction_force2<GENERAL>(ph, fl, rho, q, Fx, Fy);
  // momentum of each component as paired differences, then u of Eq. 3
  const float2 d57 = sub2(fp[5], fp[7]), d86 = sub2(fp[8], fp[6]);
  const float2 jx = add2(sub2(fp[1], fp[3]), add2(d57, d86));
  const float2 jy = add2(sub2(fp[2], fp[4]), sub2(d57, d86));
  const float inv = 1.0f / (rho.x + rho.y);
  const float ux = ((jx.x + jx.y) + 0.5f * (Fx.x + Fx.y)) * inv;
  const float uy = ((jy.x + jy.y) + 0.5f * (Fy.x + Fy.y)) * inv;
  collide2(fp, rho, ux, uy, Fx, Fy, ph);
  ux_out = ux;
  uy_out = uy;
  return rho;
}

}  // namespace lbm
