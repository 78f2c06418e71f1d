// Kernels of the two-pass schedule and the auxiliary kernels (geometry,
// initialisation, moments, populations, mass). The stored state between
// steps is the post-collision population f*_i(x) at its source node; a step
// pulls f_i(x) = f*_i(x - c_i), or f*_{opp(i)}(x) when x - c_i is solid
// (halfway bounce-back, Sec. 2), which is the post-streaming distribution
// of Eq. 1, then collides it in place.
#pragma once

#include "lbm_common.cuh"

namespace lbm {

struct Planes {
  const void* f_in;   // 18 planes of the storage type
  void* f_out;
  void* P;            // 2 planes of the compute type: rho (fluid), rho~ (solid)
  const uint16_t* flags;
};

// Pull the post-streaming populations of both components at padded index k.
template <typename T, typename C = typename Pop<T>::C>
__device__ __forceinline__ void gather(const T* __restrict__ f, const Geo& g, int k, uint16_t fl,
                                       const C ref[2][9], C out[2][9]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int o = opp_of(i);
      const bool bounce = (i != 0) && (fl & nb_bit(o));
      const int src = bounce ? k : k - cx_of(i) - cy_of(i) * g.px;
      const int slot = bounce ? o : i;
      out[s][i] = Pop<T>::ld(f + (int64_t)(s * 9 + slot) * g.plane, src, bounce ? ref[s][o] : ref[s][i]);
    }
}

template <typename C>
__device__ __forceinline__ void make_refs(const Phys& ph, C ref[2][9]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 9; ++i) ref[s][i] = w_of<C>(i) * C(ph.rho_ref[s]);
}

// ---- K1: densities --------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_density(const T* __restrict__ f, typename Pop<T>::C* __restrict__ P,
                                                 const uint16_t* __restrict__ flags, Geo g, Phys ph) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  if (fl & F_SOLID) return;
  C ref[2][9];
  make_refs(ph, ref);
  C fv[2][9];
  gather<T>(f, g, k, fl, ref, fv);
  put_with_ghosts(P, g, x, y, density(fv[0]));
  put_with_ghosts(P + g.plane, g, x, y, density(fv[1]));
}

// ---- K2: virtual solid density of Eq. 8 over the interface-solid list -----
template <typename C>
__global__ void __launch_bounds__(128) k_virtual_density(C* __restrict__ P, const uint16_t* __restrict__ flags,
                                                         const int* __restrict__ list, int n, Geo g, Phys ph) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = list[t];
  const int reach = ph.avg9 ? 1 : 2;
  C num[2] = {0, 0}, den = 0;
  for (int dy = -reach; dy <= reach; ++dy)
    for (int dx = -reach; dx <= reach; ++dx) {
      if (!(dx | dy)) continue;
      const int m = k + dx + dy * g.px;
      if (flags[m] & F_SOLID) continue;
      const int r2 = dx * dx + dy * dy;
      C w;
      if (ph.avg9) {
        w = r2 == 1 ? C(1) / C(9) : C(1) / C(36);
      } else {  // D2Q25 weights printed after Eq. 8
        w = r2 == 1 ? C(4) / C(21)
                    : r2 == 2 ? C(4) / C(45)
                              : r2 == 4 ? C(1) / C(60) : r2 == 5 ? C(2) / C(315) : C(1) / C(5040);
      }
      num[0] += w * P[m];
      num[1] += w * P[g.plane + m];
      den += w;
    }
  const int y = k / g.px - GH, x = k % g.px - GH;
  put_with_ghosts(P, g, x, y, C(ph.chi[0]) * num[0] / den);
  put_with_ghosts(P + g.plane, g, x, y, C(ph.chi[1]) * num[1] / den);
}

// Read the density plane at the 8 neighbours of padded index k.
template <typename C>
__device__ __forceinline__ void neighbour_P(const C* __restrict__ P, const Geo& g, int k, C nbP[2][9]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    nbP[s][0] = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) nbP[s][i] = __ldg(P + s * g.plane + k + cx_of(i) + cy_of(i) * g.px);
  }
}

// ---- K3: fused force + collide + stream (pull) ---------------------------
// MODE 0: write post-collision populations. MODE 1: write moments (rho, u)
// instead. MODE 2: write forces.
template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_collide(const T* __restrict__ f, T* __restrict__ fo,
                                                 const typename Pop<T>::C* __restrict__ P,
                                                 const uint16_t* __restrict__ flags, Geo g, Phys ph,
                                                 double* __restrict__ out) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  const int64_t n = (int64_t)y * g.nx + x;
  const int64_t N = (int64_t)g.nx * g.ny;
  if (fl & F_SOLID) {
    if (MODE == 1) {
      out[n] = 0; out[N + n] = 0; out[2 * N + n] = 0; out[3 * N + n] = 0;
    } else if (MODE == 2) {
      out[n] = 0; out[N + n] = 0; out[2 * N + n] = 0; out[3 * N + n] = 0;
    }
    return;
  }
  C ref[2][9];
  make_refs(ph, ref);
  C fv[2][9];
  gather<T>(f, g, k, fl, ref, fv);
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
    out[n] = rho[0];
    out[N + n] = rho[1];
    out[2 * N + n] = ux;
    out[3 * N + n] = uy;
    return;
  }
  if (MODE == 2) {
    out[n] = F[0][0];
    out[N + n] = F[0][1];
    out[2 * N + n] = F[1][0];
    out[3 * N + n] = F[1][1];
    return;
  }
  const C omega[2] = {C(ph.omega[0]), C(ph.omega[1])};
  const C kF[2] = {C(ph.kF[0]), C(ph.kF[1])};
  collide(fv, rho, ux, uy, F, omega, kF);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      T* plane = fo + (int64_t)(s * 9 + i) * g.plane;
      const C v = fv[s][i], r = ref[s][i];
      Pop<T>::st(plane, k, v, r);
      for_ghost_images(g, x, y, [&](int kk) { Pop<T>::st(plane, kk, v, r); });
    }
}

// ---- post-streaming populations out / in ---------------------------------
template <typename T>
__global__ void k_get_populations(const T* __restrict__ f, const uint16_t* __restrict__ flags, Geo g,
                                  Phys ph, double* __restrict__ out) {
  using C = typename Pop<T>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.nx) return;
  const int k = g.idx(x, y);
  const uint16_t fl = flags[k];
  const int64_t n = (int64_t)y * g.nx + x, N = (int64_t)g.nx * g.ny;
  C ref[2][9];
  make_refs(ph, ref);
  C fv[2][9];
  if (fl & F_SOLID) {
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 9; ++i) fv[s][i] = 0;
  } else {
    gather<T>(f, g, k, fl, ref, fv);
  }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 9; ++i) out[(s * 9 + i) * N + n] = fv[s][i];
}

// Wrapped compact index of (x, y) for caller arrays [ny][nx].
__device__ __forceinline__ int64_t wrap_compact(const Geo& g, int x, int y) {
  x = (x + g.nx) % g.nx;
  y = (y + g.ny) % g.ny;
  return (int64_t)y * g.nx + x;
}

// State from post-streaming populations: the stored f*_j(y) is the value
// that streaming delivers to (y + c_j, j), or to (y, opp(j)) when y + c_j
// is solid. SRC 0: read populations (d_in [2][9][ny][nx]). SRC 1: the
// populations are the equilibrium of Eq. 2 from rho/u arrays.
template <typename T, int SRC>
__global__ void k_set_state(T* __restrict__ f, const uint16_t* __restrict__ flags, Geo g, Phys ph,
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
  C ref[2][9];
  make_refs(ph, ref);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const bool bounce = (j != 0) && (fl & nb_bit(j));
      const int dx = bounce ? 0 : cx_of(j), dy = bounce ? 0 : cy_of(j);
      const int slot = bounce ? opp_of(j) : j;
      const int64_t m = wrap_compact(g, x + dx, y + dy);
      double v;
      if (SRC == 0) {
        v = fin[(s * 9 + slot) * N + m];
      } else {
        const double r = s ? rB[m] : rA[m];
        const double vx = ux ? ux[m] : 0.0, vy = uy ? uy[m] : 0.0;
        const double cu = cx_of(slot) * vx + cy_of(slot) * vy;
        v = r * w_of<double>(slot) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (vx * vx + vy * vy));
      }
      const C cv = C(v), r = ref[s][j];
      T* plane = f + (int64_t)(s * 9 + j) * g.plane;
      Pop<T>::st(plane, k, cv, r);
      for_ghost_images(g, x, y, [&](int kk) { Pop<T>::st(plane, kk, cv, r); });
    }
}

// ---- FP64 mass: per-block partial sums, then one fixed-order final sum ----
template <typename T>
__global__ void __launch_bounds__(256) k_mass_partial(const T* __restrict__ f, const uint16_t* __restrict__ flags,
                                                      Geo g, Phys ph, double* __restrict__ partial) {
  using C = typename Pop<T>::C;
  __shared__ double red[2][256 / 32];
  C ref[2][9];
  make_refs(ph, ref);
  double acc[2] = {0.0, 0.0};
  const int64_t N = (int64_t)g.nx * g.ny;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(n / g.nx), x = (int)(n % g.nx);
    const int k = g.idx(x, y);
    if (flags[k] & F_SOLID) continue;
    for (int s = 0; s < 2; ++s) {
      double r = 0.0;
      for (int i = 0; i < 9; ++i) r += (double)Pop<T>::ld(f + (int64_t)(s * 9 + i) * g.plane, k, ref[s][i]);
      acc[s] += r;
    }
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

__global__ void k_mass_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  // one warp per component, fixed lane/stride order, then a fixed shuffle tree
  const int s = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (s >= 2) return;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += partial[2 * b + s];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[s] = v;
}

}  // namespace lbm
