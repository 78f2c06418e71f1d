// On-device diagnostics of Secs. 3-4 of arXiv:2009.12584 (declared with
// lbm_diagnostics in include/lbm.h): reductions over the moments that the
// eval pass writes to the staging area (rho^A, rho^B, u_x, u_y as double
// [ny][nx] arrays), in FP64 and a fixed order.
#pragma once

#include "lbm_common.cuh"

namespace lbm {

constexpr int DIAG_BLOCKS = 256;
constexpr int DIAG_THREADS = 256;
// reduced quantities: 0 sum w, 1 sum w x, 2 sum w y, 3 sum w u_x,
// 4 sum w u_y, 5 crossings kept, 6..13 the Kasa sums over kept crossings
// (x, y, xx, yy, xy, x r, y r, r with r = x^2 + y^2, coordinates relative to
// the grid centre), 14 max |u|^2 over finite nodes, 15 fluid nodes whose
// rho^A, rho^B or u is not finite, 16 bridge radius (final kernel only)
constexpr int DIAG_NQ = 17;
constexpr int DIAG_NRED = 16;  // quantities reduced over nodes (0..15)

struct DiagArgs {
  double level, rho_out;
  double wx, wy;    // wall point
  double nx_, ny_;  // wall normal towards the fluid
  double exclude;
  double box[4];
  bool use_box;
  double ox, oy;    // origin of the fit coordinates
  int bridge_x, bridge_y0;
};

__device__ __forceinline__ int dsgn(double v) { return (v > 0.0) - (v < 0.0); }

// One contour point: drop it near the wall or outside the box, else add it
// to the fit sums.
__device__ __forceinline__ void diag_point(const DiagArgs& a, double px, double py, double acc[DIAG_NRED]) {
  const double dist = (px - a.wx) * a.nx_ + (py - a.wy) * a.ny_;
  if (!(dist > a.exclude)) return;
  if (a.use_box && !(px >= a.box[0] && px <= a.box[1] && py >= a.box[2] && py <= a.box[3])) return;
  const double x = px - a.ox, y = py - a.oy, r = x * x + y * y;
  acc[5] += 1.0;
  acc[6] += x;
  acc[7] += y;
  acc[8] += x * x;
  acc[9] += y * y;
  acc[10] += x * y;
  acc[11] += x * r;
  acc[12] += y * r;
  acc[13] += r;
}

// Per-block partial sums (and max) over a fixed grid-stride assignment of
// the owned nodes; st = [rho^A | rho^B | u_x | u_y], each nx * ny.
static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(const double* __restrict__ st,
                                                                      const uint16_t* __restrict__ flags, Geo g,
                                                                      DiagArgs a, double* __restrict__ partial) {
  __shared__ double red[DIAG_THREADS / 32][DIAG_NRED];
  double acc[DIAG_NRED];
#pragma unroll
  for (int q = 0; q < DIAG_NRED; ++q) acc[q] = 0.0;
  const int64_t N = (int64_t)g.nx * g.ny;
  for (int64_t n = (int64_t)blockIdx.x * DIAG_THREADS + threadIdx.x; n < N; n += (int64_t)DIAG_BLOCKS * DIAG_THREADS) {
    const int y = (int)(n / g.nx), x = (int)(n % g.nx);
    const int k = g.idx(x, y);
    if (flags[k] & F_SOLID) continue;
    const double rA = st[n], ux = st[2 * N + n], uy = st[3 * N + n];
    if (!isfinite(rA) || !isfinite(st[N + n]) || !isfinite(ux) || !isfinite(uy)) {
      acc[15] += 1.0;  // counted, and left out of every other sum
      continue;
    }
    const double w = fmax(rA - a.rho_out, 0.0);
    acc[0] += w;
    acc[1] += w * x;
    acc[2] += w * y;
    acc[3] += w * ux;
    acc[4] += w * uy;
    acc[14] = fmax(acc[14], ux * ux + uy * uy);
    const double d = rA - a.level;
    if (x + 1 < g.nx && !(flags[k + 1] & F_SOLID)) {  // edge to (x + 1, y)
      const double e = st[n + 1] - a.level;
      if (dsgn(d) != dsgn(e) && d != e) diag_point(a, x + d / (d - e), (double)y, acc);
    }
    if (y + 1 < g.ny && !(flags[k + g.px] & F_SOLID)) {  // edge to (x, y + 1)
      const double e = st[n + g.nx] - a.level;
      if (dsgn(d) != dsgn(e) && d != e) diag_point(a, (double)x, y + d / (d - e), acc);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < DIAG_NRED; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, v, o);
      v = q == 14 ? fmax(v, t) : v + t;
    }
    if (lane == 0) red[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_NRED) {
    const int q = threadIdx.x;
    double v = red[0][q];
    for (int w = 1; w < DIAG_THREADS / 32; ++w) v = q == 14 ? fmax(v, red[w][q]) : v + red[w][q];
    partial[(size_t)blockIdx.x * DIAG_NRED + q] = v;
  }
}

// Blocks in a fixed order, then the bridge radius by a scan of one column.
static __global__ void k_diag_final(const double* __restrict__ partial, const double* __restrict__ st, Geo g,
                                    DiagArgs a, double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q < DIAG_NRED) {
    double v = partial[q];
    for (int b = 1; b < DIAG_BLOCKS; ++b) {
      const double t = partial[(size_t)b * DIAG_NRED + q];
      v = q == 14 ? fmax(v, t) : v + t;
    }
    out[q] = v;
  }
  if (q == 0) {
    double br = 0.0;
    if (a.bridge_x >= 0) {
      const double* col = st + a.bridge_x;  // rho^A, stride nx
      int y = a.bridge_y0;
      if (col[(int64_t)y * g.nx] >= a.level) {
        while (y + 1 < g.ny && col[(int64_t)(y + 1) * g.nx] >= a.level) ++y;
        if (y + 1 >= g.ny) {
          br = g.ny - (a.bridge_y0 - 0.5);
        } else {
          const double c0 = col[(int64_t)y * g.nx], c1 = col[(int64_t)(y + 1) * g.nx];
          br = y + (c0 - a.level) / (c0 - c1) - (a.bridge_y0 - 0.5);
        }
      }
    }
    out[16] = br;
  }
}

}  // namespace lbm
