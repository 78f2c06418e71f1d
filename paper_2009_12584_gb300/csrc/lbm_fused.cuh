// Single-pass step: one kernel per time step.
//
// The density plane is double-buffered: step t reads rho(t) (and the
// populations f*(t)) and writes f*(t+1) together with rho(t+1), so no
// separate density pass runs. Each CTA owns a strip of W = NT - 2 columns and
// a segment of rows, and sweeps its rows upwards with one thread per column:
//   - it pulls f_i(x) = f*_i(x - c_i, t) straight from global memory (halfway
//     bounce-back is folded into the state, see store_bounced), takes rho(t)
//     of the node and its neighbours from the density plane, and the virtual
//     densities of Eq. 8 of its solid neighbours from a ring in shared memory
//     that is filled three rows ahead;
//   - it evaluates the forces of Eq. 5 and Eq. 7, the velocity of Eq. 3,
//     collides (Eq. 1, 2, 4), stores f*(t+1), and keeps the row in a 4-row
//     ring in shared memory;
//   - one row later the ring holds f*(t+1) around the previous row, whose
//     densities rho(t+1) (Eq. 3) it then writes for the next step.
// The strip also computes (but does not store) one column on each side and
// one row below and above its segment, so that its ring is complete. Solid
// interiors are never read; one barrier per row.
#pragma once

#include "lbm.h"
#include "lbm_common.cuh"

namespace lbm {

template <typename T, int NT>
struct StreamCfg {
  using C = typename Pop<T>::C;
  static constexpr int W = NT - 2;   // owned columns per strip
  static constexpr int RC = NT + 2;  // virtual-density ring columns: x0 - 2 ... x0 + W + 1
  static constexpr int NO = 4;       // f*(t+1) ring rows: y - 2 ... y + 1
  static constexpr int NR = 5;       // virtual-density ring rows: y - 1 ... y + 3
  static constexpr size_t O_BYTES = (size_t)NO * 18 * NT * sizeof(T);
  static constexpr size_t R_BYTES = (size_t)NR * 2 * RC * sizeof(C);
  static constexpr size_t SMEM = O_BYTES + R_BYTES;
  static_assert(O_BYTES % 16 == 0, "ring alignment");
};

template <int N>
__device__ __forceinline__ int ring(int r) {
  return (r + 64 * N) % N;  // rows are >= -GH > -64 N
}

// Weight of neighbour (dx, dy) in the average of Eq. 8: the D2Q25 set
// printed after Eq. 8, or the D2Q9 set (the variant the paper compares).
template <typename C, bool AVG9>
__host__ __device__ constexpr C avg_weight(int dx, int dy) {
  return AVG9 ? ((dx * dx + dy * dy) == 1 ? C(1) / C(9) : C(1) / C(36))
              : ((dx * dx + dy * dy) == 1   ? C(4) / C(21)
                 : (dx * dx + dy * dy) == 2 ? C(4) / C(45)
                 : (dx * dx + dy * dy) == 4 ? C(1) / C(60)
                 : (dx * dx + dy * dy) == 5 ? C(2) / C(315)
                                            : C(1) / C(5040));
}

template <typename T, bool VAVG, bool AVG9, int NT>
__global__ void __launch_bounds__(NT, 4) k_stream(const T* __restrict__ f, T* __restrict__ fo,
                                               const typename Pop<T>::C* __restrict__ P,
                                               typename Pop<T>::C* __restrict__ Po,
                                               const uint16_t* __restrict__ flags, Geo g,
                                               PhysK<typename Pop<T>::C> ph, int H) {
  using Cfg = StreamCfg<T, NT>;
  using C = typename Cfg::C;
  constexpr int W = Cfg::W, RC = Cfg::RC, NO = Cfg::NO, NR = Cfg::NR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* so = (T*)smem_raw;                           // [NO][18][NT] f*(t+1), storage encoding
  C* srt = (C*)(smem_raw + Cfg::O_BYTES);         // [NR][2][RC] rho~ at interface-solid cells

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * W;
  const int xc = x0 - 1 + tid;  // the column this thread computes
  const int y0 = blockIdx.y * H;
  const int y_end = min(g.ny, y0 + H);
  const bool own = tid >= 1 && tid <= W && xc < g.nx;
  const bool computable = xc <= g.nx;  // x0 - 1 ... nx: ghost column nx images column 0
  const int64_t PL = g.plane;

  C ref[2][9];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int i = 0; i < 9; ++i) ref[s][i] = w_of<C>(i) * ph.rho_ref[s];

  // rho~ of Eq. 8 at the interface-solid cells of row r, columns x0-2 ... x0+W+1
  auto compute_rt_row = [&](int r) {
    constexpr int REACH = AVG9 ? 1 : 2;
    C* dst = srt + ring<NR>(r) * 2 * RC;
    for (int rc = tid; rc < RC; rc += NT) {
      const int x = x0 - 2 + rc;
      C v0 = 0, v1 = 0;
      if (x <= g.nx + 1) {
        const int k = g.idx(x, r);
        if (flags[k] & F_IFACE) {
          C num0 = 0, num1 = 0, den = 0;
#pragma unroll
          for (int dy = -REACH; dy <= REACH; ++dy)
#pragma unroll
            for (int dx = -REACH; dx <= REACH; ++dx) {
              if (dx == 0 && dy == 0) continue;
              const int m = k + dx + dy * g.px;
              if (__ldg(flags + m) & F_SOLID) continue;
              const C w = avg_weight<C, AVG9>(dx, dy);
              num0 += w * __ldg(P + m);
              num1 += w * __ldg(P + PL + m);
              den += w;
            }
          v0 = ph.chi[0] * num0 / den;
          v1 = ph.chi[1] * num1 / den;
        }
      }
      dst[rc] = v0;
      dst[RC + rc] = v1;
    }
  };

  // force, collision and stores of row y at column xc; keeps f*(t+1) in the ring
  auto output_row = [&](int y) {
    if (!computable) return;
    const int k = g.idx(xc, y);
    const uint16_t fl = flags[k];
    if (fl & F_SOLID) return;
    C fv[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i)
        fv[s][i] = Pop<T>::ld(f + (s * 9 + i) * PL, k - cx_of(i) - cy_of(i) * g.px, ref[s][i]);
    const C rho[2] = {__ldg(P + k), __ldg(P + PL + k)};
    C nbP[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      nbP[s][0] = 0;
#pragma unroll
      for (int i = 1; i < 9; ++i) nbP[s][i] = __ldg(P + s * PL + k + cx_of(i) + cy_of(i) * g.px);
    }
    if (VAVG && (fl & NB_ANY)) {
      // solid neighbours: rho~ from the ring (ring column of x + c_i is tid + 1 + c_x)
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if (fl & nb_bit(i)) {
          const C* rr = srt + ring<NR>(y + cy_of(i)) * 2 * RC + tid + 1 + cx_of(i);
          nbP[0][i] = rr[0];
          nbP[1][i] = rr[RC];
        }
    }
    C F[2][2];
    interaction_force(ph, fl, rho, nbP, F);
    C jxA, jyA, jxB, jyB;
    momentum(fv[0], jxA, jyA);
    momentum(fv[1], jxB, jyB);
    const C inv = C(1) / (rho[0] + rho[1]);
    const C ux = ((jxA + jxB) + C(0.5) * (F[0][0] + F[1][0])) * inv;
    const C uy = ((jyA + jyB) + C(0.5) * (F[0][1] + F[1][1])) * inv;
    collide(fv, rho, ux, uy, F, ph.omega, ph.kF);
    T* orow = so + ring<NO>(y) * 18 * NT + tid;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) orow[(s * 9 + i) * NT] = Pop<T>::enc(fv[s][i], ref[s][i]);
    if (own && y >= y0 && y < y_end) {
      store_node(fo, g, xc, y, k, fv, ref);
      store_bounced(fo, g, xc, y, fl, fv, ref);
    }
  };

  // rho(t+1) of row r at an owned column, from the ring (rows r-1 ... r+1)
  auto rho_next_row = [&](int r) {
    if (!own || r < y0 || r >= y_end) return;
    const int k = g.idx(xc, r);
    const uint16_t fl = flags[k];
    if (fl & F_SOLID) return;
    const T* b0 = so + ring<NO>(r) * 18 * NT + tid;
    const T* bm = so + ring<NO>(r - 1) * 18 * NT + tid;
    const T* bp = so + ring<NO>(r + 1) * 18 * NT + tid;
    C fv[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int o = opp_of(i);
        const bool bounce = (i != 0) && (fl & nb_bit(o));
        const T* rb = cy_of(i) > 0 ? bm : (cy_of(i) < 0 ? bp : b0);  // row of x - c_i
        const T raw = bounce ? b0[(s * 9 + o) * NT] : rb[(s * 9 + i) * NT - cx_of(i)];
        fv[s][i] = Pop<T>::dec(raw, ref[s][i]);
      }
    put_with_ghosts(Po, g, xc, r, density(fv[0]));
    put_with_ghosts(Po + PL, g, xc, r, density(fv[1]));
  };

  if (VAVG)
    for (int r = y0 - 2; r <= y0 + 1; ++r) compute_rt_row(r);
  __syncthreads();
  for (int y = y0 - 1; y <= y_end; ++y) {
    output_row(y);  // writes ring row y; reads rho~ rows y-1 ... y+1
    __syncthreads();
    rho_next_row(y - 1);  // reads ring rows y-2 ... y
    if (VAVG && y + 3 <= y_end + 1) compute_rt_row(y + 3);  // into the slot of row y-2
  }
}

constexpr int STREAM_NT = 128;

template <typename T>
inline bool fused_supported(const Geo&, const Phys&) {
  return true;
}

template <typename T, bool VAVG, bool AVG9>
inline lbm_status launch_stream_t(const Geo& g, const Phys& ph, const T* fin, T* fout,
                                  const typename Pop<T>::C* P, typename Pop<T>::C* Po, const uint16_t* flags,
                                  int num_sms, cudaStream_t stream) {
  using Cfg = StreamCfg<T, STREAM_NT>;
  auto kern = k_stream<T, VAVG, AVG9, STREAM_NT>;
  static bool configured[64] = {};  // the attribute is set per function and device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LBM_ERR_CUDA;
  if (!configured[dev]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess)
      return LBM_ERR_CUDA;
    configured[dev] = true;
  }
  const int nstrips = (g.nx + Cfg::W - 1) / Cfg::W;
  int per_sm = (int)((220 * 1024) / (Cfg::SMEM + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  const int target = 4 * num_sms * per_sm;  // about four waves of CTAs
  int nseg = (target + nstrips - 1) / nstrips;
  int H = (g.ny + nseg - 1) / nseg;
  if (H < 16) H = 16;
  nseg = (g.ny + H - 1) / H;
  kern<<<dim3(nstrips, nseg), STREAM_NT, Cfg::SMEM, stream>>>(fin, fout, P, Po, flags, g,
                                                               kphys<typename Pop<T>::C>(ph), H);
  return LBM_OK;
}

template <typename T>
inline lbm_status launch_fused(const Geo& g, const Phys& ph, const T* fin, T* fout, const typename Pop<T>::C* P,
                               typename Pop<T>::C* Po, const uint16_t* flags, int num_sms, cudaStream_t stream) {
  if (ph.bc == BC_VAVG) {
    if (ph.avg9) return launch_stream_t<T, true, true>(g, ph, fin, fout, P, Po, flags, num_sms, stream);
    return launch_stream_t<T, true, false>(g, ph, fin, fout, P, Po, flags, num_sms, stream);
  }
  return launch_stream_t<T, false, false>(g, ph, fin, fout, P, Po, flags, num_sms, stream);
}

}  // namespace lbm
