// C ABI of the GB300 lattice-Boltzmann library (declared in include/lbm.h):
// context, workspace carve-up, argument checks and kernel launches.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "lbm_diag.cuh"
#include "lbm_internal.cuh"

using namespace lbm;

namespace {

size_t elem_size(int storage) {
  switch (storage) {
    case LBM_STORE_FP32: return 4;
    case LBM_STORE_FP64: return 8;
    case LBM_STORE_FP16: return 2;
    case LBM_STORE_BF16: return 2;
  }
  return 0;
}
size_t compute_size(int storage) { return storage == LBM_STORE_FP64 ? 8 : 4; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool make_geo(const lbm_params* p, Geo* g) {
  if (p->nx < 4 || p->ny < 4) return false;
  g->nx = p->nx;
  g->ny = p->ny;
  g->px = (int)align_up((size_t)LP + p->nx + GH, 32);
  g->py = p->ny + 2 * GH;
  g->plane = (int64_t)g->px * g->py;
  g->per_x = p->periodic_x ? 1 : 0;
  g->per_y = p->periodic_y ? 1 : 0;
  return g->plane < (int64_t(1) << 30);  // list entries carry two tag bits
}

struct Layout {
  size_t f, P, U, flags, list, imask, flist, tent, toff, tcnt, twork, hent, hoff, hcnt, hmask, counts, small, partial, mass,
      smask, stage, dpart, total;
};

// Whether a context keeps the per-tile lists of the tiled schedule (the
// schedule AUTO picks for 4- and 8-byte storage; 16-bit storage runs it
// only when asked for).
bool uses_tiles(const lbm_params* p) {
  const bool wide = p->storage == LBM_STORE_FP32 || p->storage == LBM_STORE_FP64;
  return p->kernel == LBM_KERNEL_TILED || p->kernel == LBM_KERNEL_TMA || (p->kernel == LBM_KERNEL_AUTO && wide);
}

// Whether the TMA variant of the tiled schedule runs (FP32 storage).
bool uses_tma(const lbm_params* p) {
  return TMA_AVAILABLE && p->kernel == LBM_KERNEL_TMA && p->storage == LBM_STORE_FP32;
}

// Whether a context keeps the per-tile lists of the halo schedule (4- and
// 8-byte storage; 16-bit storage runs the two-pass schedule instead). AUTO
// keeps room for them: it runs the halo schedule under the wetting schemes
// whose force reaches one node (Martys-Chen, LLKC, constant rho_s), where
// it is the fastest, and builds the lists at the first such step.
bool uses_halo(const lbm_params* p) {
  const bool wide = p->storage == LBM_STORE_FP32 || p->storage == LBM_STORE_FP64;
  return (p->kernel == LBM_KERNEL_HALO || p->kernel == LBM_KERNEL_AUTO) && wide;
}

// The tiled schedule with 16-bit storage keeps a third density plane: a step
// reads the encoding references rho(t - 1) and rho(t) and writes rho(t + 1).
bool tiled16(const lbm_params* p) {
  return (p->kernel == LBM_KERNEL_TILED || p->kernel == LBM_KERNEL_TMA) &&
         (p->storage == LBM_STORE_FP16 || p->storage == LBM_STORE_BF16);
}

constexpr int MASS_BLOCKS = 1024;

bool layout(const lbm_params* p, const Geo& g, Layout* L) {
  const size_t A = 256;
  const size_t es = elem_size(p->storage), cs = compute_size(p->storage);
  if (!es) return false;
  const int64_t N = (int64_t)p->nx * p->ny;
  const int64_t cap = p->max_interface > 0 ? p->max_interface : N;
  const int64_t scan_blocks = (N + SCAN_BLOCK - 1) / SCAN_BLOCK;
  size_t off = 0;
  L->f = off;        off = align_up(off + 2 * 18 * (size_t)g.plane * es, A);
  L->P = off;        off = align_up(off + (tiled16(p) ? 6 : 4) * (size_t)g.plane * cs, A);
  L->U = off;        off = align_up(off + (es == 2 && p->velocity_refs ? 2 * (size_t)g.plane * sizeof(UPair) : 0), A);
  L->flags = off;    off = align_up(off + (size_t)g.plane * 2, A);
  L->list = off;     off = align_up(off + (size_t)cap * 4, A);
  L->imask = off;    off = align_up(off + (size_t)cap * 4, A);
  L->flist = off;    off = align_up(off + (size_t)N * 4, A);
  const int64_t nt = uses_tiles(p) ? tile_count(g) : 0;
  L->tent = off;     off = align_up(off + (size_t)nt * TILE_RS * 2, A);
  L->toff = off;     off = align_up(off + (size_t)(nt ? nt + 1 : 0) * 4, A);
  L->tcnt = off;     off = align_up(off + (size_t)nt * 8, A);
  L->twork = off;    off = align_up(off + (size_t)(uses_tma(p) ? nt : 0) * 16, A);
  const int64_t nh = uses_halo(p) ? halo_tile_count(g) : 0;
  L->hent = off;     off = align_up(off + (size_t)nh * HALO_RS * 2, A);
  L->hoff = off;     off = align_up(off + (size_t)(nh ? nh + 1 : 0) * 4, A);
  L->hcnt = off;     off = align_up(off + (size_t)nh * 16, A);
  L->hmask = off;    off = align_up(off + (size_t)nh * HALO_MW * 4, A);
  L->counts = off;   off = align_up(off + (size_t)scan_blocks * 4, A);
  L->small = off;    off = align_up(off + 64, A);
  L->partial = off;  off = align_up(off + 2 * MASS_BLOCKS * 8, A);
  L->mass = off;     off = align_up(off + 16, A);
  L->smask = off;    off = align_up(off + (size_t)N, A);
  L->stage = off;    off = align_up(off + 4 * (size_t)N * 8, A);
  L->dpart = off;    off = align_up(off + ((size_t)DIAG_BLOCKS * DIAG_NRED + DIAG_NQ) * 8, A);
  L->total = off;
  return true;
}

// cuTensorMapEncodeTiled, resolved through the runtime (no link against the
// driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor maps of the TMA schedule: each population buffer as (2 px floats,
// py rows, 9 planes) and each density plane as (2 px floats, py rows), both
// with the (2 (TILE_W + 4), TILE_H + 4) box of one tile's window. Out-of-
// range rows and columns of a window (beyond the padded grid) read as zero
// and are never used.
bool encode_tma_maps(lbm_ctx* c) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const Geo& g = c->g;
  for (int b = 0; b < 2; ++b) {
    const cuuint64_t dimf[3] = {(cuuint64_t)2 * g.px, (cuuint64_t)g.py, 9};
    const cuuint64_t strf[2] = {(cuuint64_t)8 * g.px, (cuuint64_t)8 * g.plane};
    const cuuint32_t boxf[3] = {(cuuint32_t)TMA_BOX_X, (cuuint32_t)TMA_WH, 1};
    const cuuint32_t ones[3] = {1, 1, 1};
    if (enc(&c->tmap_f[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->f[b], dimf, strf, boxf, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    const cuuint64_t dimP[2] = {(cuuint64_t)2 * g.px, (cuuint64_t)g.py};
    const cuuint64_t strP[1] = {(cuuint64_t)8 * g.px};
    const cuuint32_t boxP[2] = {(cuuint32_t)TMA_BOX_X, (cuuint32_t)TMA_WH};
    if (enc(&c->tmap_P[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->Pbuf[b], dimP, strP, boxP, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

lbm_status fail(lbm_ctx* c, lbm_status s, const char* msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

lbm_status check_cuda(lbm_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return LBM_OK;
  if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
  return LBM_ERR_CUDA;
}

// The TMA schedule's bounded waits set small[4] when a copy was not seen to
// complete; synchronising calls report it (and clear it).
lbm_status check_timeout(lbm_ctx* c) {
  if (!c->tma) return LBM_OK;
  int v = 0;
  lbm_status s = check_cuda(c, cudaMemcpyAsync(&v, c->small + 4, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                            "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (s) return s;
  if (v) {
    s = check_cuda(c, cudaMemsetAsync(c->small + 4, 0, sizeof(int), c->stream), "cudaMemsetAsync");
    return s ? s : fail(c, LBM_ERR_TIMEOUT, "a TMA copy of the tiled step did not complete within its bounded wait");
  }
  return LBM_OK;
}

lbm_status after_launch(lbm_ctx* c, const char* where) {
  c->launches++;
  return check_cuda(c, cudaGetLastError(), where);
}

// Launch helper: runs fn() (which enqueues one kernel) and, while profiling,
// records an event on each side of it.
template <typename Fn>
lbm_status launch(lbm_ctx* c, int cls, const char* where, Fn&& fn) {
  const bool rec = c->prof_on && c->prof_n < c->prof_cap;
  if (rec) cudaEventRecord(c->prof_ev[2 * c->prof_n], c->stream);
  fn();
  lbm_status s = after_launch(c, where);
  if (rec) {
    cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->stream);
    c->prof_cls[c->prof_n++] = cls;
  }
  return s;
}

dim3 node_grid(const Geo& g, int bx) { return dim3((g.nx + bx - 1) / bx, g.ny); }

// Densities of the current state (and rho~ at interface-solid nodes) into
// the spare density plane Pbuf[pcur ^ 1]; Pbuf[pcur] keeps the references
// the current populations were encoded with.
template <typename T>
lbm_status launch_density_and_virtual(lbm_ctx* c, const T* f) {
  using C = typename Pop<T>::C;
  C* P = (C*)c->Pbuf[c->pcur ^ 1];
  const C* Pref = (const C*)c->Pbuf[c->pcur];
  lbm_status s = launch(c, LBM_KC_DENSITY, "k_density", [&] {
    k_density<T><<<node_grid(c->g, 128), 128, 0, c->stream>>>(f, P, Pref, c->Ubuf[c->cur], c->flags, c->g,
                                                                kphys<C>(c->ph));
  });
  if (s) return s;
  c->p_valid = false;
  if (c->ph.bc == BC_VAVG && c->n_iface > 0) {
    s = launch(c, LBM_KC_VIRTUAL, "k_virtual_density", [&] {
      k_virtual_density<C><<<(c->n_iface + 127) / 128, 128, 0, c->stream>>>(P, c->iface_mask, c->iface_list,
                                                                             c->n_iface, c->g, kphys<C>(c->ph));
    });
  }
  return s;
}

// Two-pass step: densities of the pulled populations into the spare plane,
// rho~ there, then force + collide + stream, whose output is encoded with
// those densities; the planes then swap roles.
template <typename T>
lbm_status step_two_pass(lbm_ctx* c, int nsteps) {
  using C = typename Pop<T>::C;
  const int nb = (c->n_fluid + 255) / 256;
  const int nbc = (c->n_fluid + COLLIDE_THREADS - 1) / COLLIDE_THREADS;
  for (int t = 0; t < nsteps && c->n_fluid > 0; ++t) {
    const T* fin = (const T*)c->f[c->cur];
    T* fout = (T*)c->f[c->cur ^ 1];
    C* P = (C*)c->Pbuf[c->pcur ^ 1];
    const C* Pref = (const C*)c->Pbuf[c->pcur];
    // velocity references (16-bit storage only) run their own instantiations
    const bool vr = kDev<T> && c->prm.velocity_refs;
    lbm_status s = launch(c, LBM_KC_DENSITY, "k_density_list", [&] {
      auto kd = vr ? k_density_list<T, kDev<T>> : k_density_list<T, false>;
      kd<<<nb, 256, 0, c->stream>>>(fin, P, Pref, c->Ubuf[c->cur], c->flags, c->fluid_list, c->n_fluid, c->g,
                                    kphys<C>(c->ph));
    });
    if (s) return s;
    if (c->ph.bc == BC_VAVG && c->n_iface > 0) {
      s = launch(c, LBM_KC_VIRTUAL, "k_virtual_density", [&] {
        k_virtual_density<C><<<(c->n_iface + 127) / 128, 128, 0, c->stream>>>(P, c->iface_mask, c->iface_list,
                                                                               c->n_iface, c->g, kphys<C>(c->ph));
      });
      if (s) return s;
    }
    s = launch(c, LBM_KC_COLLIDE, "k_collide_list", [&] {
      auto kc = vr ? k_collide_list<T, kDev<T>> : k_collide_list<T, false>;
      kc<<<nbc, COLLIDE_THREADS, 0, c->stream>>>(fin, fout, P, Pref, c->Ubuf[c->cur], c->Ubuf[c->cur ^ 1], c->flags,
                                                 c->fluid_list, c->n_fluid, c->g, kphys<C>(c->ph));
    });
    if (s) return s;
    c->cur ^= 1;
    c->pcur ^= 1;
    c->P = c->Pbuf[c->pcur];
    c->p_valid = false;
  }
  return LBM_OK;
}

template <typename T>
lbm_status step_fused(lbm_ctx* c, int nsteps) {
  using C = typename Pop<T>::C;
  if (nsteps > 0 && !c->p_valid) {
    // rho of the current state, once; every fused step then produces the next
    lbm_status s = launch(c, LBM_KC_DENSITY, "k_density", [&] {
      k_density<T><<<node_grid(c->g, 128), 128, 0, c->stream>>>((const T*)c->f[c->cur], (C*)c->P, (const C*)c->P,
                                                                  nullptr, c->flags, c->g, kphys<C>(c->ph));
    });
    if (s) return s;
    c->p_valid = true;
  }
  for (int t = 0; t < nsteps; ++t) {
    const T* fin = (const T*)c->f[c->cur];
    T* fout = (T*)c->f[c->cur ^ 1];
    C* Pin = (C*)c->Pbuf[c->pcur];
    C* Pout = (C*)c->Pbuf[c->pcur ^ 1];
    lbm_status s;
    if (c->ph.bc == BC_VAVG && c->n_iface > 0) {
      // rho~(t) of Eq. 8 into the solid cells of the plane the step reads
      s = launch(c, LBM_KC_VIRTUAL, "k_virtual_density", [&] {
        k_virtual_density<C><<<(c->n_iface + 127) / 128, 128, 0, c->stream>>>(Pin, c->iface_mask, c->iface_list,
                                                                               c->n_iface, c->g, kphys<C>(c->ph));
      });
      if (s) return s;
    }
    lbm_status ls = LBM_OK;
    if constexpr (sizeof(T) == 4) {
      if (c->tma) {
        s = launch(c, LBM_KC_FUSED, "k_tile_tma", [&] {
          constexpr size_t SMEM = tma_smem<T>();
          if (!c->tma_smem_set) {
            if (cudaFuncSetAttribute(k_tile_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) !=
                cudaSuccess) {
              ls = LBM_ERR_CUDA;
              return;
            }
            c->tma_smem_set = true;
          }
          const int ntx = (c->g.nx + TILE_W - 1) / TILE_W;
          // TMA_MINB persistent CTAs per SM
          const int slots = c->num_sms * TMA_MINB;
          const int grid = c->n_work < slots ? (c->n_work > 0 ? c->n_work : 1) : slots;
          k_tile_tma<<<grid, TMA_THREADS, SMEM, c->stream>>>(
              c->tmap_f[c->cur], c->tmap_P[c->pcur], (float*)fout, (float*)Pout, c->flags, c->tile_entries,
              c->tile_work, c->n_work, c->g, ntx, kphys<float>(c->ph), c->small + 4, c->tma_extra_tx);
        });
        if (ls) return fail(c, ls, "k_tile_tma launch rejected");
        if (s) return s;
        c->cur ^= 1;
        c->pcur ^= 1;
        c->P = c->Pbuf[c->pcur];
        continue;
      }
    }
    if (c->n_tiles > 0) {
      s = launch(c, LBM_KC_FUSED, "k_tile", [&] {
        ls = launch_tiled<T>(c->g, c->ph, fin, fout, Pin, Pin, nullptr, nullptr, Pout, c->flags, c->tile_entries, c->tile_off,
                             c->tile_cnt, &c->tile_smem_set, c->stream);
      });
    } else {
      s = launch(c, LBM_KC_FUSED, "k_march", [&] {
        ls = launch_fused<T>(c->g, c->ph, fin, fout, Pin, Pout, c->flags, c->num_sms, &c->march_smem_set, c->stream);
      });
    }
    if (ls) return fail(c, ls, "fused kernel launch rejected");
    if (s) return s;
    c->cur ^= 1;
    c->pcur ^= 1;
    c->P = c->Pbuf[c->pcur];
  }
  return LBM_OK;
}

// Tiled step with 16-bit storage. Between steps Pbuf[pcur] holds the
// densities the current populations were encoded with (as for the two-pass
// schedule) and, when p_valid, Pbuf[pcur ^ 1] the densities of the current
// state. A step reads both and writes the next densities into Pbuf[2]; the
// three pointers then rotate.
template <typename T>
lbm_status step_tiled16(lbm_ctx* c, int nsteps) {
  using C = typename Pop<T>::C;
  if (nsteps > 0 && !c->p_valid) {
    lbm_status s = launch(c, LBM_KC_DENSITY, "k_density", [&] {
      k_density<T><<<node_grid(c->g, 128), 128, 0, c->stream>>>((const T*)c->f[c->cur], (C*)c->Pbuf[c->pcur ^ 1],
                                                                  (const C*)c->Pbuf[c->pcur], c->Ubuf[c->cur],
                                                                  c->flags, c->g,
                                                                  kphys<C>(c->ph));
    });
    if (s) return s;
    c->p_valid = true;
  }
  for (int t = 0; t < nsteps; ++t) {
    const T* fin = (const T*)c->f[c->cur];
    T* fout = (T*)c->f[c->cur ^ 1];
    const C* Pref = (const C*)c->Pbuf[c->pcur];
    C* P = (C*)c->Pbuf[c->pcur ^ 1];
    C* Po = (C*)c->Pbuf[2];
    lbm_status s;
    if (c->ph.bc == BC_VAVG && c->n_iface > 0) {
      s = launch(c, LBM_KC_VIRTUAL, "k_virtual_density", [&] {
        k_virtual_density<C><<<(c->n_iface + 127) / 128, 128, 0, c->stream>>>(P, c->iface_mask, c->iface_list,
                                                                               c->n_iface, c->g, kphys<C>(c->ph));
      });
      if (s) return s;
    }
    lbm_status ls = LBM_OK;
    s = launch(c, LBM_KC_FUSED, "k_tile", [&] {
      ls = launch_tiled<T>(c->g, c->ph, fin, fout, P, Pref, c->Ubuf[c->cur], c->Ubuf[c->cur ^ 1], Po, c->flags,
                           c->tile_entries, c->tile_off,
                           c->tile_cnt, &c->tile_smem_set, c->stream);
    });
    if (ls) return fail(c, ls, "tiled kernel launch rejected");
    if (s) return s;
    c->cur ^= 1;
    // the new populations were encoded with rho(t), their densities are
    // rho(t + 1); the plane of rho(t - 1) is free
    void* freed = c->Pbuf[c->pcur];
    c->Pbuf[c->pcur] = c->Pbuf[c->pcur ^ 1];
    c->Pbuf[c->pcur ^ 1] = c->Pbuf[2];
    c->Pbuf[2] = freed;
    c->P = c->Pbuf[c->pcur];
  }
  return LBM_OK;
}

// Per-tile lists of the halo schedule for the current geometry: counts and
// fluid bitmasks, offsets (fixed-order scan, total at halo_off[n_halo_tiles]),
// entries. Built by lbm_set_geometry for HALO, at the first halo step for AUTO.
lbm_status build_halo_lists(lbm_ctx* c) {
  const Geo& g = c->g;
  const int ntx = (g.nx + HALO_W - 1) / HALO_W;
  const int nt = (int)c->n_halo_tiles;
  lbm_status s;
  k_halo_lists<<<nt, HALO_LIST_THREADS, 0, c->stream>>>(c->flags, g, ntx, nullptr, c->halo_off, c->halo_cnt,
                                                        c->halo_fmask, nullptr);
  if ((s = after_launch(c, "k_halo_lists(count)"))) return s;
  k_iface_scan<<<1, 1024, 0, c->stream>>>(c->halo_off, nt, c->halo_off + nt);
  if ((s = after_launch(c, "k_iface_scan(halo)"))) return s;
  k_halo_lists<<<nt, HALO_LIST_THREADS, 0, c->stream>>>(c->flags, g, ntx, c->halo_off, nullptr, nullptr, nullptr,
                                                        c->halo_entries);
  if ((s = after_launch(c, "k_halo_lists(write)"))) return s;
  c->halo_built = true;
  return LBM_OK;
}

// Halo schedule: one kernel per step, densities recomputed per tile from the
// populations (no density plane).
template <typename T>
lbm_status step_halo(lbm_ctx* c, int nsteps) {
  for (int t = 0; t < nsteps; ++t) {
    const T* fin = (const T*)c->f[c->cur];
    T* fout = (T*)c->f[c->cur ^ 1];
    lbm_status ls = LBM_OK;
    lbm_status s = launch(c, LBM_KC_FUSED, "k_halo", [&] {
      ls = launch_halo<T>(c->g, c->ph, fin, fout, c->flags, c->halo_entries, c->halo_off, c->halo_cnt,
                          c->halo_fmask, c->stream);
    });
    if (ls) return fail(c, ls, "halo kernel launch rejected");
    if (s) return s;
    c->cur ^= 1;
    c->p_valid = false;
  }
  return LBM_OK;
}

template <typename T>
lbm_status do_step(lbm_ctx* c, int nsteps) {
  if constexpr (sizeof(T) >= 4) {  // the marching kernel stores 4- and 8-byte populations only
    // HALO always; AUTO under the one-node-reach schemes (the improved
    // scheme's Eq. 8 reaches three rings, where the tiled schedule wins)
    const bool halo = c->prm.kernel == LBM_KERNEL_HALO || (c->prm.kernel == LBM_KERNEL_AUTO && c->ph.bc != BC_VAVG);
    if (halo && c->n_halo_tiles > 0) {
      if (!c->halo_built) {
        lbm_status s = build_halo_lists(c);
        if (s) return s;
      }
      return step_halo<T>(c, nsteps);
    }
    if (c->prm.kernel == LBM_KERNEL_FUSED && fused_supported<T>(c->g, c->ph)) return step_fused<T>(c, nsteps);
    const bool tiled = c->prm.kernel == LBM_KERNEL_TILED || c->prm.kernel == LBM_KERNEL_AUTO || c->prm.kernel == LBM_KERNEL_TMA;
    if (tiled && c->n_tiles > 0) return step_fused<T>(c, nsteps);
  } else {
    if (c->Pbuf[2] && c->n_tiles > 0) return step_tiled16<T>(c, nsteps);
  }
  return step_two_pass<T>(c, nsteps);
}

template <typename T, int MODE, typename O = double>
lbm_status do_eval(lbm_ctx* c, O* out) {
  const T* fin = (const T*)c->f[c->cur];
  lbm_status s = launch_density_and_virtual<T>(c, fin);
  if (s) return s;
  using C = typename Pop<T>::C;
  k_collide<T, MODE, O><<<node_grid(c->g, 128), 128, 0, c->stream>>>(
      fin, (const C*)c->Pbuf[c->pcur ^ 1], (const C*)c->Pbuf[c->pcur], c->Ubuf[c->cur], c->flags, c->g,
      kphys<C>(c->ph), out);
  return after_launch(c, "k_collide(eval)");
}

template <typename T>
lbm_status do_get_pops(lbm_ctx* c, double* out) {
  using C = typename Pop<T>::C;
  k_get_populations<T><<<node_grid(c->g, 128), 128, 0, c->stream>>>((const T*)c->f[c->cur], (const C*)c->P,
                                                                     c->Ubuf[c->cur],
                                                                     c->flags, c->g, kphys<C>(c->ph), out);
  return after_launch(c, "k_get_populations");
}

template <typename T, int SRC>
lbm_status do_set_state(lbm_ctx* c, const double* fin, const double* rA, const double* rB, const double* ux,
                        const double* uy) {
  using C = typename Pop<T>::C;
  k_set_state<T, SRC><<<node_grid(c->g, 128), 128, 0, c->stream>>>((T*)c->f[c->cur], (C*)c->P, c->Ubuf[c->cur],
                                                                     c->flags, c->g,
                                                                     kphys<C>(c->ph), fin, rA, rB, ux, uy);
  return after_launch(c, "k_set_state");
}

template <typename T>
lbm_status do_mass(lbm_ctx* c) {
  using C = typename Pop<T>::C;
  k_mass_partial<T><<<c->mass_blocks, 256, 0, c->stream>>>((const T*)c->f[c->cur], (const C*)c->P,
                                                           c->Ubuf[c->cur], c->flags,
                                                           c->g, kphys<C>(c->ph), c->partial);
  lbm_status s = after_launch(c, "k_mass_partial");
  if (s) return s;
  k_mass_final<<<1, 64, 0, c->stream>>>(c->partial, c->mass_blocks, c->mass_out);
  return after_launch(c, "k_mass_final");
}

// Dispatch on the storage type.
#define LBM_DISPATCH(c, CALL)                            \
  switch ((c)->prm.storage) {                            \
    case LBM_STORE_FP32: { using T = float; CALL; }      \
    case LBM_STORE_FP64: { using T = double; CALL; }     \
    case LBM_STORE_FP16: { using T = __half; CALL; }     \
    default: { using T = __nv_bfloat16; CALL; }          \
  }

bool valid_params(const lbm_params* p) {
  if (!p) return false;
  if (p->nx < 4 || p->ny < 4) return false;
  if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5)) return false;
  if (p->storage < LBM_STORE_FP32 || p->storage > LBM_STORE_BF16) return false;
  if (p->kernel < LBM_KERNEL_AUTO || p->kernel > LBM_KERNEL_TMA) return false;
  if (p->max_interface < 0) return false;
  if (p->velocity_refs != 0 && p->velocity_refs != 1) return false;
  return true;
}

}  // namespace

extern "C" {

const char* lbm_status_str(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_STATE: return "call out of order";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_SPACE: return "workspace too small";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err : ""; }

int64_t lbm_launch_count(const lbm_ctx* ctx) { return ctx ? ctx->launches : 0; }

lbm_status lbm_debug_tma_expect_extra(lbm_ctx* c, int32_t bytes) {
  if (!c || bytes < 0 || bytes > 4096) return LBM_ERR_ARG;
  c->tma_extra_tx = (uint32_t)bytes;
  return LBM_OK;
}

lbm_status lbm_workspace_bytes(const lbm_params* params, size_t* bytes) {
  if (!valid_params(params) || !bytes) return LBM_ERR_ARG;
  Geo g;
  if (!make_geo(params, &g)) return LBM_ERR_ARG;
  Layout L;
  if (!layout(params, g, &L)) return LBM_ERR_ARG;
  *bytes = L.total;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_params* params, void* d_workspace, size_t bytes, void* cuda_stream,
                      lbm_ctx** out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!valid_params(params) || !d_workspace) return LBM_ERR_ARG;
  if (((uintptr_t)d_workspace) % 256) return LBM_ERR_ARG;
  Geo g;
  Layout L;
  if (!make_geo(params, &g) || !layout(params, g, &L)) return LBM_ERR_ARG;
  if (bytes < L.total) return LBM_ERR_SPACE;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_SPACE;
  c->prm = *params;
  if (!(c->prm.rho_ref[0] > 0)) c->prm.rho_ref[0] = 1.0;
  if (!(c->prm.rho_ref[1] > 0)) c->prm.rho_ref[1] = 1.0;
  c->g = g;
  c->stream = (cudaStream_t)cuda_stream;
  c->ws = (char*)d_workspace;
  c->ws_bytes = bytes;
  const size_t es = elem_size(params->storage);
  c->f[0] = c->ws + L.f;
  c->f[1] = c->ws + L.f + 18 * (size_t)g.plane * es;
  c->Pbuf[0] = c->ws + L.P;
  c->Pbuf[1] = c->ws + L.P + 2 * (size_t)g.plane * compute_size(params->storage);
  c->Pbuf[2] = tiled16(params) ? c->ws + L.P + 4 * (size_t)g.plane * compute_size(params->storage) : nullptr;
  c->Pbase = c->ws + L.P;
  const bool uplanes = es == 2 && params->velocity_refs;
  c->Ubuf[0] = uplanes ? (UPair*)(c->ws + L.U) : nullptr;
  c->Ubuf[1] = uplanes ? (UPair*)(c->ws + L.U + (size_t)g.plane * sizeof(UPair)) : nullptr;
  c->pcur = 0;
  c->P = c->Pbuf[0];
  c->p_valid = false;
  c->flags = (uint16_t*)(c->ws + L.flags);
  c->iface_list = (int*)(c->ws + L.list);
  c->iface_mask = (uint32_t*)(c->ws + L.imask);
  c->fluid_list = (int*)(c->ws + L.flist);
  c->n_tiles = uses_tiles(params) ? tile_count(g) : 0;
  c->tma = uses_tma(params);
  c->tile_entries = c->n_tiles ? (uint16_t*)(c->ws + L.tent) : nullptr;
  c->tile_off = c->n_tiles ? (int*)(c->ws + L.toff) : nullptr;
  c->tile_cnt = c->n_tiles ? (int2*)(c->ws + L.tcnt) : nullptr;
  c->tile_work = c->n_tiles && uses_tma(params) ? (int4*)(c->ws + L.twork) : nullptr;
  c->n_halo_tiles = uses_halo(params) ? halo_tile_count(g) : 0;
  c->halo_entries = c->n_halo_tiles ? (uint16_t*)(c->ws + L.hent) : nullptr;
  c->halo_off = c->n_halo_tiles ? (int*)(c->ws + L.hoff) : nullptr;
  c->halo_cnt = c->n_halo_tiles ? (int4*)(c->ws + L.hcnt) : nullptr;
  c->halo_fmask = c->n_halo_tiles ? (uint32_t*)(c->ws + L.hmask) : nullptr;
  c->scan_counts = (int*)(c->ws + L.counts);
  c->small = (int*)(c->ws + L.small);
  c->partial = (double*)(c->ws + L.partial);
  c->mass_out = (double*)(c->ws + L.mass);
  c->stage_mask = (uint8_t*)(c->ws + L.smask);
  c->stage = (double*)(c->ws + L.stage);
  c->dpart = (double*)(c->ws + L.dpart);
  const int64_t N = (int64_t)params->nx * params->ny;
  c->if_capacity = params->max_interface > 0 ? params->max_interface : N;
  c->scan_blocks = (int)((N + SCAN_BLOCK - 1) / SCAN_BLOCK);
  c->mass_blocks = MASS_BLOCKS;
  // physics defaults: Martys-Chen with no adhesion until lbm_set_wetting
  Phys& ph = c->ph;
  memset(&ph, 0, sizeof(ph));
  for (int s = 0; s < 2; ++s) {
    ph.omega[s] = 1.0 / params->tau[s];
    ph.kF[s] = 1.0 - 0.5 / params->tau[s];
    ph.chi[s] = 1.0;
    ph.rho_ref[s] = params->storage >= LBM_STORE_FP16 ? c->prm.rho_ref[s] : 0.0;
  }
  ph.G_AB = params->G_AB;
  ph.bc = BC_MC;
  lbm_status s = check_cuda(c, cudaGetDevice(&c->device), "cudaGetDevice");
  if (!s) s = check_cuda(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device),
                         "cudaDeviceGetAttribute");
  if (!s) s = check_cuda(c, cudaMemsetAsync(c->ws, 0, L.total, c->stream), "cudaMemsetAsync");
  if (!s && c->tma && !encode_tma_maps(c)) s = LBM_ERR_CUDA;
  if (s) {
    delete c;
    return s;
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* cuda_stream) {
  if (!c) return LBM_ERR_ARG;
  c->stream = (cudaStream_t)cuda_stream;
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* d_mask) {
  if (!c || !d_mask) return LBM_ERR_ARG;
  const Geo& g = c->g;
  c->has_fields = false;
  c->has_geometry = false;
  lbm_status s = check_cuda(c, cudaMemsetAsync(c->small, 0, 64, c->stream), "cudaMemsetAsync");
  if (s) return s;
  k_flags<<<dim3((g.px + 127) / 128, g.py), 128, 0, c->stream>>>(d_mask, c->flags, g, c->small);
  if ((s = after_launch(c, "k_flags"))) return s;
  // interface-solid list, then the fluid list: bulk nodes first, then edge
  // nodes (appended after the bulk count, read on the device)
  const int64_t N = (int64_t)g.nx * g.ny;
  struct Pass { int cls; int* list; int* total; const int* base; int64_t cap; };
  const Pass passes[2] = {{CLS_IFACE, c->iface_list, c->small + 1, nullptr, c->if_capacity},
                          {CLS_FLUID, c->fluid_list, c->small + 2, nullptr, N}};
  for (const Pass& ps : passes) {
    k_class_count<<<c->scan_blocks, SCAN_BLOCK, 0, c->stream>>>(c->flags, g, ps.cls, c->scan_counts);
    if ((s = after_launch(c, "k_class_count"))) return s;
    k_iface_scan<<<1, 1024, 0, c->stream>>>(c->scan_counts, c->scan_blocks, ps.total);
    if ((s = after_launch(c, "k_iface_scan"))) return s;
    k_class_write<<<c->scan_blocks, SCAN_BLOCK, 0, c->stream>>>(c->flags, g, ps.cls, c->scan_counts, ps.base,
                                                                (int)ps.cap, ps.list);
    if ((s = after_launch(c, "k_class_write"))) return s;
  }
  // clear the density planes so solid cells read as zero
  c->p_valid = false;
  s = check_cuda(c, cudaMemsetAsync(c->Pbase, 0, (c->Pbuf[2] ? 6 : 4) * (size_t)g.plane * compute_size(c->prm.storage),
                                    c->stream), "cudaMemsetAsync");
  if (s) return s;
  int h[3];
  s = check_cuda(c, cudaMemcpyAsync(h, c->small, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (s) return s;
  if (h[0] > 0) return fail(c, LBM_ERR_ARG, "fluid node on a non-periodic border");
  if (h[1] > c->if_capacity) return fail(c, LBM_ERR_SPACE, "interface-solid list exceeds max_interface");
  c->n_iface = h[1];
  c->n_fluid = h[2];
  if (c->n_iface > 0) {
    k_iface_mask<<<(c->n_iface + 127) / 128, 128, 0, c->stream>>>(c->flags, c->iface_list, c->n_iface, g,
                                                                  c->iface_mask);
    if ((s = after_launch(c, "k_iface_mask"))) return s;
  }
  if (c->n_tiles > 0) {
    // per-tile lists of the tiled schedule: counts, offsets (fixed-order
    // scan, total at tile_off[n_tiles]), entries
    const int ntx = (g.nx + TILE_W - 1) / TILE_W;
    const int nt = (int)c->n_tiles;
    k_tile_lists<<<nt, TILE_LIST_THREADS, 0, c->stream>>>(c->flags, g, ntx, nullptr, c->tile_off, c->tile_cnt, nullptr);
    if ((s = after_launch(c, "k_tile_lists(count)"))) return s;
    k_iface_scan<<<1, 1024, 0, c->stream>>>(c->tile_off, nt, c->tile_off + nt);
    if ((s = after_launch(c, "k_iface_scan(tiles)"))) return s;
    k_tile_lists<<<nt, TILE_LIST_THREADS, 0, c->stream>>>(c->flags, g, ntx, c->tile_off, nullptr, nullptr,
                                                     c->tile_entries);
    if ((s = after_launch(c, "k_tile_lists(write)"))) return s;
    if (c->tile_work) {
      // the TMA schedule's work list: the tiles with owned nodes, in order
      k_tile_work<<<1, 1024, 0, c->stream>>>(c->tile_cnt, c->tile_off, nt, c->tile_work, c->small + 5);
      if ((s = after_launch(c, "k_tile_work"))) return s;
      int nw = 0;
      s = check_cuda(c, cudaMemcpyAsync(&nw, c->small + 5, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                     "cudaMemcpyAsync");
      if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
      if (s) return s;
      c->n_work = nw;
    }
  }
  c->halo_built = false;
  if (c->n_halo_tiles > 0 && c->prm.kernel == LBM_KERNEL_HALO && (s = build_halo_lists(c))) return s;
  c->has_geometry = true;
  return LBM_OK;
}

lbm_status lbm_set_wetting(lbm_ctx* c, const lbm_wetting_params* w) {
  if (!c || !w) return LBM_ERR_ARG;
  if (w->kind < LBM_WET_MARTYS_CHEN || w->kind > LBM_WET_CONSTANT) return fail(c, LBM_ERR_ARG, "unknown wetting kind");
  if (w->pairing != LBM_PAIR_CROSS && w->pairing != LBM_PAIR_SELF) return fail(c, LBM_ERR_ARG, "unknown pairing");
  if (w->avg_stencil != 9 && w->avg_stencil != 25) return fail(c, LBM_ERR_ARG, "avg_stencil must be 9 or 25");
  if (w->kind == LBM_WET_VIRTUAL_AVG)
    for (int s = 0; s < 2; ++s)
      if (!(w->chi[s] > 0.0 && w->chi[s] <= 2.0)) return fail(c, LBM_ERR_ARG, "chi outside (0, 2]");
  c->ph.bc = w->kind;
  c->ph.pairing = w->pairing;
  c->ph.avg9 = w->avg_stencil == 9 ? 1 : 0;
  for (int s = 0; s < 2; ++s) {
    c->ph.G_s[s] = w->G_s[s];
    c->ph.chi[s] = w->chi[s];
    c->ph.rho_s[s] = w->rho_s[s];
  }
  c->ph.uniform = w->kind == LBM_WET_VIRTUAL_AVG && w->pairing == LBM_PAIR_CROSS && w->G_s[0] == c->ph.G_AB &&
                  w->G_s[1] == c->ph.G_AB;
  c->has_wetting = true;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rA, const double* rB, const double* ux, const double* uy) {
  if (!c || !rA || !rB) return LBM_ERR_ARG;
  if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_init_fields before lbm_set_geometry");
  c->cur = 0;
  c->p_valid = false;
  lbm_status s;
  LBM_DISPATCH(c, s = (do_set_state<T, 1>(c, nullptr, rA, rB, ux, uy)); break);
  if (!s) c->has_fields = true;
  return s;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* fin) {
  if (!c || !fin) return LBM_ERR_ARG;
  if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_set_populations before lbm_set_geometry");
  c->cur = 0;
  c->p_valid = false;
  lbm_status s;
  LBM_DISPATCH(c, s = (do_set_state<T, 0>(c, fin, nullptr, nullptr, nullptr, nullptr)); break);
  if (!s) c->has_fields = true;
  return s;
}

lbm_status lbm_step(lbm_ctx* c, int32_t nsteps) {
  if (!c || nsteps < 0) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_step before geometry and fields");
  lbm_status s;
  LBM_DISPATCH(c, s = do_step<T>(c, nsteps); break);
  return s;
}

lbm_status lbm_step_profiled(lbm_ctx* c, int32_t nsteps, double* h_ms, int64_t* h_launches) {
  if (!c || nsteps < 0) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_step before geometry and fields");
  const int cap = 3 * nsteps + 4;
  c->prof_ev = (cudaEvent_t*)calloc((size_t)2 * cap, sizeof(cudaEvent_t));
  c->prof_cls = (int*)calloc((size_t)cap, sizeof(int));
  if (!c->prof_ev || !c->prof_cls) {
    free(c->prof_ev);
    free(c->prof_cls);
    c->prof_ev = nullptr;
    c->prof_cls = nullptr;
    return fail(c, LBM_ERR_SPACE, "host allocation for profiling events failed");
  }
  lbm_status s = LBM_OK;
  int created = 0;
  for (; created < 2 * cap && !s; ++created)
    s = check_cuda(c, cudaEventCreate(&c->prof_ev[created]), "cudaEventCreate");
  if (!s) {
    c->prof_on = true;
    c->prof_n = 0;
    c->prof_cap = cap;
    LBM_DISPATCH(c, s = do_step<T>(c, nsteps); break);
    c->prof_on = false;
  }
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  double ms[LBM_KC_COUNT] = {0, 0, 0, 0};
  int64_t cnt[LBM_KC_COUNT] = {0, 0, 0, 0};
  if (!s)
    for (int i = 0; i < c->prof_n && !s; ++i) {
      float t = 0.f;
      s = check_cuda(c, cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]),
                     "cudaEventElapsedTime");
      ms[c->prof_cls[i]] += t;
      cnt[c->prof_cls[i]] += 1;
    }
  for (int i = 0; i < created; ++i) cudaEventDestroy(c->prof_ev[i]);
  free(c->prof_ev);
  free(c->prof_cls);
  c->prof_ev = nullptr;
  c->prof_cls = nullptr;
  c->prof_n = c->prof_cap = 0;
  if (!s) s = check_timeout(c);
  if (s) return s;
  for (int k = 0; k < LBM_KC_COUNT; ++k) {
    if (h_ms) h_ms[k] = ms[k];
    if (h_launches) h_launches[k] = cnt[k];
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* c, double* rA, double* rB, double* ux, double* uy) {
  if (!c) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_moments before geometry and fields");
  const int64_t N = (int64_t)c->g.nx * c->g.ny;
  double* tmp = c->stage;  // 4 * N doubles
  lbm_status s;
  LBM_DISPATCH(c, s = (do_eval<T, 1>(c, tmp)); break);
  if (s) return s;
  double* outs[4] = {rA, rB, ux, uy};
  for (int a = 0; a < 4 && !s; ++a)
    if (outs[a])
      s = check_cuda(c, cudaMemcpyAsync(outs[a], tmp + a * N, N * 8, cudaMemcpyDeviceToDevice, c->stream),
                     "cudaMemcpyAsync");
  return s;
}

lbm_status lbm_forces(lbm_ctx* c, double* F) {
  if (!c || !F) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_forces before geometry and fields");
  lbm_status s;
  LBM_DISPATCH(c, s = (do_eval<T, 2>(c, F)); break);
  return s;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* out) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_get_populations before fields");
  lbm_status s;
  LBM_DISPATCH(c, s = do_get_pops<T>(c, out); break);
  return s;
}

lbm_status lbm_mass(lbm_ctx* c, double* h_out) {
  if (!c || !h_out) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_mass before geometry and fields");
  lbm_status s;
  LBM_DISPATCH(c, s = do_mass<T>(c); break);
  if (s) return s;
  s = check_cuda(c, cudaMemcpyAsync(h_out, c->mass_out, 16, cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (!s) s = check_timeout(c);
  return s;
}

lbm_status lbm_set_l2_fetch_granularity(int32_t bytes, int32_t* previous) {
  if (bytes != 32 && bytes != 64 && bytes != 128) return LBM_ERR_ARG;
  size_t old = 0;
  if (cudaDeviceGetLimit(&old, cudaLimitMaxL2FetchGranularity) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes) != cudaSuccess) return LBM_ERR_CUDA;
  if (previous) *previous = (int32_t)old;
  return LBM_OK;
}

lbm_status lbm_diagnostics(lbm_ctx* c, const lbm_diag_params* p, lbm_diag* h_out) {
  if (!c || !p || !h_out) return LBM_ERR_ARG;
  if (!c->has_geometry || !c->has_fields) return fail(c, LBM_ERR_STATE, "lbm_diagnostics before geometry and fields");
  const double vals[] = {p->level, p->rho_out, p->tangent[0], p->tangent[1], p->wall_point[0], p->wall_point[1],
                         p->wall_angle_deg, p->exclude, p->box[0], p->box[1], p->box[2], p->box[3]};
  for (double v : vals)
    if (!isfinite(v)) return fail(c, LBM_ERR_ARG, "lbm_diagnostics: non-finite parameter");
  if (!(p->level > 0.0 && p->level < 2.0)) return fail(c, LBM_ERR_ARG, "lbm_diagnostics: level outside (0, 2)");
  if (p->bridge_x >= 0 && (p->bridge_x >= c->g.nx || p->bridge_y0 < 0 || p->bridge_y0 >= c->g.ny))
    return fail(c, LBM_ERR_ARG, "lbm_diagnostics: bridge column or row outside the grid");
  DiagArgs a;
  a.level = p->level;
  a.rho_out = p->rho_out;
  a.wx = p->wall_point[0];
  a.wy = p->wall_point[1];
  const double b = p->wall_angle_deg * (M_PI / 180.0);
  a.nx_ = -sin(b);
  a.ny_ = cos(b);
  a.exclude = p->exclude;
  for (int i = 0; i < 4; ++i) a.box[i] = p->box[i];
  a.use_box = p->box[1] >= p->box[0];
  a.ox = 0.5 * c->g.nx;  // the fit is translation invariant; centring keeps its sums well scaled
  a.oy = 0.5 * c->g.ny;
  a.bridge_x = p->bridge_x;
  a.bridge_y0 = p->bridge_y0;
  lbm_status s;
  LBM_DISPATCH(c, s = (do_eval<T, 1>(c, c->stage)); break);
  if (s) return s;
  double* out_d = c->dpart + (size_t)DIAG_BLOCKS * DIAG_NRED;
  k_diag_partial<<<DIAG_BLOCKS, DIAG_THREADS, 0, c->stream>>>(c->stage, c->flags, c->g, a, c->dpart);
  if ((s = after_launch(c, "k_diag_partial"))) return s;
  k_diag_final<<<1, 32, 0, c->stream>>>(c->dpart, c->stage, c->g, a, out_d);
  if ((s = after_launch(c, "k_diag_final"))) return s;
  double q[DIAG_NQ];
  s = check_cuda(c, cudaMemcpyAsync(q, out_d, sizeof(q), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (s) return s;
  const double nan = NAN;
  lbm_diag& o = *h_out;
  o.weight = q[0];
  o.com[0] = q[0] > 0 ? q[1] / q[0] : nan;
  o.com[1] = q[0] > 0 ? q[2] / q[0] : nan;
  o.com_velocity[0] = q[0] > 0 ? q[3] / q[0] : nan;
  o.com_velocity[1] = q[0] > 0 ? q[4] / q[0] : nan;
  o.sliding_velocity = o.com_velocity[0] * p->tangent[0] + o.com_velocity[1] * p->tangent[1];
  o.nonfinite_nodes = (int64_t)q[15];
  o.max_u = q[15] > 0 ? nan : sqrt(q[14]);
  o.contour_points = (int64_t)q[5];
  o.circle[0] = o.circle[1] = o.circle[2] = nan;
  o.contact_angle_deg = nan;
  o.bridge_radius = q[16];
  if (q[5] >= 3) {
    // normal equations of min sum (x^2 + y^2 - A x - B y - C)^2 (Kasa fit),
    // solved by Gaussian elimination with partial pivoting
    double M[3][4] = {{q[8], q[10], q[6], q[11]}, {q[10], q[9], q[7], q[12]}, {q[6], q[7], q[5], q[13]}};
    bool ok = true;
    for (int col = 0; col < 3 && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < 3; ++r)
        if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
      if (!(fabs(M[piv][col]) > 0)) {
        ok = false;
        break;
      }
      if (piv != col)
        for (int j = 0; j < 4; ++j) {
          const double t = M[col][j];
          M[col][j] = M[piv][j];
          M[piv][j] = t;
        }
      for (int r = col + 1; r < 3; ++r) {
        const double fct = M[r][col] / M[col][col];
        for (int j = col; j < 4; ++j) M[r][j] -= fct * M[col][j];
      }
    }
    if (ok) {
      double sol[3];
      for (int r = 2; r >= 0; --r) {
        double v = M[r][3];
        for (int j = r + 1; j < 3; ++j) v -= M[r][j] * sol[j];
        sol[r] = v / M[r][r];
      }
      const double xc = 0.5 * sol[0], yc = 0.5 * sol[1];
      const double R2 = sol[2] + xc * xc + yc * yc;
      if (R2 > 0) {
        const double R = sqrt(R2);
        o.circle[0] = xc + a.ox;
        o.circle[1] = yc + a.oy;
        o.circle[2] = R;
        const double h = (o.circle[0] - a.wx) * a.nx_ + (o.circle[1] - a.wy) * a.ny_;
        const double cth = fmax(-1.0, fmin(1.0, -h / R));
        o.contact_angle_deg = acos(cth) * (180.0 / M_PI);
      }
    }
  }
  return LBM_OK;
}

lbm_status lbm_interface_count(lbm_ctx* c, int64_t* n) {
  if (!c || !n) return LBM_ERR_ARG;
  if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "no geometry");
  *n = c->n_iface;
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_ERR_ARG;
  lbm_status s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return s ? s : check_timeout(c);
}

lbm_status lbm_run_host(lbm_ctx* c, const lbm_wetting_params* w, const uint8_t* h_mask, const double* h_rhoA,
                        const double* h_rhoB, int32_t nsteps, double* oA, double* oB, double* oux, double* ouy) {
  if (!c || !w || !h_mask || !h_rhoA || !h_rhoB || nsteps < 0) return LBM_ERR_ARG;
  const int64_t N = (int64_t)c->g.nx * c->g.ny;
  double* in = c->stage;  // rhoA at [0, N), rhoB at [N, 2N)
  lbm_status s = check_cuda(c, cudaMemcpyAsync(c->stage_mask, h_mask, N, cudaMemcpyHostToDevice, c->stream),
                            "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaMemcpyAsync(in, h_rhoA, N * 8, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaMemcpyAsync(in + N, h_rhoB, N * 8, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  if (!s) s = lbm_set_geometry(c, c->stage_mask);
  if (!s) s = lbm_set_wetting(c, w);
  if (!s) s = lbm_init_fields(c, in, in + N, nullptr, nullptr);
  if (!s) s = lbm_step(c, nsteps);
  if (s) return s;
  LBM_DISPATCH(c, s = (do_eval<T, 1>(c, c->stage)); break);
  double* outs[4] = {oA, oB, oux, ouy};
  for (int a = 0; a < 4 && !s; ++a)
    if (outs[a])
      s = check_cuda(c, cudaMemcpyAsync(outs[a], c->stage + a * N, N * 8, cudaMemcpyDeviceToHost, c->stream),
                     "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return s;
}

lbm_status lbm_run_host_f32(lbm_ctx* c, const lbm_wetting_params* w, const uint8_t* h_mask, const float* h_rhoA,
                            const float* h_rhoB, int32_t nsteps, float* oA, float* oB, float* oux, float* ouy) {
  if (!c || !w || !h_mask || !h_rhoA || !h_rhoB || nsteps < 0) return LBM_ERR_ARG;
  const int64_t N = (int64_t)c->g.nx * c->g.ny;
  // staging (4 N doubles): the FP32 inputs in its last quarter, widened to
  // doubles in its first half; the FP32 moments later in its first half
  float* in32 = reinterpret_cast<float*>(c->stage + 3 * N);
  double* in = c->stage;
  lbm_status s = check_cuda(c, cudaMemcpyAsync(c->stage_mask, h_mask, N, cudaMemcpyHostToDevice, c->stream),
                            "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaMemcpyAsync(in32, h_rhoA, N * 4, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaMemcpyAsync(in32 + N, h_rhoB, N * 4, cudaMemcpyHostToDevice, c->stream),
                         "cudaMemcpyAsync");
  if (s) return s;
  k_widen<<<(unsigned)((2 * N + 255) / 256), 256, 0, c->stream>>>(in32, in, 2 * N);
  if ((s = after_launch(c, "k_widen"))) return s;
  s = lbm_set_geometry(c, c->stage_mask);
  if (!s) s = lbm_set_wetting(c, w);
  if (!s) s = lbm_init_fields(c, in, in + N, nullptr, nullptr);
  if (!s) s = lbm_step(c, nsteps);
  if (s) return s;
  float* out = reinterpret_cast<float*>(c->stage);
  LBM_DISPATCH(c, s = (do_eval<T, 1, float>(c, out)); break);
  float* outs[4] = {oA, oB, oux, ouy};
  for (int a = 0; a < 4 && !s; ++a)
    if (outs[a])
      s = check_cuda(c, cudaMemcpyAsync(outs[a], out + a * N, N * 4, cudaMemcpyDeviceToHost, c->stream),
                     "cudaMemcpyAsync");
  if (!s) s = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return s;
}

lbm_status lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_ERR_ARG;
  delete c;
  return LBM_OK;
}

}  // extern "C"
