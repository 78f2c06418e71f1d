// Internal definitions shared by the translation units of the library: the
// context object behind the opaque lbm_ctx handle.
#pragma once

#include "lbm.h"
#include "lbm_fused.cuh"
#include "lbm_geometry.cuh"
#include "lbm_halo.cuh"
#include "lbm_kernels.cuh"
#include "lbm_tiled.cuh"
#include "lbm_tma.cuh"

using lbm::Geo;
using lbm::Phys;
using lbm::UPair;

struct lbm_ctx {
  // TMA schedule: tensor maps of the population buffers f[0], f[1] (rank 3:
  // 2 px floats, py rows, 9 planes) and the density planes Pbuf[0], Pbuf[1]
  // (rank 2), encoded at creation
  alignas(64) CUtensorMap tmap_f[2];
  alignas(64) CUtensorMap tmap_P[2];
  bool tma;            // the TMA schedule runs (FP32 storage, LBM_KERNEL_TMA)
  bool tma_smem_set;   // k_tile_tma's dynamic shared memory limit raised
  lbm_params prm;
  Geo g;
  Phys ph;
  cudaStream_t stream;
  int device;
  int num_sms;
  // workspace carve-up
  char* ws;
  size_t ws_bytes;
  void* f[2];          // population buffers (storage type)
  void* Pbuf[3];       // density plane pairs (compute type); the third only for
                       // the tiled schedule with 16-bit storage (null otherwise)
  char* Pbase;         // start of the density planes in the workspace
  UPair* Ubuf[2];    // 16-bit storage with velocity_refs: rho and 3 u of the writers of f[0] / f[1]
                       // (the encoding references); null otherwise
  void* P;             // Pbuf[pcur]: the densities the current populations were
                       // written with (16-bit encoding references); after a
                       // single-pass step, the densities of the current state
  int pcur;
  bool p_valid;        // P holds the densities of the current state (single-pass)
  uint16_t* flags;
  int* iface_list;
  uint32_t* iface_mask; // fluid neighbours of each interface-solid cell (5 x 5 stencil bits)
  int* fluid_list;     // fluid nodes in node order, edge nodes tagged (padded indices)
  uint16_t* tile_entries; // tiled schedule: per-tile lists of region slots (null if unused)
  int* tile_off;       // tiled schedule: first entry of each tile, total at [ntiles]
  int2* tile_cnt;      // tiled schedule: (owned fluid nodes, listed fluid nodes) of each tile
  int4* tile_work;     // TMA schedule: the tiles with owned nodes, in order: (tile, first entry,
                       // listed nodes, owned nodes); their number at small[5]
  int n_work;          // entries of tile_work (read back by lbm_set_geometry)
  int64_t n_tiles;
  bool tile_smem_set;  // k_tile's dynamic shared memory limit raised on this context's device
  bool march_smem_set;  // k_march's (FP64: above 48 KB) likewise
  bool halo_built;      // the halo lists match the current geometry
  uint32_t tma_extra_tx;  // test hook of the TMA schedule's bounded wait (lbm_debug_tma_expect_extra); 0
  uint16_t* halo_entries; // halo schedule: per-tile lists of region slots (null if unused)
  int* halo_off;       // halo schedule: first entry of each tile, total at [n_halo_tiles]
  int4* halo_cnt;      // halo schedule: cumulative counts (own, +ring 1, +ring 2, +ring 3) per tile
  uint32_t* halo_fmask; // halo schedule: fluid bitmask of each tile's region
  int64_t n_halo_tiles;
  int* scan_counts;    // per-block interface counts / offsets
  int* small;          // [0] error count, [1] interface total, [2] fluid total
  double* partial;     // mass partial sums
  double* mass_out;    // 2 doubles
  uint8_t* stage_mask; // lbm_run_host staging
  double* stage;       // 4 arrays of nx*ny doubles
  double* dpart;       // diagnostics: per-block partial sums, then the reduced values
  int64_t if_capacity;
  int scan_blocks;
  int mass_blocks;
  int n_iface;
  int n_fluid;
  int cur;             // index of the buffer holding the current state
  bool has_geometry, has_fields, has_wetting;
  int64_t launches;
  // lbm_step_profiled: when prof_on, every launch is bracketed by a pair of
  // events from this pool and tagged with its kernel class
  bool prof_on;
  cudaEvent_t* prof_ev;
  int* prof_cls;
  int prof_n, prof_cap;
  char err[512];
};
