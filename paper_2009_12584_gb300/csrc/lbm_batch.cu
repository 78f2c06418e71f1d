// Batched stepping of many independent simulations (contexts): each step is
// one launch per kernel class over all members, through block tables that
// map a CTA to (member, first list entry) or (member, tile), replayed from
// a CUDA graph. Two schedules, as for a single simulation: the two-pass one
// (density pass, Eq. 8 pass, collide pass) and, for 4- and 8-byte storage
// with tile lists, the tiled single pass (Eq. 8 pass, tiled step).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

// What a batched kernel needs of one simulation. cur / pcur are the
// context's buffer indices at the start of an lbm_batch_step call; step k of
// the call uses parity k & 1 relative to them.
template <typename C>
struct BatchDesc {
  const void* f[2];
  void* Pbuf[2];
  UPair* Ubuf[2];  // 16-bit storage with velocity references: writers' rho and 3 u of f[0] / f[1]
  const uint16_t* flags;
  const uint16_t* tile_entries;  // tiled schedule: the member's per-tile lists
  const int* tile_off;
  const int2* tile_cnt;
  int n_tiles, ntx;
  const int* fluid_list;
  const int* iface_list;
  const uint32_t* iface_mask;
  int n_fluid, n_iface;
  int cur, pcur;
  Geo g;
  PhysK<C> ph;
};

// Densities of the members' current populations. into: 1 into Pbuf[pcur ^ 1]
// (two-pass: the plane the collide pass reads), 0 into Pbuf[pcur] (tiled:
// rho(t) before the first tiled step; 4- and 8-byte storage).
// VR: whether members' velocity planes may be read (16-bit storage with
// velocity references in at least one member; a member without them has
// null planes). Without it the kernels carry no code for them.
template <typename T, bool VR = false>
__global__ void __launch_bounds__(256) k_density_batch(const BatchDesc<typename Pop<T>::C>* __restrict__ d,
                                                       const int2* __restrict__ blk, int parity, int into) {
  using C = typename Pop<T>::C;
  const int2 b = blk[blockIdx.x];
  const BatchDesc<C>& D = d[b.x];
  const int cur = D.cur ^ parity, pcur = D.pcur ^ parity;
  const int t = b.y + threadIdx.x;
  if (t < D.n_fluid)
    density_node<T>((const T*)D.f[cur], (C*)D.Pbuf[pcur ^ into], (const C*)D.Pbuf[pcur], VR ? D.Ubuf[cur] : nullptr,
                    D.flags,
                    D.fluid_list, t, D.g);
}

// Eq. 8 into the plane the next pass reads: Pbuf[pcur ^ into] (into as
// above).
template <typename C>
__global__ void __launch_bounds__(128) k_virtual_batch(const BatchDesc<C>* __restrict__ d,
                                                       const int2* __restrict__ blk, int parity, int into) {
  const int2 b = blk[blockIdx.x];
  const BatchDesc<C>& D = d[b.x];
  const int pcur = D.pcur ^ parity;
  const int t = b.y + threadIdx.x;
  if (t < D.n_iface) virtual_density_node<C>((C*)D.Pbuf[pcur ^ into], D.iface_mask, D.iface_list, t, D.g, D.ph);
}

// Tiled single-pass step of every member: CTA -> (member, tile).
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS, TILE_MINB)
    k_tile_batch(const BatchDesc<typename Pop<T>::C>* __restrict__ d, const int2* __restrict__ blk, int parity) {
  using C = typename Pop<T>::C;
  const int2 b = blk[blockIdx.x];
  const BatchDesc<C>& D = d[b.x];
  const int cur = D.cur ^ parity, pcur = D.pcur ^ parity;
  tile_step<T>(b.y, D.n_tiles, (const T*)D.f[cur], (T*)D.f[cur ^ 1], (const C*)D.Pbuf[pcur],
               (const C*)D.Pbuf[pcur], nullptr, nullptr, (C*)D.Pbuf[pcur ^ 1], D.flags, D.tile_entries,
               D.tile_off, D.tile_cnt, D.g, D.ntx, D.ph);
}

template <typename T, bool VR = false>
__global__ void __launch_bounds__(256, 4) k_collide_batch(const BatchDesc<typename Pop<T>::C>* __restrict__ d,
                                                       const int2* __restrict__ blk, int parity) {
  using C = typename Pop<T>::C;
  const int2 b = blk[blockIdx.x];
  const BatchDesc<C>& D = d[b.x];
  const int cur = D.cur ^ parity, pcur = D.pcur ^ parity;
  collide_node<T>((const T*)D.f[cur], (T*)D.f[cur ^ 1], (const C*)D.Pbuf[pcur ^ 1], (const C*)D.Pbuf[pcur],
                  VR ? D.Ubuf[cur] : nullptr, VR ? D.Ubuf[cur ^ 1] : nullptr, D.flags, D.fluid_list, b.y + threadIdx.x,
                  D.n_fluid, D.g, D.ph);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
size_t desc_bytes(int storage) {
  return storage == LBM_STORE_FP64 ? sizeof(BatchDesc<double>) : sizeof(BatchDesc<float>);
}

// block-table entries for lists of the given lengths and block size
int64_t table_entries(const int* lens, int n, int bs) {
  int64_t e = 0;
  for (int s = 0; s < n; ++s) e += (lens[s] + bs - 1) / bs;
  return e;
}

}  // namespace

struct lbm_batch {
  int n;
  lbm_ctx** ctx;
  int storage;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  void* d_desc;
  int2* d_fblk;
  int2* d_iblk;
  int2* d_tblk;         // tiled schedule: (member, tile) per CTA (null if unavailable)
  int n_fblk, n_iblk, n_tblk;
  int schedule;         // LBM_KERNEL_TWO_PASS or LBM_KERNEL_TILED
  bool tiled_ok;        // 4- or 8-byte storage and every member keeps tile lists
  bool vr;              // 16-bit storage and some member keeps velocity references
  int bs;               // threads per block of the density and collide kernels
  void* h_desc;         // host staging of the descriptors
  int2* h_tab;          // host staging of the block tables
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int graph_steps;      // steps per graph replay (even), 0 = no graph
  int64_t launches;
  char err[256];
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const char* msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
  return s;
}

lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return LBM_OK;
  if (b) snprintf(b->err, sizeof(b->err), "%s: %s", where, cudaGetErrorString(e));
  return LBM_ERR_CUDA;
}

// Device layout of a batch workspace: descriptors, fluid block table (sized
// for the smallest block size), interface block table, tile block table.
struct BLayout {
  size_t desc, fblk, iblk, tblk, total;
};

// The tiled schedule runs when the storage is 4 or 8 bytes and every member
// keeps the per-tile lists (contexts created with LBM_KERNEL_AUTO or TILED).
bool batch_tiled_ok(int n, lbm_ctx* const* ctxs) {
  if (ctxs[0]->prm.storage != LBM_STORE_FP32 && ctxs[0]->prm.storage != LBM_STORE_FP64) return false;
  for (int s = 0; s < n; ++s)
    if (ctxs[s]->n_tiles <= 0) return false;
  return true;
}

BLayout blayout(int n, lbm_ctx* const* ctxs) {
  int* lf = (int*)malloc(sizeof(int) * n);
  int* li = (int*)malloc(sizeof(int) * n);
  for (int s = 0; s < n; ++s) {
    lf[s] = ctxs[s]->n_fluid;
    li[s] = ctxs[s]->ph.bc == BC_VAVG ? ctxs[s]->n_iface : 0;
  }
  BLayout L;
  size_t off = 0;
  L.desc = off;  off = align_up(off + (size_t)n * desc_bytes(ctxs[0]->prm.storage), 256);
  L.fblk = off;  off = align_up(off + (size_t)table_entries(lf, n, 128) * sizeof(int2), 256);
  L.iblk = off;  off = align_up(off + (size_t)table_entries(li, n, 128) * sizeof(int2), 256);
  int64_t nt = 0;
  if (batch_tiled_ok(n, ctxs))
    for (int s = 0; s < n; ++s) nt += ctxs[s]->n_tiles;
  L.tblk = off;  off = align_up(off + (size_t)nt * sizeof(int2), 256);
  L.total = off;
  free(lf);
  free(li);
  return L;
}

// Build a block table in h_tab for lists of length len(s), bs per block.
template <typename LenFn>
int build_table(int2* h_tab, int n, int bs, LenFn len) {
  int e = 0;
  for (int s = 0; s < n; ++s)
    for (int first = 0; first < len(s); first += bs) h_tab[e++] = make_int2(s, first);
  return e;
}

lbm_status upload_fluid_table(lbm_batch* b, int bs) {
  b->bs = bs;
  b->n_fblk = build_table(b->h_tab, b->n, bs, [&](int s) { return b->ctx[s]->n_fluid; });
  lbm_status st = bcuda(b, cudaMemcpyAsync(b->d_fblk, b->h_tab, (size_t)b->n_fblk * sizeof(int2),
                                           cudaMemcpyHostToDevice, b->stream), "cudaMemcpyAsync");
  if (!st) st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  return st;
}

template <typename C>
void fill_descs(lbm_batch* b) {
  BatchDesc<C>* h = (BatchDesc<C>*)b->h_desc;
  for (int s = 0; s < b->n; ++s) {
    const lbm_ctx* c = b->ctx[s];
    BatchDesc<C>& d = h[s];
    d.f[0] = c->f[0];
    d.f[1] = c->f[1];
    d.Pbuf[0] = c->Pbuf[0];
    d.Pbuf[1] = c->Pbuf[1];
    d.Ubuf[0] = c->Ubuf[0];
    d.Ubuf[1] = c->Ubuf[1];
    d.flags = c->flags;
    d.tile_entries = c->tile_entries;
    d.tile_off = c->tile_off;
    d.tile_cnt = c->tile_cnt;
    d.n_tiles = (int)c->n_tiles;
    d.ntx = (c->g.nx + TILE_W - 1) / TILE_W;
    d.fluid_list = c->fluid_list;
    d.iface_list = c->iface_list;
    d.iface_mask = c->iface_mask;
    d.n_fluid = c->n_fluid;
    d.n_iface = c->ph.bc == BC_VAVG ? c->n_iface : 0;
    d.cur = c->cur;
    d.pcur = c->pcur;
    d.g = c->g;
    d.ph = kphys<C>(c->ph);
  }
}

// Enqueue one step (parity p) directly on the stream.
template <typename T>
lbm_status launch_step(lbm_batch* b, int p) {
  using C = typename Pop<T>::C;
  const BatchDesc<C>* d = (const BatchDesc<C>*)b->d_desc;
  if (b->schedule == LBM_KERNEL_TILED) {
    if constexpr (sizeof(T) >= 4) {
      if (b->n_iblk > 0) {
        k_virtual_batch<C><<<b->n_iblk, 128, 0, b->stream>>>(d, b->d_iblk, p, 0);
        b->launches++;
      }
      if (b->n_tblk > 0) {
        k_tile_batch<T><<<b->n_tblk, TILE_THREADS, tile_smem<T>(), b->stream>>>(d, b->d_tblk, p);
        b->launches++;
      }
    }
    return bcuda(b, cudaGetLastError(), "batched tiled step launch");
  }
  const bool vr = kDev<T> && b->vr;
  if (b->n_fblk > 0) {
    auto kd = vr ? k_density_batch<T, kDev<T>> : k_density_batch<T, false>;
    kd<<<b->n_fblk, b->bs, 0, b->stream>>>(d, b->d_fblk, p, 1);
    b->launches++;
  }
  if (b->n_iblk > 0) {
    k_virtual_batch<C><<<b->n_iblk, 128, 0, b->stream>>>(d, b->d_iblk, p, 1);
    b->launches++;
  }
  if (b->n_fblk > 0) {
    auto kc = vr ? k_collide_batch<T, kDev<T>> : k_collide_batch<T, false>;
    kc<<<b->n_fblk, b->bs, 0, b->stream>>>(d, b->d_fblk, p);
    b->launches++;
  }
  return bcuda(b, cudaGetLastError(), "batched step launch");
}

// Kernel launches per step of the current schedule.
int launches_per_step(const lbm_batch* b) {
  if (b->schedule == LBM_KERNEL_TILED) return (b->n_iblk > 0) + (b->n_tblk > 0);
  return (b->n_fblk > 0) * 2 + (b->n_iblk > 0);
}

void drop_graph(lbm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_steps = 0;
}

// Build (without stream capture) a graph of `steps` consecutive steps.
template <typename T>
lbm_status build_graph(lbm_batch* b, int steps) {
  using C = typename Pop<T>::C;
  drop_graph(b);
  if (steps <= 0) return LBM_OK;
  lbm_status st = bcuda(b, cudaGraphCreate(&b->graph, 0), "cudaGraphCreate");
  if (st) return st;
  const BatchDesc<C>* d = (const BatchDesc<C>*)b->d_desc;
  cudaGraphNode_t prev = nullptr;
  const bool tiled = b->schedule == LBM_KERNEL_TILED;
  void* tile_fn = nullptr;
  if constexpr (sizeof(T) >= 4) tile_fn = (void*)k_tile_batch<T>;
  for (int k = 0; k < steps && !st; ++k) {
    int p = k & 1;
    int into = tiled ? 0 : 1;
    const int2* tabs[3] = {b->d_fblk, b->d_iblk, tiled ? b->d_tblk : b->d_fblk};
    const bool vr = kDev<T> && b->vr;
    void* fns[3] = {vr ? (void*)k_density_batch<T, kDev<T>> : (void*)k_density_batch<T, false>,
                    (void*)k_virtual_batch<C>,
                    tiled ? tile_fn : vr ? (void*)k_collide_batch<T, kDev<T>> : (void*)k_collide_batch<T, false>};
    const int grids[3] = {tiled ? 0 : b->n_fblk, b->n_iblk, tiled ? b->n_tblk : b->n_fblk};
    const int blocks[3] = {b->bs, 128, tiled ? TILE_THREADS : b->bs};
    const size_t smem[3] = {0, 0, tiled ? tile_smem<T>() : 0};
    for (int q = 0; q < 3 && !st; ++q) {
      if (grids[q] <= 0) continue;
      const int2* tab = tabs[q];
      void* args[4] = {(void*)&d, (void*)&tab, (void*)&p, (void*)&into};
      cudaKernelNodeParams kp;
      memset(&kp, 0, sizeof(kp));
      kp.func = fns[q];
      kp.gridDim = dim3(grids[q]);
      kp.blockDim = dim3(blocks[q]);
      kp.sharedMemBytes = (unsigned)smem[q];
      kp.kernelParams = args;
      cudaGraphNode_t node;
      st = bcuda(b, cudaGraphAddKernelNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp),
                 "cudaGraphAddKernelNode");
      prev = node;
    }
  }
  if (!st) st = bcuda(b, cudaGraphInstantiate(&b->exec, b->graph, 0), "cudaGraphInstantiate");
  if (st) {
    drop_graph(b);
    return st;
  }
  b->graph_steps = steps;
  return LBM_OK;
}

template <typename T>
lbm_status batch_step(lbm_batch* b, int nsteps) {
  using C = typename Pop<T>::C;
  fill_descs<C>(b);
  lbm_status st = bcuda(b, cudaMemcpyAsync(b->d_desc, b->h_desc, (size_t)b->n * sizeof(BatchDesc<C>),
                                           cudaMemcpyHostToDevice, b->stream), "cudaMemcpyAsync");
  // the staging buffer is rewritten by the next call: wait for the copy
  if (!st) st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  const bool tiled = b->schedule == LBM_KERNEL_TILED;
  if (!st && tiled && nsteps > 0) {
    // the tiled step reads rho(t) from Pbuf[pcur]: compute it for every
    // member once (a member whose plane already holds it gets the same bits)
    bool all_valid = true;
    for (int s = 0; s < b->n; ++s) all_valid = all_valid && b->ctx[s]->p_valid;
    if (!all_valid && b->n_fblk > 0) {
      k_density_batch<T><<<b->n_fblk, b->bs, 0, b->stream>>>((const BatchDesc<C>*)b->d_desc, b->d_fblk, 0, 0);
      b->launches++;
      st = bcuda(b, cudaGetLastError(), "batched density launch");
    }
  }
  int done = 0;
  if (b->exec && b->graph_steps > 0)
    for (; !st && done + b->graph_steps <= nsteps; done += b->graph_steps) {
      st = bcuda(b, cudaGraphLaunch(b->exec, b->stream), "cudaGraphLaunch");
      b->launches += (int64_t)b->graph_steps * launches_per_step(b);
    }
  for (; !st && done < nsteps; ++done) st = launch_step<T>(b, done & 1);
  if (st) return st;
  for (int s = 0; s < b->n; ++s) {
    lbm_ctx* c = b->ctx[s];
    if (nsteps & 1) {
      c->cur ^= 1;
      c->pcur ^= 1;
      c->P = c->Pbuf[c->pcur];
    }
    // after tiled steps Pbuf[pcur] holds rho of the current state
    c->p_valid = tiled && (nsteps > 0 || c->p_valid);
  }
  return LBM_OK;
}

#define BATCH_DISPATCH(b, CALL)                          \
  switch ((b)->storage) {                                \
    case LBM_STORE_FP32: { using T = float; CALL; }      \
    case LBM_STORE_FP64: { using T = double; CALL; }     \
    case LBM_STORE_FP16: { using T = __half; CALL; }     \
    default: { using T = __nv_bfloat16; CALL; }          \
  }

lbm_status check_members(int32_t n, lbm_ctx* const* ctxs) {
  if (n < 1 || !ctxs) return LBM_ERR_ARG;
  for (int s = 0; s < n; ++s) {
    if (!ctxs[s]) return LBM_ERR_ARG;
    if (ctxs[s]->prm.storage != ctxs[0]->prm.storage || ctxs[s]->device != ctxs[0]->device) return LBM_ERR_ARG;
    if (!ctxs[s]->has_geometry || !ctxs[s]->has_fields) return LBM_ERR_STATE;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_bytes(int32_t n, lbm_ctx* const* ctxs, size_t* bytes) {
  if (!bytes) return LBM_ERR_ARG;
  lbm_status st = check_members(n, ctxs);
  if (st) return st;
  *bytes = blayout(n, ctxs).total;
  return LBM_OK;
}

lbm_status lbm_batch_create(int32_t n, lbm_ctx* const* ctxs, void* d_workspace, size_t bytes, void* cuda_stream,
                            lbm_batch** out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_status st = check_members(n, ctxs);
  if (st) return st;
  if (!d_workspace || ((uintptr_t)d_workspace) % 256) return LBM_ERR_ARG;
  const BLayout L = blayout(n, ctxs);
  if (bytes < L.total) return LBM_ERR_SPACE;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_SPACE;
  b->n = n;
  b->storage = ctxs[0]->prm.storage;
  b->stream = (cudaStream_t)cuda_stream;
  b->ws = (char*)d_workspace;
  b->ws_bytes = bytes;
  b->d_desc = b->ws + L.desc;
  b->d_fblk = (int2*)(b->ws + L.fblk);
  b->d_iblk = (int2*)(b->ws + L.iblk);
  b->tiled_ok = batch_tiled_ok(n, ctxs);
  b->vr = false;
  for (int i = 0; i < n; ++i) b->vr = b->vr || ctxs[i]->Ubuf[0] != nullptr;
  b->d_tblk = b->tiled_ok ? (int2*)(b->ws + L.tblk) : nullptr;
  b->schedule = LBM_KERNEL_TWO_PASS;
  b->ctx = (lbm_ctx**)malloc(sizeof(lbm_ctx*) * n);
  b->h_desc = malloc((size_t)n * desc_bytes(b->storage));
  // host staging large enough for any table (fluid and interface tables at
  // 128 threads per block, the tile table)
  int64_t tab_cap = 1;
  {
    int64_t ef = 0, ei = 0, et = 0;
    for (int s = 0; s < n; ++s) {
      ef += (ctxs[s]->n_fluid + 127) / 128;
      ei += ctxs[s]->ph.bc == BC_VAVG ? (ctxs[s]->n_iface + 127) / 128 : 0;
      et += b->tiled_ok ? ctxs[s]->n_tiles : 0;
    }
    tab_cap += ef > ei ? (ef > et ? ef : et) : (ei > et ? ei : et);
  }
  b->h_tab = (int2*)malloc((size_t)tab_cap * sizeof(int2));
  if (!b->ctx || !b->h_desc || !b->h_tab) {
    free(b->ctx);
    free(b->h_desc);
    free(b->h_tab);
    delete b;
    return LBM_ERR_SPACE;
  }
  for (int s = 0; s < n; ++s) b->ctx[s] = ctxs[s];
  // interface blocks (128 threads), only for simulations with the improved scheme
  b->n_iblk = build_table(b->h_tab, n, 128, [&](int s) {
    return b->ctx[s]->ph.bc == BC_VAVG ? b->ctx[s]->n_iface : 0;
  });
  st = bcuda(b, cudaMemcpyAsync(b->d_iblk, b->h_tab, (size_t)b->n_iblk * sizeof(int2), cudaMemcpyHostToDevice,
                                b->stream), "cudaMemcpyAsync");
  if (!st) st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (!st) st = upload_fluid_table(b, 256);
  if (!st && b->tiled_ok) {
    // tile blocks: every tile of every member, member by member
    int e = 0;
    for (int s = 0; s < n; ++s)
      for (int64_t t = 0; t < b->ctx[s]->n_tiles; ++t) b->h_tab[e++] = make_int2(s, (int)t);
    b->n_tblk = e;
    st = bcuda(b, cudaMemcpyAsync(b->d_tblk, b->h_tab, (size_t)e * sizeof(int2), cudaMemcpyHostToDevice, b->stream),
               "cudaMemcpyAsync");
    if (!st) st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (!st && b->storage == LBM_STORE_FP64)
      st = bcuda(b, cudaFuncSetAttribute(k_tile_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tile_smem<double>()), "cudaFuncSetAttribute");
  }
  if (st) {
    free(b->ctx);
    free(b->h_desc);
    free(b->h_tab);
    delete b;
    return st;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_set_graph_steps(lbm_batch* b, int32_t steps) {
  if (!b || steps < 0 || (steps & 1)) return LBM_ERR_ARG;
  lbm_status st;
  BATCH_DISPATCH(b, st = build_graph<T>(b, steps); break);
  return st;
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return LBM_ERR_ARG;
  for (int s = 0; s < b->n; ++s)
    if (!b->ctx[s]->has_geometry || !b->ctx[s]->has_fields) return bfail(b, LBM_ERR_STATE, "member without fields");
  lbm_status st;
  BATCH_DISPATCH(b, st = batch_step<T>(b, nsteps); break);
  return st;
}

lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t kernel) {
  if (!b) return LBM_ERR_ARG;
  if (kernel != LBM_KERNEL_TWO_PASS && kernel != LBM_KERNEL_TILED) return bfail(b, LBM_ERR_ARG, "unknown schedule");
  if (kernel == LBM_KERNEL_TILED && !b->tiled_ok)
    return bfail(b, LBM_ERR_ARG, "tiled schedule needs 4- or 8-byte storage and members with tile lists");
  b->schedule = kernel;
  return b->graph_steps > 0 ? lbm_batch_set_graph_steps(b, b->graph_steps) : LBM_OK;
}

lbm_status lbm_batch_config(const lbm_batch* b, int32_t* h_cfg) {
  if (!b || !h_cfg) return LBM_ERR_ARG;
  h_cfg[0] = b->schedule;
  h_cfg[1] = b->schedule == LBM_KERNEL_TILED ? TILE_THREADS : b->bs;
  h_cfg[2] = b->graph_steps;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, int32_t* h_choice) {
  if (!b || trial_steps < 2) return LBM_ERR_ARG;
  // candidates: the two-pass schedule at 128 or 256 threads per block, and
  // the tiled one when available; 2, 8 or 32 steps per graph replay
  struct Cand { int schedule, bs; };
  const Cand kCand[3] = {{LBM_KERNEL_TWO_PASS, 128}, {LBM_KERNEL_TWO_PASS, 256}, {LBM_KERNEL_TILED, 256}};
  static const int kSteps[3] = {2, 8, 32};
  cudaEvent_t e0, e1;
  lbm_status st = bcuda(b, cudaEventCreate(&e0), "cudaEventCreate");
  if (st) return st;
  st = bcuda(b, cudaEventCreate(&e1), "cudaEventCreate");
  if (st) {
    cudaEventDestroy(e0);
    return st;
  }
  float best = 1e30f;
  Cand best_c = kCand[1];
  int best_steps = 2;
  for (int ic = 0; ic < 3 && !st; ++ic) {
    if (kCand[ic].schedule == LBM_KERNEL_TILED && !b->tiled_ok) continue;
    st = upload_fluid_table(b, kCand[ic].bs);
    if (!st) st = lbm_batch_set_schedule(b, kCand[ic].schedule);
    for (int is = 0; is < 3 && !st; ++is) {
      const int S = kSteps[is];
      st = lbm_batch_set_graph_steps(b, S);
      const int reps = (trial_steps + S - 1) / S;
      if (!st) st = lbm_batch_step(b, S);  // warm-up
      if (!st) st = bcuda(b, cudaEventRecord(e0, b->stream), "cudaEventRecord");
      if (!st) st = lbm_batch_step(b, reps * S);
      if (!st) st = bcuda(b, cudaEventRecord(e1, b->stream), "cudaEventRecord");
      if (!st) st = bcuda(b, cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      if (!st) st = bcuda(b, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (!st && ms / (reps * S) < best) {
        best = ms / (reps * S);
        best_c = kCand[ic];
        best_steps = S;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!st) st = upload_fluid_table(b, best_c.bs);
  if (!st) st = lbm_batch_set_schedule(b, best_c.schedule);
  if (!st) st = lbm_batch_set_graph_steps(b, best_steps);
  if (!st && h_choice) {
    h_choice[0] = best_c.schedule == LBM_KERNEL_TILED ? TILE_THREADS : best_c.bs;
    h_choice[1] = best_steps;
  }
  return st;
}

int64_t lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : ""; }

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_ERR_ARG;
  drop_graph(b);
  free(b->ctx);
  free(b->h_desc);
  free(b->h_tab);
  delete b;
  return LBM_OK;
}

}  // extern "C"
