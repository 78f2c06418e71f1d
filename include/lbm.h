/*
 * lbm.h - C ABI of the GB300 library for the two-component Shan-Chen
 * pseudopotential lattice Boltzmann step on D2Q9 with wetting boundary
 * conditions (Coelho, Moura, Telo da Gama, Araujo, "Wetting boundary
 * conditions for multicomponent pseudopotential lattice Boltzmann",
 * arXiv:2009.12584).
 *
 * One time step (lbm_step) computes, for both components A and B:
 *   - the densities rho^sigma = sum_i f_i^sigma and pseudopotentials
 *     psi = rho (Eq. 3, Eq. 5),
 *   - the virtual solid densities of the improved scheme at interface-solid
 *     nodes (Eq. 8, D2Q25 weights),
 *   - the Shan-Chen force summed over fluid neighbours (Eq. 5) plus the
 *     adhesion force (Eq. 7) of the selected wetting scheme,
 *   - the common velocity u^eq (Eq. 3), BGK collision towards Eq. 2 with the
 *     Guo source of Eq. 4, streaming and halfway bounce-back (Eq. 1, Sec. 2).
 *
 * Conventions shared by every entry point
 *   - Grids are nx * ny nodes, row-major, node (x, y) at index y*nx + x.
 *     Component 0 is A (the droplet fluid), 1 is B. D2Q9 directions:
 *     0 rest, 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1),
 *     7 (-1,-1), 8 (1,-1).
 *   - "d_" pointers are device pointers the caller owns (e.g. torch tensor
 *     storage); "h_" pointers are host pointers. The library never frees
 *     caller memory and allocates no device memory of its own: every device
 *     buffer lives in the caller-provided workspace. The context object
 *     itself is a small host allocation released by lbm_destroy.
 *   - All device work is enqueued on the context's stream (a cudaStream_t
 *     passed as void*; NULL is the legacy default stream). Calls return when
 *     the work is enqueued, except where a call says it synchronises.
 *   - Every call returns an lbm_status; no call aborts, throws or exits. A
 *     CUDA error is returned as LBM_ERR_CUDA and its text is kept in the
 *     context (lbm_last_error). An asynchronous kernel fault surfaces at the
 *     next call that synchronises.
 *   - Masks: 1 = solid (phi = 1), 0 = fluid (Sec. 2). On a non-periodic axis
 *     the first and last row/column must be solid (the paper's walls on the
 *     box borders, Sec. 3.1); lbm_set_geometry rejects masks with fluid
 *     there.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,     /* invalid argument (null pointer, size, range) */
  LBM_ERR_STATE = 2,   /* call out of order (e.g. step before geometry) */
  LBM_ERR_CUDA = 3,    /* CUDA runtime error; see lbm_last_error */
  LBM_ERR_SPACE = 4,   /* workspace too small for the request */
  LBM_ERR_TIMEOUT = 5  /* a bounded device-side wait gave up */
} lbm_status;

/* Wetting boundary conditions compared in Sec. 2 / Sec. 3. */
typedef enum {
  LBM_WET_MARTYS_CHEN = 0, /* S^sigma = phi; strength G_sigma,s (Eq. 7) */
  LBM_WET_LLKC = 1,        /* S^sigma(x+c_i) = phi(x+c_i) rho^sigma(x) */
  LBM_WET_VIRTUAL_AVG = 2, /* improved scheme: S^sigma = phi rho~^sigma, Eq. 8 */
  LBM_WET_CONSTANT = 3     /* Chen et al.: S^sigma = phi rho_s^sigma */
} lbm_wetting;

/* Which component's solid pseudopotential enters Eq. 7 for the force on
 * sigma. CROSS follows Eq. 7 as printed (S of sigma-bar); SELF uses S of
 * sigma itself, the other reading found in the literature. */
typedef enum { LBM_PAIR_CROSS = 0, LBM_PAIR_SELF = 1 } lbm_pairing;

/* Storage type of the populations. Arithmetic is FP32 for FP32/FP16/BF16
 * and FP64 for FP64. FP16/BF16 store each population as its deviation from
 * a reference its writer and reader both know: w_i times the density of the
 * node that wrote it (kept in a density plane of the workspace), or, with
 * lbm_params.velocity_refs, w_i rho (1 + 3 c_i . u) with that node's
 * velocity too, so the 16 bits carry the non-equilibrium (and, without
 * velocity_refs, the velocity) part only. */
typedef enum {
  LBM_STORE_FP32 = 0,
  LBM_STORE_FP64 = 1,
  LBM_STORE_FP16 = 2,
  LBM_STORE_BF16 = 3
} lbm_storage;

/* Kernel schedule for lbm_step. All schedules give the same results bit for
 * bit.
 * TWO_PASS: a density pass, the virtual density pass, then one fused
 *   force+collide+stream pull kernel.
 * FUSED: one kernel per step that also writes the densities of the next
 *   step (the density plane is double-buffered), warps marching up column
 *   strips; 4- and 8-byte storage only (16-bit storage runs TWO_PASS).
 * TILED: the same single-pass contract on 32 x 14 tiles, one CTA per tile,
 *   each a compacted list of its fluid nodes plus the one-node ring around
 *   it (computed again), built by lbm_set_geometry: the workspace grows by 2
 *   bytes per ring-extended region slot (about 2.4 bytes per node), and for
 *   16-bit storage by a third density plane (8 bytes per padded node), since
 *   a 16-bit step decodes with the densities of the step before.
 * HALO: one kernel per step and no density plane: each CTA takes a 32 x 14
 *   tile, recomputes rho(t) from the pulled populations for the tile and the
 *   1 to 3 node rings its force and Eq. 8 reach (3 for the D2Q25 average, 2
 *   for the D2Q9 average, 1 for the other schemes), evaluates Eq. 8 in
 *   shared memory and updates its own nodes. 4- and 8-byte storage (16-bit
 *   storage runs TWO_PASS); the workspace grows by about 4 bytes per node.
 *   The fastest schedule under Martys-Chen, LLKC and the constant solid
 *   density (one ring); slower than TILED under the improved scheme.
 * TMA: the TILED schedule (same lists, same results bit for bit) with two
 *   persistent CTAs per SM walking a list of the tiles that own fluid
 *   nodes; each tile's inputs, the nine population planes and the density
 *   plane over its (32 + 4) x (14 + 4) window and its entry list, are
 *   copied into shared memory by the Tensor Memory Accelerator into a
 *   two-stage ring, one tile ahead of the update. FP32 storage (other
 *   storage runs TILED); the workspace grows by 16 bytes per tile. A copy
 *   not seen to complete within about a second stops the kernel and is
 *   reported as LBM_ERR_TIMEOUT by the next lbm_sync, lbm_mass or
 *   lbm_step_profiled. Slower than TILED on GB300 (the windows also carry
 *   the solid slots that the tiled kernel's lists skip).
 * AUTO picks the schedule measured fastest on GB300, at each step from the
 * installed wetting scheme: for 4- and 8-byte storage TILED under the
 * improved scheme (a quarter fewer bytes than TWO_PASS and 8% faster on the
 * 8192^2 porous medium) and HALO under Martys-Chen, LLKC and the constant
 * solid density (6% faster than TILED there); the workspace keeps both sets
 * of lists and the halo lists are built at the first step that needs them.
 * TWO_PASS for 16-bit storage. */
typedef enum {
  LBM_KERNEL_AUTO = 0,
  LBM_KERNEL_TWO_PASS = 1,
  LBM_KERNEL_FUSED = 2,
  LBM_KERNEL_TILED = 3,
  LBM_KERNEL_HALO = 4,
  LBM_KERNEL_TMA = 5
} lbm_kernel;

typedef struct {
  int32_t nx, ny;             /* grid size, each >= 4 */
  int32_t periodic_x;         /* 1: periodic along x; 0: walls */
  int32_t periodic_y;         /* 1: periodic along y; 0: walls */
  double tau[2];              /* BGK relaxation times, > 0.5 (Eq. 1) */
  double G_AB;                /* Shan-Chen strength G_AB = G_BA (Eq. 5) */
  int32_t storage;            /* lbm_storage */
  int32_t kernel;             /* lbm_kernel */
  double rho_ref[2];          /* reserved, ignored (set to 0) */
  int64_t max_interface;      /* capacity of the interface-solid list;
                                 0 -> nx*ny (always enough) */
  int32_t velocity_refs;      /* 16-bit storage only: 1 stores each population
                                 as its deviation from w_i rho (1 + 3 c_i . u)
                                 of its writer (per component; the writer's
                                 rho in FP32 and u in FP16 kept in two
                                 velocity planes, 32 more bytes per padded
                                 node; slower, holds moving droplets far more
                                 accurately); 0 (default) from w_i rho */
} lbm_params;

typedef struct {
  int32_t kind;               /* lbm_wetting */
  int32_t pairing;            /* lbm_pairing */
  int32_t avg_stencil;        /* Eq. 8 weights: 25 (D2Q25, the paper's
                                 choice) or 9 (D2Q9 variant) */
  int32_t reserved;
  double G_s[2];              /* G_As, G_Bs of Eq. 7. Martys-Chen and LLKC
                                 in the paper: G_As = -G_Bs = G_w (Sec. 3.1);
                                 virtual densities: G_As = G_Bs = G_AB */
  double chi[2];              /* chi^A, chi^B of Eq. 8 (VIRTUAL_AVG) */
  double rho_s[2];            /* rho_s^A, rho_s^B (CONSTANT) */
} lbm_wetting_params;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of device workspace a context with these parameters needs.
 * Returns LBM_ERR_ARG for invalid parameters (nx or ny < 4, tau <= 0.5,
 * unknown storage/kernel, a grid whose padded index space, (nx + 36 rounded
 * up to a multiple of 32) x (ny + 8), reaches 2^30: about 32,700 x 32,700 nodes). */
lbm_status lbm_workspace_bytes(const lbm_params* params, size_t* bytes);

/* Create a context on the caller's workspace (device memory of at least
 * lbm_workspace_bytes, 256-byte aligned, owned by the caller and kept alive
 * until lbm_destroy) and stream. Enqueues a clear of the workspace. */
lbm_status lbm_create(const lbm_params* params, void* d_workspace, size_t bytes,
                      void* cuda_stream, lbm_ctx** out);

/* Replace the stream later work is enqueued on. */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Install the solid mask d_mask (uint8 [ny][nx], 1 = solid, device).
 * Builds the per-node neighbour flags and the list of interface-solid nodes
 * (solid nodes with a fluid D2Q9 neighbour, Sec. 2 last paragraph; done
 * once, Sec. 3.2). Synchronises. LBM_ERR_ARG if a fluid node lies on a
 * non-periodic border; LBM_ERR_SPACE if the interface list exceeds
 * max_interface. Invalidates the populations (call lbm_init_fields). */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* d_mask);

/* Select the wetting scheme and its parameters (Sec. 2). LBM_ERR_ARG for an
 * unknown kind/pairing, avg_stencil not 9 or 25, or chi outside (0, 2]. */
lbm_status lbm_set_wetting(lbm_ctx* ctx, const lbm_wetting_params* w);

/* Initialise the populations to the equilibrium of Eq. 2 with the given
 * densities and velocity (double [ny][nx] device arrays; d_ux/d_uy may be
 * NULL for u = 0). Solid nodes are ignored. Requires lbm_set_geometry. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* d_rhoA, const double* d_rhoB,
                           const double* d_ux, const double* d_uy);

/* Advance nsteps time steps (Eq. 1). Requires geometry and fields. */
lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps);

/* Kernel classes reported by lbm_step_profiled. */
enum {
  LBM_KC_DENSITY = 0, /* two-pass density pass */
  LBM_KC_VIRTUAL = 1, /* virtual solid densities of Eq. 8 */
  LBM_KC_COLLIDE = 2, /* two-pass force + collide + stream */
  LBM_KC_FUSED = 3,   /* single-pass step */
  LBM_KC_COUNT = 4
};

/* lbm_step with a CUDA event recorded on the context's stream around every
 * kernel launch. Writes the summed device time per kernel class to
 * h_ms[LBM_KC_COUNT] and the launch counts to h_launches[LBM_KC_COUNT]
 * (host arrays; either may be NULL). Synchronises. */
lbm_status lbm_step_profiled(lbm_ctx* ctx, int32_t nsteps, double* h_ms, int64_t* h_launches);

/* Current densities and common velocity u^eq of Eq. 3 (which includes half
 * the force) as double [ny][nx] device arrays; any pointer may be NULL.
 * Solid nodes get 0 (rho~ is not reported). */
lbm_status lbm_moments(lbm_ctx* ctx, double* d_rhoA, double* d_rhoB, double* d_ux,
                       double* d_uy);

/* Interaction force F^sigma (Eq. 5 + Eq. 7) of the current state: double
 * [2 components][2 axes][ny][nx] device array, 0 at solid nodes. */
lbm_status lbm_forces(lbm_ctx* ctx, double* d_F);

/* Post-streaming populations f_i^sigma(x, t) (the left-hand side of Eq. 1)
 * as double [2][9][ny][nx] device array, 0 at solid nodes. */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* d_f);

/* Overwrite the state with post-streaming populations in the layout of
 * lbm_get_populations (checkpoint restore). Requires lbm_set_geometry. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* d_f);

/* Total mass of each component, sum over fluid nodes of rho^sigma,
 * accumulated in FP64 in a fixed order (deterministic). Synchronises and
 * writes h_out[2] on the host. */
lbm_status lbm_mass(lbm_ctx* ctx, double* h_out);

/* Set the L2 fetch granularity hint (cudaLimitMaxL2FetchGranularity) of the
 * current device's context to `bytes` (32, 64 or 128) and write the previous
 * value to *previous (may be NULL). The step pulls populations from rows of
 * fluid nodes broken by solid cells; with 32-byte fetches the L2 stops
 * reading the unused neighbouring sectors at every wall segment end (on the
 * 8192^2 porous medium: density pass -13%, collide pass -3%, step -6% against
 * the 128-byte default). The hint applies to every kernel of the calling
 * process on that device, which is why the library never sets it by itself;
 * it lasts until changed or the process exits. Host-only, not stream-ordered.
 * LBM_ERR_ARG for another size, LBM_ERR_CUDA if the runtime refuses. The
 * paper has no counterpart. */
lbm_status lbm_set_l2_fetch_granularity(int32_t bytes, int32_t* previous);

/* Test hook of the TMA schedule's bounded wait (not for production use):
 * from the next step on, the barrier of every tile's copies expects `bytes`
 * (0 ... 4096) more than the copies deliver, so that its wait runs out
 * after about a second, each CTA stops after waiting (bounded) for the
 * copies it has in flight, and the next lbm_sync, lbm_mass or
 * lbm_step_profiled returns LBM_ERR_TIMEOUT; the populations of that step
 * are then incomplete (re-initialise or restore them). 0, the default,
 * restores normal operation. No effect on other schedules. LBM_ERR_ARG for
 * a null context or a size out of range. */
lbm_status lbm_debug_tma_expect_extra(lbm_ctx* ctx, int32_t bytes);

/* ---- On-device diagnostics ----------------------------------------------
 * The measurements of Secs. 3-4 of arXiv:2009.12584, reduced on the device
 * from the current moments (rho^A, u of Eq. 3) so that long runs copy no
 * fields to the host:
 *  - sliding velocity (Sec. 3.1): centre-of-mass velocity of the A phase
 *    weighted by w = max(rho^A - rho_out, 0) at fluid nodes, and its
 *    projection on a unit tangent;
 *  - contact angle (Sec. 3.2): the points where rho^A crosses `level` on grid
 *    edges joining two fluid nodes (linear interpolation), minus those within
 *    `exclude` of the wall line (and outside `box`), fitted by the algebraic
 *    least-squares (Kasa) circle; cos(theta) = -h / R with h the signed
 *    distance from the wall line to the centre, positive on the fluid side
 *    (the left-hand normal of the wall direction (cos b, sin b));
 *  - bridge radius (Sec. 4): on column bridge_x, the distance from the
 *    halfway wall (half a node below bridge_y0, the first fluid node above
 *    the surface) to the first point above it where rho^A drops through
 *    `level`; 0 while rho^A(bridge_x, bridge_y0) < level;
 *  - max |u| over fluid nodes (the spurious-current level of Sec. 4), and the
 *    number of fluid nodes whose moments are not finite (a diverged run).
 * Sums are FP64 in a fixed order (deterministic); the 3x3 normal equations of
 * the fit are solved on the host. Contour edges do not wrap periodic axes. */
typedef struct {
  double level;           /* rho^A level of the interface, e.g. 0.5 */
  double rho_out;         /* weight offset: w = max(rho^A - rho_out, 0) */
  double tangent[2];      /* unit direction of the sliding velocity */
  double wall_point[2];   /* a point of the wall line (lattice units) */
  double wall_angle_deg;  /* direction of the wall line, degrees from +x */
  double exclude;         /* contour points closer than this to the wall are dropped */
  double box[4];          /* x0, x1, y0, y1: points outside are dropped; x1 < x0: no box */
  int32_t bridge_x;       /* column of the bridge radius; -1: not measured */
  int32_t bridge_y0;      /* first fluid node above the surface on that column */
} lbm_diag_params;

typedef struct {
  double weight;           /* sum of w */
  double com[2];           /* centre of mass of w (NaN if the weight is 0) */
  double com_velocity[2];  /* w-weighted mean of u */
  double sliding_velocity; /* com_velocity . tangent */
  double max_u;            /* max |u| over fluid nodes */
  int64_t contour_points;  /* crossings kept for the fit */
  double circle[3];        /* xc, yc, R of the fit (NaN with fewer than 3 points) */
  double contact_angle_deg;/* through the A phase (NaN without a circle) */
  double bridge_radius;    /* 0 if not measured */
  int64_t nonfinite_nodes; /* fluid nodes whose rho^A, rho^B or u is NaN or infinite (a run
                              that has diverged); they are left out of every other quantity and
                              max_u is NaN when there are any */
} lbm_diag;

/* Fill *h_out (host) for the current state. Uses the workspace's staging
 * area (as lbm_moments does) and synchronises. LBM_ERR_ARG for a null
 * pointer, level outside (0, 2), a non-finite parameter or a bridge column
 * or row outside the grid; LBM_ERR_STATE before geometry and fields. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, const lbm_diag_params* params, lbm_diag* h_out);

/* Number of interface-solid nodes of the installed geometry. */
lbm_status lbm_interface_count(lbm_ctx* ctx, int64_t* n);

/* Wait for the context's stream; returns LBM_ERR_CUDA on a pending fault. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* End-to-end run on host buffers: copies the mask and initial densities
 * from host memory into the workspace, installs geometry and wetting,
 * initialises, runs nsteps, and copies densities and velocity back (double
 * [ny][nx] each; output pointers may be NULL). Uses the context's stream
 * and workspace only (plus the staging area inside the workspace).
 * Synchronises. */
lbm_status lbm_run_host(lbm_ctx* ctx, const lbm_wetting_params* w, const uint8_t* h_mask,
                        const double* h_rhoA, const double* h_rhoB, int32_t nsteps,
                        double* h_rhoA_out, double* h_rhoB_out, double* h_ux_out,
                        double* h_uy_out);

/* lbm_run_host with FP32 host arrays: initial densities in, densities and
 * velocity out (float [ny][nx] each; outputs may be NULL). The inputs are
 * widened to FP64 on the device and the moments rounded to FP32 there, so
 * the host transfers carry half the bytes (9 + 16 bytes per node against
 * 17 + 32). Same staging, stream and synchronisation as lbm_run_host; the
 * paper has no counterpart. */
lbm_status lbm_run_host_f32(lbm_ctx* ctx, const lbm_wetting_params* w, const uint8_t* h_mask,
                            const float* h_rhoA, const float* h_rhoB, int32_t nsteps,
                            float* h_rhoA_out, float* h_rhoB_out, float* h_ux_out,
                            float* h_uy_out);

/* Per-component mass of two density fields without any device allocation
 * and without a workspace. The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory at the point they need the
 * reduction, e.g. code running inside a memory-capped or pre-allocated pool,
 * or a host thread that must not call cudaMalloc because it would
 * synchronise the device under work it does not own.
 *
 * Computes d_out[0] = sum of d_rhoA, d_out[1] = sum of d_rhoB over the nodes
 * where d_mask is 0 (all nodes when d_mask is NULL), in FP64 and in a fixed
 * order (deterministic). d_rhoA, d_rhoB: double [ny][nx]; d_mask: uint8
 * [ny][nx] or NULL; d_out: 2 doubles; all device pointers owned by the
 * caller. Enqueued on cuda_stream (NULL = legacy default stream); does not
 * synchronise.
 *
 * Scratch: one partial sum per component and block of 4096 nodes, held in
 * a 256 KiB file-scope __device__ array that every GPU which loads the
 * library keeps until the process exits. Hence nx * ny may not exceed
 * 67,108,864 (8192 * 8192); larger sizes, null pointers and nx or ny < 1
 * return LBM_ERR_ARG. The array is shared by every call on a device and
 * keeps the last call's partials (each call overwrites all it reads, so
 * nothing needs clearing): calls that overlap on the GPU (different streams
 * without ordering) race and must be serialised by the caller.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. The address is remembered per CUDA context
 * (by the driver's context identifier), so a context created again after
 * cudaDeviceReset gets a fresh lookup. Returns LBM_ERR_CUDA if the lookup or
 * a launch fails, or if an earlier error is pending (cudaPeekAtLastError;
 * the pending error is left for the caller). */
lbm_status lbm_field_mass_noalloc(const double* d_rhoA, const double* d_rhoB,
                                  const uint8_t* d_mask, int32_t nx, int32_t ny,
                                  double* d_out, void* cuda_stream);

/* ---- Batched stepping ------------------------------------------------------
 * Many independent simulations (contexts with their own geometry, wetting
 * and size, all of the same storage type on one device) advance together:
 * each step is one launch per kernel class over all of them, and repeated
 * steps replay a CUDA graph (kernel nodes, one per launch; the batch is not
 * one persistent kernel). Two schedules: TWO_PASS (density, Eq. 8 and
 * collide launches over the members' fluid lists, any storage) and TILED
 * (the Eq. 8 launch and one tiled single-pass launch over all members'
 * 32 x 14 tiles; 4- and 8-byte storage, members created with
 * LBM_KERNEL_AUTO or LBM_KERNEL_TILED so that they keep tile lists). The batch keeps pointers to the contexts; they
 * must outlive it, keep their geometry and wetting, and may still be
 * queried individually (lbm_moments, lbm_mass, ...) between batch steps.
 * The batch snapshots which members use the improved scheme at creation. */
typedef struct lbm_batch lbm_batch;

/* Device workspace bytes of a batch over ctxs[0..n). Every member must have
 * geometry and fields (LBM_ERR_STATE otherwise); all members must share the
 * storage type and device (LBM_ERR_ARG). */
lbm_status lbm_batch_workspace_bytes(int32_t n, lbm_ctx* const* ctxs, size_t* bytes);

/* Create a batch on a caller-owned workspace (256-byte aligned) and stream.
 * Synchronises. */
lbm_status lbm_batch_create(int32_t n, lbm_ctx* const* ctxs, void* d_workspace, size_t bytes,
                            void* cuda_stream, lbm_batch** out);

/* Replay steps in CUDA graphs of `steps` steps (even; 0 = launch each step
 * directly). The graph is built with kernel nodes, not stream capture. */
lbm_status lbm_batch_set_graph_steps(lbm_batch* b, int32_t steps);

/* Advance every member by nsteps steps. Uploads the members' descriptors
 * (synchronising on that small copy), then enqueues the work. */
lbm_status lbm_batch_step(lbm_batch* b, int32_t nsteps);

/* Time the candidate configurations (the two-pass schedule at 128 or 256
 * threads per block, and the tiled schedule when available; 2, 8 or 32
 * steps per graph replay) on the batch itself, keep the fastest, and write
 * {threads per block, steps} to h_choice (may be NULL; lbm_batch_config
 * tells the schedule). Advances every member by the steps it times (about
 * 9 x trial_steps plus warm-up). */
lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, int32_t* h_choice);

/* Select the schedule (LBM_KERNEL_TWO_PASS, the default, or
 * LBM_KERNEL_TILED); rebuilds the replay graph. LBM_ERR_ARG for another
 * value or TILED without 4-/8-byte storage and member tile lists. */
lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t kernel);

/* Current configuration: h_cfg[3] = {schedule (lbm_kernel), threads per
 * block, steps per graph replay (0: no graph)}. */
lbm_status lbm_batch_config(const lbm_batch* b, int32_t* h_cfg);

/* Kernels launched by the batch so far (graph replays count their nodes). */
int64_t lbm_batch_launch_count(const lbm_batch* b);

/* Text of the last error recorded in the batch ("" if none). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Release the batch (not its workspace or members). */
lbm_status lbm_batch_destroy(lbm_batch* b);

/* Release the host context (not the caller's workspace). */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Static description of a status code. */
const char* lbm_status_str(lbm_status s);

/* Text of the last error recorded in ctx ("" if none). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Number of kernels this context has launched since creation. */
int64_t lbm_launch_count(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
