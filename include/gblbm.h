/*
 * gblbm.h -- C ABI of the GB300 (sm_103a) D2Q9 lattice Boltzmann solver for
 * unconfined flow past a cylinder (Sahiti, Gurugubelli, Surasani, "Lattice
 * Boltzmann methodology for unconfined flows", arXiv 2605.02185).
 *
 * One time step, as the paper defines it (Section 2.1), is: BGK collision
 * (Eq. 2) towards the equilibrium of Eq. 3 with the moments of Eq. 4;
 * streaming; then the boundary corrections of Section 2.3 -- top/bottom
 * free-slip (Eq. 7), periodic (Eq. 8) or Zou-He velocity (Eqs. 9-10), the
 * Zou-He uniform inlet (Section 3.1) and the zero-gradient outlet (Eq. 13) --
 * with half-way bounce-back on the staircased cylinder (Section 2.4,
 * Section 3.1).  Every step also forms the momentum-exchange force on the
 * cylinder (Eq. 14) and thereby the drag and lift coefficients (Eq. 15).
 *
 * The library keeps the post-collision populations f* resident on the GPU and
 * runs each step as ONE fused kernel: pull-stream from the previous f*, the
 * boundary rules, the collision, the store of the new f*, and the force
 * partial sums of the cylinder links, reduced in a fixed order into a double
 * precision history on the device.
 *
 * Conventions for every function below:
 *   - Return value 0 (LBM_OK) or a negative LBM_ERR_* code; nothing throws.
 *   - Host pointers are read or written synchronously before return; the
 *     caller keeps ownership.  Device pointers are named as such.
 *   - Lattice arrays on the host are row-major [ny][nx] (index y*nx + x),
 *     y = 0 the bottom row, x = 0 the inlet column.
 *   - Populations use the paper's direction order i = 1..9 (Table 1) as
 *     plane index k = i - 1.
 *   - All work of one context runs in order on one CUDA stream.
 */
#ifndef GBLBM_H
#define GBLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define LBM_OK 0
#define LBM_ERR_ARG (-1)      /* invalid argument or geometry */
#define LBM_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define LBM_ERR_UNSTABLE (-3) /* |u| > 0.3 or NaN seen on a fluid node */
#define LBM_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define LBM_ERR_OOM (-5)      /* device memory or workspace too small */
#define LBM_ERR_RANGE (-6)    /* requested history entries not available */
#define LBM_ERR_STATE (-7)    /* call out of order (e.g. step before init) */

/* ---- top/bottom boundary modes (Section 2.3) --------------------------- */
#define LBM_BC_FREESLIP 0 /* Eq. 7: specular same-node copy */
#define LBM_BC_PERIODIC 1 /* Eq. 8: wrap in y */
#define LBM_BC_ZOUHE 2    /* Eqs. 9-10: Zou-He velocity (U, 0) */
#define LBM_BC_MOVINGWALL 3 /* Eq. 11: constant-velocity bounce-back, walls at (U, 0) */

/* ---- population storage ------------------------------------------------
 * Populations are stored as offsets h_i = f_i - r_i from the free-stream
 * equilibrium r_i = f_eq_i(rho = 1, u = (U, 0)) of Eq. 3. */
#define LBM_F32 0      /* float offsets, float arithmetic */
#define LBM_F16_OFS 1  /* IEEE half holding 4096 x the offset (exact power-of-two scale that keeps
                          small offsets out of the binary16 subnormals), float arithmetic */
#define LBM_BF16_OFS 2 /* bfloat16 offsets, float arithmetic */
#define LBM_F64 3      /* double offsets, double arithmetic */
#define LBM_F16_SR 4   /* as LBM_F16_OFS, but each stored value rounded stochastically: up with the
                          probability of its distance from the grid point below (deterministic: the
                          random bits hash the value, its node and direction), so updates smaller
                          than the 16-bit step accumulate instead of being rounded away */
#define LBM_BF16_SR 5  /* as LBM_BF16_OFS, rounded stochastically the same way */

/* ---- collision model ---------------------------------------------------- */
#define LBM_COLLIDE_BGK 0 /* Eq. 2: single relaxation time tau */
#define LBM_COLLIDE_MRT 1 /* Eq. 6: M^-1 S M with S = diag[1, s_e, s_eps, 1, s_q, 1, s_q, 1/tau, 1/tau] */

/* ---- step kernel variants --------------------------------------------- */
#define LBM_KERNEL_AUTO 0   /* the tuned default for the storage type */
#define LBM_KERNEL_DIRECT 1 /* one thread per cell, loads straight from HBM */
#define LBM_KERNEL_TMA 2    /* persistent; bulk-async (TMA) row staging */
#define LBM_KERNEL_TMA_BULK 3 /* TMA row staging and TMA bulk stores of the new rows
                                 (single lattices; not for batches) */
#define LBM_KERNEL_TMA_WAVE 4 /* the TMA kernel run for up to 64 steps per launch
                                 (single lattices; not for batches): a cooperative
                                 launch in which a row tile of step s starts as
                                 soon as the tiles of its own and the two
                                 neighbouring rows have finished step s - 1
                                 (per-row completion counters, bounded waits),
                                 so steps are not separated by a launch, its
                                 pipeline fill and its tail.  Results are
                                 bit-identical to LBM_KERNEL_TMA.  Built for the
                                 shapes that lbm_kernel_shapes_for lists;
                                 half-way bounce-back only (interpolated
                                 bounce-back runs on the kernels named under
                                 lbm_opts.bounce).  No CUDA graph is captured
                                 for it.  An option, not the default: on the
                                 1.3M-32M-node lattices measured it is 7-27 %
                                 slower than LBM_KERNEL_TMA (its per-tile
                                 synchronisation costs more than the launch
                                 boundaries it removes). */

typedef struct lbm_ctx lbm_ctx;

/* Creation options.  Fill with lbm_opts_default() and override fields. */
typedef struct lbm_opts {
  int nx, ny;          /* lattice size, nodes; both >= 5 */
  double tau;          /* BGK relaxation time (Eq. 2), > 0.5 */
  double U;            /* inlet speed, lattice units, 0 <= U < 0.3 */
  int bc_top_bottom;   /* LBM_BC_* */
  int storage;         /* LBM_F32 etc. */
  double D_ref;        /* length in Eq. 15; <= 0: (rows holding solid) - 1 */
  double rho_in;       /* density in Eq. 15; <= 0: 1 */
  int64_t history_capacity; /* force-history ring entries; <= 0: 1 << 20 */
  int kernel;          /* LBM_KERNEL_* */
  int consumer_warps;  /* TMA kernel: compute warps per CTA (0: tuned) */
  int cells_per_thread;/* TMA kernel: cells per compute thread per row tile */
  int stages;          /* TMA kernel: pipeline depth (row tiles in flight) */
  int ctas_per_sm;     /* TMA kernel: resident CTAs per SM (0: tuned default) */
  int graph_steps;     /* steps per captured CUDA graph (even); 0: auto; < 0: none */
  void *stream;        /* cudaStream_t to run on; NULL: the context makes its own */
  void *workspace;     /* device memory >= lbm_workspace_bytes(); NULL: the library allocates */
  size_t workspace_bytes;
  int collision;       /* LBM_COLLIDE_BGK (Eq. 2) or LBM_COLLIDE_MRT (Eq. 6) */
  double s_e, s_eps, s_q; /* MRT rates of the e, epsilon and q moments (paper: 1.1 each);
                             the stress moments relax at 1/tau, rho and j are conserved */
  int bounce;          /* LBM_BOUNCE_HALFWAY or LBM_BOUNCE_INTERPOLATED */
  double body_xc, body_yc, body_r; /* LBM_BOUNCE_INTERPOLATED: the body's true surface, a circle
                                      (nodes at integer coordinates); the mask stays the solid set */
} lbm_opts;

/* ---- body bounce-back (Section 2.4) ---------------------------------------
 * HALFWAY: the staircase rule the paper uses, f_i(x, n+1) = f*_opp(i)(x, n).
 * INTERPOLATED: the link-wise alternative the paper names (Bouzidi, Firdaouss
 * and Lallemand, linear): a population leaving fluid node x along c_i meets
 * the circle a fraction q of the link from x and returns as
 *   q <  1/2:  2q f*_i(x) + (1 - 2q) f*_i(x - c_i),
 *   q >= 1/2:  f*_i(x)/(2q) + (1 - 1/(2q)) f*_opp(i)(x).
 * Its momentum exchange adds c_i (f*_i(x, n) + f_opp(i)(x, n+1)) per link, so
 * the force of step n is known only after step n+1: with INTERPOLATED the
 * history is empty after lbm_init_fields and holds F(0..k-1) after k steps
 * (HALFWAY: F(0..k)).  Single lattices only (not batches, not
 * lbm_step_noalloc).  With float storage it runs on the TMA kernel in the
 * float default shapes (12, 2, 4), (10, 2, 4) and (8, 2, 4); in every other
 * case on the direct step kernel (LBM_KERNEL_DIRECT whatever opts.kernel
 * asks), so that the 16-bit TMA kernels carry no code for it. */
#define LBM_BOUNCE_HALFWAY 0
#define LBM_BOUNCE_INTERPOLATED 1

/* Defaults: F32 storage, BGK, MRT rates 1.1, auto kernel with the tuned
 * shape and CTAs per SM of the lattice size (ctas_per_sm 0), free-slip,
 * capacity 1 << 20. */
int lbm_opts_default(lbm_opts *opts);

/* Bytes of device workspace lbm_create_ex needs for opts and this mask
 * (host, [ny][nx], 1 = solid).  Lets a caller hand in memory it allocated
 * (e.g. a torch tensor) instead of letting the library allocate. */
int lbm_workspace_bytes(const lbm_opts *opts, const uint8_t *mask, size_t *bytes);

/* Create a lattice.  mask: host [ny][nx], nonzero = solid node of the
 * staircased body (Section 2.4).  Solid nodes must lie in
 * 2 <= x <= nx-3, 2 <= y <= ny-3 (the inlet, outlet and wall rules assume
 * fluid there).  The populations start at rest (rho = 1, u = 0); call
 * lbm_init_fields before stepping. */
int lbm_create(int nx, int ny, double tau, double U, const uint8_t *mask, int bc_top_bottom,
               lbm_ctx **out);
int lbm_create_ex(const lbm_opts *opts, const uint8_t *mask, lbm_ctx **out);
void lbm_destroy(lbm_ctx *ctx);

/* Initial state: f(0) = f_eq(rho, u) of Eq. 3 on fluid nodes (host double
 * arrays [ny][nx]), then the first collision, so the device holds f*(0), and
 * history entry 0 = the Eq. 14 force of f*(0).  Resets the history. */
int lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *u, const double *v);

/* The same from DEVICE float arrays [ny][nx] (e.g. a network's prediction).
 * with_noneq != 0 makes f(0) = f_eq + f_neq with the first-order
 * Chapman-Enskog non-equilibrium part f_neq_i = -(tau w_i rho / c_s^2)
 * Q_i : grad u, Q_i = c_i c_i - c_s^2 I, central differences (one-sided next
 * to the lattice edge or the body), so the start carries the stresses of the
 * given velocity field; the device then holds its collision
 * f*(0) = f_eq + (1 - 1/tau) f_neq (the shear moments relax at 1/tau in BGK
 * and in the MRT of Eq. 6 alike). */
int lbm_init_fields_device(lbm_ctx *ctx, const float *rho, const float *u, const float *v, int with_noneq);

/* Advance n >= 0 steps (asynchronous on the context stream).  Step n maps
 * f*(n-1) to f*(n) and appends the force of f*(n) to the history. */
int lbm_step(lbm_ctx *ctx, int64_t n);

/* Wait for the context stream; report LBM_ERR_UNSTABLE / LBM_ERR_TIMEOUT if
 * a step flagged one since the last lbm_init_fields. */
int lbm_sync(lbm_ctx *ctx);

/* Number of force-history entries (= steps + 1 after init). */
int lbm_force_count(lbm_ctx *ctx, int64_t *count);

/* Drag and lift coefficients (Eq. 15, Cd = Fx / (rho_in U^2 D / 2)) of
 * history entries [first, first + n) into host arrays.  LBM_ERR_RANGE if an
 * entry is not yet written or already overwritten in the ring. */
int lbm_forces(lbm_ctx *ctx, int64_t first, int64_t n, double *cd, double *cl);

/* The same entries as raw lattice-unit forces (Eq. 14), host [n][2]. */
int lbm_forces_raw(lbm_ctx *ctx, int64_t first, int64_t n, double *fxy);

/* Reference length and density used by lbm_forces. */
int lbm_set_reference(lbm_ctx *ctx, double D_ref, double rho_in);

/* Moments (Eq. 4) of the current f*, which equal those of the post-boundary
 * f of the same step; solid nodes report rho = 1, u = v = 0.
 * dtype 0: float arrays, 1: double arrays; host [ny][nx] each. */
int lbm_fields(lbm_ctx *ctx, int dtype, void *rho, void *u, void *v);

/* The same into DEVICE float arrays [ny][nx] (asynchronous). */
int lbm_fields_device(lbm_ctx *ctx, float *rho, float *u, float *v);

/* Double-precision sum of rho over fluid nodes (mass-drift check). */
int lbm_mass(lbm_ctx *ctx, double *mass);

/* Checkpoint: the current f* as stored offsets f*_i - r_i, packed host
 * [9][ny][nx] of the storage type (4, 2, 2 or 8 bytes per value).
 * bytes must equal 9 * nx * ny * element size. */
int lbm_get_populations(lbm_ctx *ctx, void *dst, size_t bytes);
/* Restore a checkpoint written by lbm_get_populations.  history_count is
 * the lbm_force_count value at the time of the checkpoint; the next step
 * writes history entry history_count.  Earlier history entries are not
 * restored. */
int lbm_set_populations(lbm_ctx *ctx, const void *src, size_t bytes, int64_t history_count);

/* Self-describing checkpoint (no counterpart in the paper): an 88-byte header
 * (magic "GBLBMCK1", version, nx, ny, storage, collision, top/bottom rule,
 * bounce-back rule, tau, U, history count, stored history entries, payload
 * bytes, 64-bit checksum), then the populations as lbm_get_populations
 * writes them, then the force-history entries still in the ring (raw
 * (Fx, Fy) doubles, oldest first).  The checksum is FNV-1a taken over the
 * payload's little-endian 64-bit words.  All buffers are host memory owned
 * by the caller.
 *   lbm_checkpoint_bytes: the image size for the context's current state.
 *   lbm_checkpoint_save:  write the image; bytes must equal that size.
 *   lbm_checkpoint_load:  restore populations, step count and history.
 *     LBM_ERR_ARG, with the context unchanged, when the image is truncated
 *     or padded, its checksum does not match (corruption), or it describes
 *     another lattice (size, storage, collision, rules, tau or U). */
int lbm_checkpoint_bytes(lbm_ctx *ctx, size_t *bytes);
int lbm_checkpoint_save(lbm_ctx *ctx, void *dst, size_t bytes);
int lbm_checkpoint_load(lbm_ctx *ctx, const void *src, size_t bytes);

/* A rectangular window [x0, x0+w) x [y0, y0+h) of the current f* offsets,
 * packed host [9][h][w] of the storage type (probes, sampled checks). */
int lbm_get_window(lbm_ctx *ctx, int x0, int y0, int w, int h, void *dst);

/* Switch the step kernel (LBM_KERNEL_*) and its shape; re-captures graphs. */
int lbm_set_kernel(lbm_ctx *ctx, int kernel, int consumer_warps, int cells_per_thread, int stages,
                   int ctas_per_sm);
/* The kernel shape in use: kernel, consumer warps, cells/thread, stages,
 * CTAs per SM, grid size (CTAs) -- 6 ints. */
int lbm_get_kernel(lbm_ctx *ctx, int *out6);

/* Host only (no GPU call): the kernel, consumer warps, cells/thread, stages
 * and CTAs per SM (5 ints into out5) that lbm_create_ex picks for *opts
 * before it checks them against the device -- LBM_KERNEL_AUTO resolved, the
 * default shape of the lattice size where none is given, ctas_per_sm 0
 * resolved.  A shape given in opts that the kernel is not built for is
 * LBM_ERR_ARG, as are options lbm_create_ex would refuse.  (Interpolated
 * bounce-back on a storage type or shape without its TMA kernel runs on the
 * direct kernel; that choice is made on creation, not here.) */
int lbm_default_kernel(const lbm_opts *opts, int *out5);

/* The shapes the TMA kernel is built for: up to cap triples (compute warps,
 * cells per thread, stages) into out; *count receives how many exist. */
int lbm_kernel_shapes(int *out, int cap, int *count);

/* The same for LBM_KERNEL_TMA, LBM_KERNEL_TMA_BULK or LBM_KERNEL_TMA_WAVE. */
int lbm_kernel_shapes_for(int kernel, int *out, int cap, int *count);

/* Failure-path testing (no counterpart in the paper).  Every wait of the
 * step kernels on another warp or on an asynchronous copy is bounded; when
 * one gives up, the step stops its remaining work, waits (bounded again)
 * for its own copies in flight and returns, and lbm_sync reports
 * LBM_ERR_TIMEOUT -- the GPU is never trapped or hung.  This call makes that
 * path testable: the waits give up after wait_seconds (<= 0: the default
 * 1 s; at most 60), and if tile >= 0 the TMA producer announces the copies
 * of row tile `tile` (row * tiles per row + segment, as the kernel numbers
 * them) but never issues them, so the waits on that tile run out.  The
 * populations are then partly stale: restore a checkpoint or re-initialise.
 * The context must use LBM_KERNEL_TMA, LBM_KERNEL_TMA_BULK or
 * LBM_KERNEL_TMA_WAVE (LBM_ERR_ARG otherwise).  tile < 0 and wait_seconds <= 0 restore normal operation. */
int lbm_set_fault_injection(lbm_ctx *ctx, int64_t tile, double wait_seconds);

/* The CUDA stream the context launches on (cudaStream_t). */
int lbm_get_stream(lbm_ctx *ctx, void **stream);

/* Step-kernel launches issued since creation (counts each kernel once; a
 * launch of LBM_KERNEL_TMA_WAVE counts 2, with its force reduction). */
int lbm_launch_count(lbm_ctx *ctx, int64_t *count);

/* Algorithmic bytes one step moves through HBM: 2 * 9 * element size per
 * node (read f*(n-1), write f*(n)). */
int lbm_bytes_per_step(lbm_ctx *ctx, double *bytes);

/* One step WITHOUT ANY ALLOCATION, for callers that may not allocate device
 * memory (their memory comes from a pool or arena they manage, or another
 * runtime owns the allocator).  The paper has no counterpart: this is a
 * service of the library.
 *
 * Reads f*(n) from f_in and writes f*(n+1) to f_out, both DEVICE buffers
 * owned by the caller, packed [9][ny][nx] in the context's storage type as
 * offsets from the free-stream equilibrium (the layout of
 * lbm_get_populations), and writes the Eq. 14 force (Fx, Fy) of f*(n+1) to
 * force_out, a DEVICE array of 2 doubles.  Geometry and parameters come from
 * ctx; the context's own populations and history are neither read nor
 * changed.  Runs the direct step kernel, asynchronously on the context
 * stream.  f_in and f_out must not overlap.
 *
 * Scratch (force partials and reduction counters) lives in a 1 MiB device
 * array inside the library, held by every GPU that loads the library until
 * the process exits.  Bodies whose link-owning nodes span more than 65,520
 * row tiles of 256 nodes are rejected with LBM_ERR_ARG.  lbm_create and
 * lbm_create_ex look up the array's address on their device
 * (cudaGetSymbolAddress, which may load the module holding it), so that
 * lookup is done before this entry point is first called on a context of
 * that device.  Every call clears and reuses the
 * same array: calls whose kernels overlap on the GPU (different streams, or
 * several contexts) race on it.  The |u| > 0.3 stability check is not
 * reported by this entry point.  No cudaMalloc, cudaFree or other
 * allocating call is made. */
int lbm_step_noalloc(lbm_ctx *ctx, const void *f_in, void *f_out, double *force_out);

/* ---- batches of independent lattices --------------------------------------
 * Many cylinder cases of different size and Reynolds number advanced by ONE
 * step-kernel launch per step (the cases' row tiles are concatenated), with
 * multi-step CUDA graphs.  Each case is a full lattice context; per-case
 * reads (lbm_forces, lbm_fields, lbm_mass, lbm_get_populations, ...) use the
 * context returned by lbm_batch_case.  Do not call lbm_step, lbm_init_fields,
 * lbm_set_kernel or lbm_destroy on a case context: use the lbm_batch_*
 * functions, which keep all cases on one step parity. */
typedef struct lbm_batch lbm_batch;

typedef struct lbm_case {
  int nx, ny;          /* lattice size of this case */
  double tau, U;       /* relaxation time (Eq. 2) and inlet speed */
  int bc_top_bottom;   /* LBM_BC_* */
  const uint8_t *mask; /* host [ny][nx], 1 = solid (same rules as lbm_create), or NULL */
  double D_ref;        /* Eq. 15 length; <= 0: (rows holding solid) - 1 */
  double rho_in;       /* Eq. 15 density; <= 0: 1 */
} lbm_case;

/* Workspace bytes for these cases; common supplies storage, history
 * capacity, kernel shape, graph steps (its nx, ny, tau, U, bc are ignored). */
int lbm_batch_workspace_bytes(int ncases, const lbm_case *cases, const lbm_opts *common, size_t *bytes);
/* Create the batch; common->stream / common->workspace as for lbm_create_ex. */
int lbm_batch_create(int ncases, const lbm_case *cases, const lbm_opts *common, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *batch);
/* The lattice context of case c (owned by the batch). */
int lbm_batch_case(lbm_batch *batch, int c, lbm_ctx **ctx);
/* Initial fields of case c (host double arrays, as lbm_init_fields). */
int lbm_batch_init_fields(lbm_batch *batch, int c, const double *rho, const double *u, const double *v);
/* Advance every case n steps (asynchronous); all cases must be initialised. */
int lbm_batch_step(lbm_batch *batch, int64_t n);
/* Wait; the worst error any case reported (LBM_ERR_TIMEOUT first). */
int lbm_batch_sync(lbm_batch *batch);
/* Kernel shape for the whole batch (as lbm_set_kernel); re-captures graphs. */
int lbm_batch_set_kernel(lbm_batch *batch, int kernel, int consumer_warps, int cells_per_thread, int stages,
                         int ctas_per_sm);
int lbm_batch_get_kernel(lbm_batch *batch, int *out6);
int lbm_batch_get_stream(lbm_batch *batch, void **stream);
int lbm_batch_launch_count(lbm_batch *batch, int64_t *count);
/* Total nodes of all cases, and the algorithmic HBM bytes of one batch step. */
int lbm_batch_nodes(lbm_batch *batch, int64_t *nodes, double *bytes_per_step);

/* Diagnostic (no counterpart in the paper): -1/x as the float collisions
 * compute it (the hardware reciprocal estimate refined by one
 * Newton-Raphson step, see Eq. 4's 1/rho), for x DEVICE float [n], into
 * DEVICE y_single (one node per lane) and y_pair (packed pairs of nodes),
 * asynchronously on `stream` (cudaStream_t).  Lets a test bound its error
 * against the correctly rounded quotient. */
int lbm_probe_neg_recip(const float *x, float *y_single, float *y_pair, int64_t n, void *stream);

/* Diagnostic (no counterpart in the paper): the store rounding of
 * LBM_F16_SR / LBM_BF16_SR on its own.  x: DEVICE float [n] offsets, salt:
 * DEVICE uint32 [n] (in the kernels, a hash of node and direction), out:
 * DEVICE uint16 [n] receiving the stored bit patterns (binary16 of 4096 x the
 * offset, or bfloat16 of the offset), asynchronously on `stream`. */
int lbm_probe_stochastic_round(int storage, const float *x, const uint32_t *salt, uint16_t *out, int64_t n,
                               void *stream);

const char *lbm_error_string(int code);
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBLBM_H */
