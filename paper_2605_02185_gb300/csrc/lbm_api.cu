// lbm_api.cu -- the C ABI declared in include/gblbm.h: context, device
// memory layout, geometry preprocessing, CUDA-graph stepping, read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gblbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_ctx.h"
#include "lbm_host.h"

using namespace gblbm;



namespace {

constexpr int kLayoutParts = 10;

size_t layout(const lbm_opts *o, const Geometry &g, int *pitch_out, size_t offs[kLayoutParts], int *slot_cap_out,
              int *band_rows_out) {
  const int elem = elem_size(o->storage);
  const int pitch = (int)align_up((size_t)o->nx, 64);
  const size_t pop = align_up((size_t)9 * o->ny * pitch * elem, kAlign);
  const size_t lmap = align_up(std::max<size_t>(g.lmap.size(), 1) * sizeof(uint16_t), kAlign) +
                      align_up(g.qmap.size() * sizeof(float), kAlign);  // link fractions follow the map
  int slot_cap = 1;
  if (g.fx1 >= g.fx0) slot_cap = (g.fy1 - g.fy0 + 1) * (g.fx1 / 256 - g.fx0 / 256 + 1);
  const size_t slots = align_up((size_t)slot_cap * sizeof(double2), kAlign);
  const long long cap = o->history_capacity > 0 ? o->history_capacity : (1ll << 20);
  const size_t hist = align_up((size_t)cap * 2 * sizeof(double), kAlign);
  const size_t ctrl = kAlign;
  const size_t wave_slots = align_up((size_t)kWaveSteps * slot_cap * sizeof(double2), kAlign);
  const size_t wave_rows = align_up((size_t)o->ny * sizeof(unsigned), kAlign);
  const int band_rows = (int)std::max<size_t>(1, std::min<size_t>((size_t)o->ny, kBandCells / (size_t)o->nx));
  const size_t staging =
      align_up(std::max<size_t>((size_t)band_rows * o->nx * 3 * sizeof(double), (size_t)o->ny * sizeof(double)), kAlign);
  size_t off = 0;
  offs[0] = off; off += pop;      // A
  offs[1] = off; off += pop;      // B
  offs[2] = off; off += lmap;
  offs[3] = off; off += slots;
  offs[4] = off; off += hist;
  offs[5] = off; off += ctrl;
  offs[6] = off; off += staging;
  offs[7] = off; off += wave_slots;
  offs[8] = off; off += wave_rows;
  offs[9] = off;
  *pitch_out = pitch;
  *slot_cap_out = slot_cap;
  *band_rows_out = band_rows;
  return off;
}

// Index of (ncw, cpt, stages) in the shape list of `kernel`, or -1.
int find_shape(int kernel, int ncw, int cpt, int stages) {
  const TmaShape *list = kernel == LBM_KERNEL_TMA_BULK ? kTmaBulkShapes : kTmaShapes;
  const int n = kernel == LBM_KERNEL_TMA_BULK ? kNumTmaBulkShapes : kNumTmaShapes;
  for (int s = 0; s < n; ++s)
    if (list[s].ncw == ncw && list[s].cpt == cpt && list[s].stages == stages) return s;
  return -1;
}

// The kernel, shape and CTAs per SM a context asks for: AUTO takes the
// storage type's default kernel; an explicit shape (ncw, cpt, stages) is
// looked up in the kernel's list (-1 if absent), else the default shape of
// the lattice size; ctas_per_sm <= 0 takes the default of that shape for
// the TMA kernels and 1 for the others.  Returns the kernel or -1.
int choose_kernel(int storage, int nx, int ny, bool interp, int kernel, int ncw, int cpt, int stages, int ctas_per_sm,
                  int *shape, int *ctas) {
  if (kernel == LBM_KERNEL_AUTO) kernel = default_kernel(storage);
  const DefaultShape d = default_shape(storage, (long long)nx * ny, interp || kernel == LBM_KERNEL_TMA_WAVE);
  *ctas = ctas_per_sm > 0 ? ctas_per_sm : 1;
  if (kernel != LBM_KERNEL_DIRECT && (ncw || cpt || stages)) {
    *shape = find_shape(kernel, ncw, cpt, stages);
    if (*shape < 0) return -1;
  } else if (kernel == LBM_KERNEL_TMA_BULK) {
    *shape = 0;
  } else {
    *shape = d.shape;
    if (ctas_per_sm <= 0 && kernel != LBM_KERNEL_DIRECT) *ctas = d.ctas;
  }
  return kernel;
}

// Fill the step parameters for the chosen kernel shape (tile width, force
// slots) and capture the multi-step graph.
int configure_kernel(lbm_ctx *c, int kernel, int shape, int ctas_per_sm) {
  if (kernel == LBM_KERNEL_AUTO) kernel = LBM_KERNEL_TMA;
  // interpolated bounce-back: the TMA kernel where it is built for this
  // storage type and shape, else the direct kernel
  if (c->qmap && (kernel != LBM_KERNEL_TMA ||
                  c->ops->tma_interp(shape, 0, nullptr, nullptr, c->p, nullptr, 1) != cudaSuccess))
    kernel = LBM_KERNEL_DIRECT;
  int seg;
  if (kernel == LBM_KERNEL_DIRECT) {
    seg = kDirectThreads;
  } else if (kernel == LBM_KERNEL_TMA_BULK) {
    if (shape < 0 || shape >= kNumTmaBulkShapes) return LBM_ERR_ARG;
    if (c->ops->bulk_smem(shape) > 227 * 1024) return LBM_ERR_ARG;
    CK(c->ops->bulk_prep(shape));
    const int occ = c->ops->bulk_occupancy(shape);
    if (occ <= 0) return LBM_ERR_ARG;
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, occ));
    seg = kTmaBulkShapes[shape].ncw * 32 * kTmaBulkShapes[shape].cpt;
  } else if (kernel == LBM_KERNEL_TMA_WAVE) {
    if (shape < 0 || shape >= kNumTmaShapes) return LBM_ERR_ARG;
    if (c->ops->smem(shape) > 227 * 1024) return LBM_ERR_ARG;
    const cudaError_t e = c->ops->wave_prep(shape);
    if (e == cudaErrorNotSupported) return LBM_ERR_ARG;
    CK(e);
    const int occ = c->ops->wave_occupancy(shape);
    if (occ <= 0) return LBM_ERR_ARG;
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, occ));
    seg = c->ops->tma_pair * kTmaShapes[shape].ncw * 32 * kTmaShapes[shape].cpt;
  } else {
    if (shape < 0 || shape >= kNumTmaShapes) return LBM_ERR_ARG;
    if (c->ops->smem(shape) > 227 * 1024) return LBM_ERR_ARG;
    CK(c->ops->prep(shape));
    const int occ = c->ops->occupancy(shape);
    if (occ <= 0) return LBM_ERR_ARG;
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, occ));
    seg = c->ops->tma_pair * kTmaShapes[shape].ncw * 32 * kTmaShapes[shape].cpt;
  }
  const int nseg = (c->nx + seg - 1) / seg;
  StepParams &p = c->p;
  p.seg = seg;
  p.nseg = nseg;
  const Geometry &g = c->geo;
  if (g.fx1 >= g.fx0) {
    p.fy0 = g.fy0;
    p.fy1 = g.fy1;
    p.fs0 = g.fx0 / seg;
    p.fs1 = g.fx1 / seg;
  } else {
    p.fy0 = p.fy1 = 0;
    p.fs0 = p.fs1 = 0;
  }
  p.nslots = (p.fy1 - p.fy0 + 1) * (p.fs1 - p.fs0 + 1);
  if (p.nslots > c->slot_cap) return LBM_ERR_ARG;
  const long long nitems = (long long)c->ny * nseg;
  if (nitems > (1ll << 31) - 1) return LBM_ERR_ARG;
  const int grid = kernel == LBM_KERNEL_DIRECT ? (int)nitems
                                               : (int)std::min<long long>(nitems, (long long)c->sms * ctas_per_sm);
  if (kernel == LBM_KERNEL_TMA_WAVE) {
    // a new tiling starts from cleared row counters
    CK(cudaMemsetAsync(c->wave_rows, 0, (size_t)c->ny * sizeof(unsigned), c->stream));
    c->wave_base = 0;
  }
  c->kernel = kernel;
  c->shape = shape;
  c->ctas_per_sm = ctas_per_sm;
  c->seg = seg;
  c->nseg = nseg;
  c->grid = grid;
  return LBM_OK;
}

cudaError_t launch_step(lbm_ctx *c, int from) {
  const void *A = c->buf[from];
  void *B = c->buf[from ^ 1];
  if (c->kernel == LBM_KERNEL_DIRECT) return c->ops->direct(A, B, c->p, c->stream);
  if (c->kernel == LBM_KERNEL_TMA_BULK) return c->ops->tma_bulk(c->shape, c->grid, A, B, c->p, c->stream);
  if (c->qmap) return c->ops->tma_interp(c->shape, c->grid, A, B, c->p, c->stream, 0);
  return c->ops->tma(c->shape, c->grid, A, B, c->p, c->stream);
}

// Clear the multi-step kernel's row counters (a new state, or the recovery
// from a launch that gave up and left them uneven).
cudaError_t reset_wave_rows(lbm_ctx *c) {
  c->wave_base = 0;
  return cudaMemsetAsync(c->wave_rows, 0, (size_t)c->ny * sizeof(unsigned), c->stream);
}

// Steps [0, n) on the multi-step kernel, kWaveSteps per launch.
int wave_steps(lbm_ctx *c, int64_t n) {
  while (n > 0) {
    const int k = (int)std::min<int64_t>(n, kWaveSteps);
    if ((unsigned long long)(c->wave_base + k) * (unsigned)c->nseg > (1ull << 30)) {
      // keep the counters and their differences far from 2^31
      CK(cudaMemsetAsync(c->wave_rows, 0, (size_t)c->ny * sizeof(unsigned), c->stream));
      c->wave_base = 0;
    }
    WaveParams w;
    w.rows_done = c->wave_rows;
    w.base = c->wave_base;
    w.steps = k;
    w.slots = c->wave_slots;
    CK(c->ops->wave(c->shape, c->grid, c->buf[c->cur], c->buf[c->cur ^ 1], c->p, w, c->stream));
    c->wave_base += (unsigned)k;
    c->cur ^= k & 1;
    c->launches += 2;
    n -= k;
  }
  return LBM_OK;
}

int capture_graph(lbm_ctx *c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  int gs = c->o.graph_steps;
  if (gs < 0 || c->kernel == LBM_KERNEL_TMA_WAVE) {  // the multi-step kernel needs no graph
    c->graph_steps = 0;
    return LBM_OK;
  }
  if (gs == 0) {
    const long long cells = (long long)c->nx * c->ny;
    gs = (int)std::max<long long>(2, std::min<long long>(256, (16ll << 20) / std::max<long long>(cells, 1)));
  }
  gs += gs & 1;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < gs && err == cudaSuccess; ++s) err = launch_step(c, s & 1);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(err != cudaSuccess ? err : e2);
  }
  err = cudaGraphInstantiate(&c->graph, graph, 0);
  cudaGraphDestroy(graph);
  CK(err);
  CK(cudaGraphUpload(c->graph, c->stream));
  c->graph_steps = gs;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_opts_default(lbm_opts *o) {
  if (!o) return LBM_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->tau = 1.0;
  o->bc_top_bottom = LBM_BC_FREESLIP;
  o->storage = LBM_F32;
  o->history_capacity = 1ll << 20;
  o->kernel = LBM_KERNEL_AUTO;
  o->ctas_per_sm = 0;  // the tuned default of the chosen shape
  o->collision = LBM_COLLIDE_BGK;
  o->s_e = o->s_eps = o->s_q = 1.1;
  return LBM_OK;
}

int lbm_workspace_bytes(const lbm_opts *o, const uint8_t *mask, size_t *bytes) {
  int rc = check_opts(o);
  if (rc) return rc;
  if (!bytes) return LBM_ERR_ARG;
  Geometry g;
  rc = build_geometry(o, mask, &g);
  if (rc) return rc;
  int pitch, slot_cap, band_rows;
  size_t offs[kLayoutParts];
  *bytes = layout(o, g, &pitch, offs, &slot_cap, &band_rows);
  return LBM_OK;
}

int lbm_create_ex(const lbm_opts *o, const uint8_t *mask, lbm_ctx **out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  int rc = check_opts(o);
  if (rc) return rc;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->o = *o;
  rc = build_geometry(o, mask, &c->geo);
  if (rc) {
    delete c;
    return rc;
  }
  c->nx = o->nx;
  c->ny = o->ny;
  c->elem = elem_size(o->storage);
  c->ops = ops_for(o->storage);
  size_t offs[kLayoutParts];
  c->ws_bytes = layout(o, c->geo, &c->pitch, offs, &c->slot_cap, &c->band_rows);
  c->plane = (long long)c->ny * c->pitch;
  c->hist_cap = o->history_capacity > 0 ? o->history_capacity : (1ll << 20);
  auto fail = [&](int code) {
    lbm_destroy(c);
    return code;
  };
  if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(LBM_ERR_CUDA);
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) return fail(LBM_ERR_CUDA);
  rc = noalloc_prepare(c->dev);
  if (rc) return fail(rc);
  if (o->workspace) {
    if (o->workspace_bytes < c->ws_bytes || ((uintptr_t)o->workspace % kAlign) != 0) return fail(LBM_ERR_OOM);
    c->ws = o->workspace;
  } else {
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (c->ws_bytes > freeb) return fail(LBM_ERR_OOM);
    if (cudaMalloc(&c->ws, c->ws_bytes) != cudaSuccess) return fail(LBM_ERR_OOM);
    c->own_ws = true;
  }
  char *base = (char *)c->ws;
  c->buf[0] = base + offs[0];
  c->buf[1] = base + offs[1];
  c->lmap = (uint16_t *)(base + offs[2]);
  c->qmap = c->geo.qmap.empty()
                ? nullptr
                : (float *)(base + offs[2] + align_up(std::max<size_t>(c->geo.lmap.size(), 1) * sizeof(uint16_t), kAlign));
  c->slots = (double2 *)(base + offs[3]);
  c->hist = (double *)(base + offs[4]);
  c->ctrl = (unsigned *)(base + offs[5]);
  c->staging = base + offs[6];
  c->staging_bytes = offs[7] - offs[6];
  c->wave_slots = (double2 *)(base + offs[7]);
  c->wave_rows = (unsigned *)(base + offs[8]);
  if (o->stream) {
    c->stream = (cudaStream_t)o->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LBM_ERR_CUDA);
    c->own_stream = true;
  }
  if (cudaMemsetAsync(c->ws, 0, c->ws_bytes, c->stream) != cudaSuccess) return fail(LBM_ERR_CUDA);
  if (!c->geo.lmap.empty() &&
      cudaMemcpyAsync(c->lmap, c->geo.lmap.data(), c->geo.lmap.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess)
    return fail(LBM_ERR_CUDA);
  if (c->qmap && cudaMemcpyAsync(c->qmap, c->geo.qmap.data(), c->geo.qmap.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return fail(LBM_ERR_CUDA);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(LBM_ERR_CUDA);
  c->D_ref = o->D_ref > 0 ? o->D_ref : (c->geo.solid_rows > 1 ? c->geo.solid_rows - 1 : 1);
  c->rho_in = o->rho_in > 0 ? o->rho_in : 1.0;

  StepParams &p = c->p;
  p.nx = c->nx;
  p.ny = c->ny;
  p.pitch = c->pitch;
  p.bc = o->bc_top_bottom;
  p.plane = c->plane;
  p.omega = 1.0 / o->tau;
  p.U = o->U;
  p.lmap = c->lmap;
  p.qmap = c->qmap;
  p.lx0 = c->geo.lx0;
  p.ly0 = c->geo.ly0;
  p.lw = c->geo.lw;
  p.lh = c->geo.lh;
  p.slots = c->slots;
  p.done = c->ctrl;
  p.err = c->ctrl + 1;
  p.step = (unsigned long long *)(c->ctrl + 2);
  p.hist = c->hist;
  p.hist_cap = c->hist_cap;
  p.fconst_x = c->geo.fconst_x;
  p.fconst_y = c->geo.fconst_y;
  p.mrt = o->collision == LBM_COLLIDE_MRT ? 1 : 0;
  p.s_e = o->s_e;
  p.s_eps = o->s_eps;
  p.s_q = o->s_q;
  fill_coefs(p);
  p.wait_ns = 1000000000ull;  // every bounded device wait gives up after 1 s
  p.fault_tile = -1;

  int shape = -1, ctas = 1;
  const int kernel = choose_kernel(o->storage, o->nx, o->ny, !c->geo.qmap.empty(), o->kernel, o->consumer_warps,
                                   o->cells_per_thread, o->stages, o->ctas_per_sm, &shape, &ctas);
  if (kernel < 0) return fail(LBM_ERR_ARG);
  rc = configure_kernel(c, kernel, std::max(shape, 0), ctas);
  if (rc) return fail(rc);
  rc = capture_graph(c);
  if (rc) return fail(rc);
  *out = c;
  return LBM_OK;
}

int lbm_create(int nx, int ny, double tau, double U, const uint8_t *mask, int bc, lbm_ctx **out) {
  lbm_opts o;
  lbm_opts_default(&o);
  o.nx = nx;
  o.ny = ny;
  o.tau = tau;
  o.U = U;
  o.bc_top_bottom = bc;
  return lbm_create_ex(&o, mask, out);
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int lbm_init_fields(lbm_ctx *c, const double *rho, const double *u, const double *v) {
  if (!c || !rho || !u || !v) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  double *sr = (double *)c->staging;
  const size_t band = (size_t)c->band_rows * c->nx;
  double *su = sr + band, *sv = su + band;
  c->cur = 0;
  for (int y0 = 0; y0 < c->ny; y0 += c->band_rows) {
    const int rows = std::min(c->band_rows, c->ny - y0);
    const size_t n = (size_t)rows * c->nx, off = (size_t)y0 * c->nx;
    CK(cudaMemcpyAsync(sr, rho + off, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(su, u + off, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(sv, v + off, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c->ops->init(c->buf[0], c->p, sr, su, sv, y0, rows, c->stream));
  }
  CK(cudaMemsetAsync(c->ctrl, 0, kAlign, c->stream));
  CK(reset_wave_rows(c));
  CK(cudaMemsetAsync(c->buf[1], 0, (size_t)9 * c->plane * c->elem, c->stream));
  if (!c->qmap) CK(c->ops->force(c->buf[0], c->p, c->stream));  // interpolated: F(0) comes with step 1
  CK(cudaStreamSynchronize(c->stream));
  c->inited = true;
  return LBM_OK;
}

int lbm_init_fields_device(lbm_ctx *c, const float *rho, const float *u, const float *v, int with_noneq) {
  if (!c || !rho || !u || !v) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  c->cur = 0;
  CK(c->ops->init_device(c->buf[0], c->p, rho, u, v, with_noneq ? 1 : 0, 1.0 / c->p.omega, c->stream));
  CK(cudaMemsetAsync(c->ctrl, 0, kAlign, c->stream));
  CK(reset_wave_rows(c));
  CK(cudaMemsetAsync(c->buf[1], 0, (size_t)9 * c->plane * c->elem, c->stream));
  if (!c->qmap) CK(c->ops->force(c->buf[0], c->p, c->stream));  // interpolated: F(0) comes with step 1
  CK(cudaStreamSynchronize(c->stream));
  c->inited = true;
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int64_t n) {
  if (!c || n < 0) return LBM_ERR_ARG;
  if (!c->inited) return LBM_ERR_STATE;
  CK(cudaSetDevice(c->dev));
  if (c->kernel == LBM_KERNEL_TMA_WAVE) return wave_steps(c, n);
  while (n > 0) {
    if (c->graph && c->cur == 0 && n >= c->graph_steps) {
      CK(cudaGraphLaunch(c->graph, c->stream));
      n -= c->graph_steps;
      c->launches += c->graph_steps;
    } else {
      CK(launch_step(c, c->cur));
      c->cur ^= 1;
      --n;
      ++c->launches;
    }
  }
  return LBM_OK;
}

int lbm_sync(lbm_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  unsigned err = 0;
  CK(cudaMemcpy(&err, c->ctrl + 1, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (err & ERR_TIMEOUT) return LBM_ERR_TIMEOUT;
  if (err & ERR_UNSTABLE) return LBM_ERR_UNSTABLE;
  return LBM_OK;
}

int lbm_force_count(lbm_ctx *c, int64_t *count) {
  if (!c || !count) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long s = 0;
  CK(cudaMemcpy(&s, c->ctrl + 2, sizeof(s), cudaMemcpyDeviceToHost));
  *count = (int64_t)s;
  return LBM_OK;
}

int lbm_forces_raw(lbm_ctx *c, int64_t first, int64_t n, double *fxy) {
  if (!c || first < 0 || n < 0 || (n > 0 && !fxy)) return LBM_ERR_ARG;
  int64_t count = 0;
  int rc = lbm_force_count(c, &count);
  if (rc) return rc;
  if (first + n > count || first < count - c->hist_cap) return LBM_ERR_RANGE;
  int64_t done = 0;
  while (done < n) {
    const int64_t e = first + done;
    const int64_t r = e % c->hist_cap;
    const int64_t run = std::min<int64_t>(n - done, c->hist_cap - r);
    CK(cudaMemcpy(fxy + 2 * done, c->hist + 2 * r, (size_t)run * 2 * sizeof(double), cudaMemcpyDeviceToHost));
    done += run;
  }
  return LBM_OK;
}

int lbm_forces(lbm_ctx *c, int64_t first, int64_t n, double *cd, double *cl) {
  if (!c || n < 0 || (n > 0 && (!cd || !cl))) return LBM_ERR_ARG;
  std::vector<double> raw((size_t)std::max<int64_t>(n, 1) * 2);
  int rc = lbm_forces_raw(c, first, n, raw.data());
  if (rc) return rc;
  const double q = 0.5 * c->rho_in * c->o.U * c->o.U * c->D_ref;  // Eq. 15 denominator
  for (int64_t i = 0; i < n; ++i) {
    cd[i] = raw[2 * i] / q;
    cl[i] = raw[2 * i + 1] / q;
  }
  return LBM_OK;
}

int lbm_set_reference(lbm_ctx *c, double D_ref, double rho_in) {
  if (!c || !(D_ref > 0) || !(rho_in > 0)) return LBM_ERR_ARG;
  c->D_ref = D_ref;
  c->rho_in = rho_in;
  return LBM_OK;
}

int lbm_fields(lbm_ctx *c, int dtype, void *rho, void *u, void *v) {
  if (!c || !rho || !u || !v || (dtype != 0 && dtype != 1)) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  const size_t es = dtype ? sizeof(double) : sizeof(float);
  const size_t band = (size_t)c->band_rows * c->nx;
  char *sr = (char *)c->staging, *su = sr + band * es, *sv = su + band * es;
  for (int y0 = 0; y0 < c->ny; y0 += c->band_rows) {
    const int rows = std::min(c->band_rows, c->ny - y0);
    const size_t n = (size_t)rows * c->nx, off = (size_t)y0 * c->nx * es;
    CK(c->ops->fields(c->buf[c->cur], c->p, sr, su, sv, dtype, y0, rows, c->stream));
    CK(cudaMemcpyAsync((char *)rho + off, sr, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((char *)u + off, su, n * es, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((char *)v + off, sv, n * es, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_fields_device(lbm_ctx *c, float *rho, float *u, float *v) {
  if (!c || !rho || !u || !v) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(c->ops->fields(c->buf[c->cur], c->p, rho, u, v, 0, 0, c->ny, c->stream));
  return LBM_OK;
}

int lbm_mass(lbm_ctx *c, double *mass) {
  if (!c || !mass) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  std::vector<double> part((size_t)c->ny);
  CK(c->ops->mass_rows(c->buf[c->cur], c->p, (double *)c->staging, 0, c->ny, c->stream));
  CK(cudaMemcpyAsync(part.data(), c->staging, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (double d : part) s += d;
  *mass = s;
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx *c, void *dst, size_t bytes) {
  if (!c || !dst || bytes != (size_t)9 * c->nx * c->ny * c->elem) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  const size_t w = (size_t)c->nx * c->elem;
  CK(cudaMemcpy2DAsync(dst, w, c->buf[c->cur], (size_t)c->pitch * c->elem, w, (size_t)9 * c->ny,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_get_window(lbm_ctx *c, int x0, int y0, int w, int h, void *dst) {
  if (!c || !dst || w <= 0 || h <= 0 || x0 < 0 || y0 < 0 || x0 + w > c->nx || y0 + h > c->ny) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  const size_t rowb = (size_t)w * c->elem;
  for (int k = 0; k < 9; ++k) {
    const char *src = (const char *)c->buf[c->cur] + ((size_t)k * c->plane + (size_t)y0 * c->pitch + x0) * c->elem;
    CK(cudaMemcpy2DAsync((char *)dst + (size_t)k * h * rowb, rowb, src, (size_t)c->pitch * c->elem, rowb, (size_t)h,
                         cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx *c, const void *src, size_t bytes, int64_t step) {
  if (!c || !src || step < 0 || bytes != (size_t)9 * c->nx * c->ny * c->elem) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  const size_t w = (size_t)c->nx * c->elem;
  c->cur = 0;
  CK(cudaMemcpy2DAsync(c->buf[0], (size_t)c->pitch * c->elem, src, w, w, (size_t)9 * c->ny, cudaMemcpyHostToDevice,
                       c->stream));
  CK(cudaMemsetAsync(c->ctrl, 0, kAlign, c->stream));
  CK(reset_wave_rows(c));
  const unsigned long long s = (unsigned long long)step;
  CK(cudaMemcpyAsync(c->ctrl + 2, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->inited = true;
  return LBM_OK;
}

int lbm_set_kernel(lbm_ctx *c, int kernel, int ncw, int cpt, int stages, int ctas_per_sm) {
  if (!c || kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_TMA_WAVE) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  int shape = -1, ctas = 1;
  kernel = choose_kernel(c->o.storage, c->nx, c->ny, c->qmap != nullptr, kernel, ncw, cpt, stages, ctas_per_sm, &shape,
                         &ctas);
  if (kernel < 0) return LBM_ERR_ARG;
  const int rc = configure_kernel(c, kernel, std::max(shape, 0), ctas);
  if (rc) return rc;
  return capture_graph(c);
}

int lbm_set_fault_injection(lbm_ctx *c, int64_t tile, double wait_seconds) {
  if (!c) return LBM_ERR_ARG;
  if (c->kernel != LBM_KERNEL_TMA && c->kernel != LBM_KERNEL_TMA_BULK && c->kernel != LBM_KERNEL_TMA_WAVE)
    return LBM_ERR_ARG;
  if (tile >= (int64_t)c->ny * c->nseg || !(wait_seconds <= 60.0)) return LBM_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  c->p.fault_tile = tile < 0 ? -1 : (int)tile;
  c->p.wait_ns = wait_seconds > 0 ? (unsigned long long)(wait_seconds * 1e9) : 1000000000ull;
  if (c->p.wait_ns == 0) c->p.wait_ns = 1;
  return capture_graph(c);
}

int lbm_default_kernel(const lbm_opts *o, int *out5) {
  const int rc = check_opts(o);
  if (rc) return rc;
  if (!out5) return LBM_ERR_ARG;
  int shape = -1, ctas = 1;
  const int kernel = choose_kernel(o->storage, o->nx, o->ny, o->bounce == LBM_BOUNCE_INTERPOLATED, o->kernel,
                                   o->consumer_warps, o->cells_per_thread, o->stages, o->ctas_per_sm, &shape, &ctas);
  if (kernel < 0) return LBM_ERR_ARG;
  if (kernel == LBM_KERNEL_TMA_WAVE) {  // built for fewer shapes
    bool built = false;
    for (int i = 0; i < kNumWaveShapes; ++i) built = built || kWaveShapes[i].id == shape;
    if (!built) return LBM_ERR_ARG;
  }
  const bool tma = kernel != LBM_KERNEL_DIRECT;
  const TmaShape &sh = kernel == LBM_KERNEL_TMA_BULK ? kTmaBulkShapes[shape] : kTmaShapes[std::max(shape, 0)];
  out5[0] = kernel;
  out5[1] = tma ? sh.ncw : kDirectThreads / 32;
  out5[2] = tma ? sh.cpt : 1;
  out5[3] = tma ? sh.stages : 0;
  out5[4] = tma ? ctas : 0;
  return LBM_OK;
}

int lbm_get_kernel(lbm_ctx *c, int *out6) {
  if (!c || !out6) return LBM_ERR_ARG;
  const bool tma = c->kernel != LBM_KERNEL_DIRECT;
  const TmaShape &sh = c->kernel == LBM_KERNEL_TMA_BULK ? kTmaBulkShapes[c->shape] : kTmaShapes[c->shape];
  out6[0] = c->kernel;
  out6[1] = tma ? sh.ncw : kDirectThreads / 32;
  out6[2] = tma ? sh.cpt : 1;
  out6[3] = tma ? sh.stages : 0;
  out6[4] = tma ? c->ctas_per_sm : 0;
  out6[5] = c->grid;
  return LBM_OK;
}

int lbm_kernel_shapes(int *out, int cap, int *count) {
  if (!count || cap < 0 || (cap > 0 && !out)) return LBM_ERR_ARG;
  *count = kNumTmaShapes;
  for (int s = 0; s < kNumTmaShapes && s < cap; ++s) {
    out[3 * s] = kTmaShapes[s].ncw;
    out[3 * s + 1] = kTmaShapes[s].cpt;
    out[3 * s + 2] = kTmaShapes[s].stages;
  }
  return LBM_OK;
}

int lbm_kernel_shapes_for(int kernel, int *out, int cap, int *count) {
  if (kernel != LBM_KERNEL_TMA && kernel != LBM_KERNEL_TMA_BULK && kernel != LBM_KERNEL_TMA_WAVE) return LBM_ERR_ARG;
  if (!count || cap < 0 || (cap > 0 && !out)) return LBM_ERR_ARG;
  if (kernel == LBM_KERNEL_TMA_WAVE) {
    *count = kNumWaveShapes;
    for (int s = 0; s < kNumWaveShapes && s < cap; ++s) {
      out[3 * s] = kWaveShapes[s].ncw;
      out[3 * s + 1] = kWaveShapes[s].cpt;
      out[3 * s + 2] = kWaveShapes[s].stages;
    }
    return LBM_OK;
  }
  const TmaShape *list = kernel == LBM_KERNEL_TMA_BULK ? kTmaBulkShapes : kTmaShapes;
  const int n = kernel == LBM_KERNEL_TMA_BULK ? kNumTmaBulkShapes : kNumTmaShapes;
  *count = n;
  for (int s = 0; s < n && s < cap; ++s) {
    out[3 * s] = list[s].ncw;
    out[3 * s + 1] = list[s].cpt;
    out[3 * s + 2] = list[s].stages;
  }
  return LBM_OK;
}

int lbm_get_stream(lbm_ctx *c, void **stream) {
  if (!c || !stream) return LBM_ERR_ARG;
  *stream = (void *)c->stream;
  return LBM_OK;
}

int lbm_launch_count(lbm_ctx *c, int64_t *count) {
  if (!c || !count) return LBM_ERR_ARG;
  *count = c->launches;
  return LBM_OK;
}

int lbm_bytes_per_step(lbm_ctx *c, double *bytes) {
  if (!c || !bytes) return LBM_ERR_ARG;
  *bytes = 2.0 * 9.0 * c->elem * (double)c->nx * (double)c->ny;
  return LBM_OK;
}

const char *lbm_error_string(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument or geometry";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_UNSTABLE: return "unstable: |u| > 0.3 or NaN on a fluid node";
    case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
    case LBM_ERR_OOM: return "out of device memory or workspace too small";
    case LBM_ERR_RANGE: return "history entries not available";
    case LBM_ERR_STATE: return "call out of order";
  }
  return "unknown error";
}

const char *lbm_version(void) { return "gblbm 0.1 (sm_103a)"; }

}  // extern "C"
