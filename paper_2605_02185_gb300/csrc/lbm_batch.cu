// lbm_batch.cu -- many independent cylinder lattices advanced by ONE kernel
// launch per step.
//
// Each case is an ordinary lattice context (geometry, link map, force
// history, its own population buffers) carved out of one shared workspace
// and sharing one stream.  The batch concatenates the row tiles of all cases
// into one tile numbering; a single launch of the batched step kernel --
// persistent and TMA-staged, or direct -- walks that numbering, so small
// lattices that could not fill the GPU alone share it.  A CUDA graph of
// several steps removes the per-launch host cost.  Per-case queries
// (fields, forces, checkpoints) go to the case's context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gblbm.h"
#include "lbm_ctx.h"
#include "lbm_host.h"

using namespace gblbm;

struct lbm_batch {
  int dev = 0, sms = 0;
  lbm_opts common{};
  std::vector<lbm_ctx *> cases;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  CaseDesc *desc = nullptr;  // device array, one per case
  long long nitems = 0;
  long long nodes = 0;
  int kernel = LBM_KERNEL_TMA, shape = 0, ctas = 1, grid = 0;
  int cur = 0;
  long long launches = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
};

namespace {

lbm_opts case_opts(const lbm_opts &common, const lbm_case &cs) {
  lbm_opts o = common;
  o.nx = cs.nx;
  o.ny = cs.ny;
  o.tau = cs.tau;
  o.U = cs.U;
  o.bc_top_bottom = cs.bc_top_bottom;
  o.D_ref = cs.D_ref;
  o.rho_in = cs.rho_in;
  o.graph_steps = -1;  // the batch captures its own graphs
  o.workspace = nullptr;
  o.workspace_bytes = 0;
  return o;
}

size_t desc_bytes(int n) { return align_up((size_t)n * sizeof(CaseDesc), kAlign); }

int batch_sizes(int n, const lbm_case *cases, const lbm_opts *common, std::vector<size_t> *sizes, size_t *total) {
  if (n <= 0 || !cases || !common) return LBM_ERR_ARG;
  size_t sum = 0;
  sizes->assign((size_t)n, 0);
  for (int c = 0; c < n; ++c) {
    lbm_opts o = case_opts(*common, cases[c]);
    size_t b = 0;
    const int rc = lbm_workspace_bytes(&o, cases[c].mask, &b);
    if (rc) return rc;
    (*sizes)[c] = align_up(b, kAlign);
    sum += (*sizes)[c];
  }
  *total = sum + desc_bytes(n);
  return LBM_OK;
}

// Give every case the tile width of the batch kernel, then upload the
// per-case descriptors with the batch-wide tile offsets.
int configure_batch(lbm_batch *b, int kernel, int shape, int ctas) {
  if (kernel == LBM_KERNEL_TMA_BULK) return LBM_ERR_ARG;  // single-lattice kernel only
  const TmaShape &ts = kTmaShapes[shape];
  for (lbm_ctx *c : b->cases) {
    const int rc = kernel == LBM_KERNEL_DIRECT ? lbm_set_kernel(c, LBM_KERNEL_DIRECT, 0, 0, 0, 1)
                                               : lbm_set_kernel(c, LBM_KERNEL_TMA, ts.ncw, ts.cpt, ts.stages, ctas);
    if (rc) return rc;
  }
  const KernelOps *ops = b->cases[0]->ops;
  if (kernel != LBM_KERNEL_DIRECT) CK(ops->batch_prep(shape));
  std::vector<CaseDesc> h(b->cases.size());
  long long item0 = 0, nodes = 0;
  for (size_t i = 0; i < b->cases.size(); ++i) {
    lbm_ctx *c = b->cases[i];
    h[i].p = c->p;
    h[i].buf[0] = c->buf[0];
    h[i].buf[1] = c->buf[1];
    h[i].item0 = item0;
    item0 += (long long)c->ny * c->nseg;
    nodes += (long long)c->nx * c->ny;
  }
  if (item0 > (1ll << 31) - 1) return LBM_ERR_ARG;
  CK(cudaMemcpyAsync(b->desc, h.data(), h.size() * sizeof(CaseDesc), cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  b->nitems = item0;
  b->nodes = nodes;
  b->kernel = kernel;
  b->shape = shape;
  b->ctas = kernel == LBM_KERNEL_DIRECT ? 0 : b->cases[0]->ctas_per_sm;
  b->grid = kernel == LBM_KERNEL_DIRECT ? (int)item0 : (int)std::min<long long>(item0, (long long)b->sms * b->ctas);
  return LBM_OK;
}

cudaError_t launch_batch(lbm_batch *b, int parity) {
  const KernelOps *ops = b->cases[0]->ops;
  const int n = (int)b->cases.size();
  const int mrt = b->common.collision == LBM_COLLIDE_MRT ? 1 : 0;
  if (b->kernel == LBM_KERNEL_DIRECT) return ops->batch_direct(b->desc, n, b->nitems, parity, mrt, b->stream);
  return ops->batch_tma(b->shape, b->grid, b->desc, n, b->nitems, parity, mrt, b->stream);
}

int capture_batch_graph(lbm_batch *b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  int gs = b->common.graph_steps;
  if (gs < 0) {
    b->graph_steps = 0;
    return LBM_OK;
  }
  if (gs == 0) gs = (int)std::max<long long>(2, std::min<long long>(256, (16ll << 20) / std::max(b->nodes, 1ll)));
  gs += gs & 1;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int s = 0; s < gs && err == cudaSuccess; ++s) err = launch_batch(b, s & 1);
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(err != cudaSuccess ? err : e2);
  }
  err = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  CK(err);
  CK(cudaGraphUpload(b->graph, b->stream));
  b->graph_steps = gs;
  return LBM_OK;
}

bool valid_case(const lbm_batch *b, int c) { return b && c >= 0 && c < (int)b->cases.size(); }

}  // namespace

extern "C" {

int lbm_batch_workspace_bytes(int ncases, const lbm_case *cases, const lbm_opts *common, size_t *bytes) {
  if (!bytes) return LBM_ERR_ARG;
  std::vector<size_t> sizes;
  return batch_sizes(ncases, cases, common, &sizes, bytes);
}

int lbm_batch_create(int ncases, const lbm_case *cases, const lbm_opts *common, lbm_batch **out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (common && common->bounce != LBM_BOUNCE_HALFWAY) return LBM_ERR_ARG;  // single lattices only
  std::vector<size_t> sizes;
  size_t total = 0;
  int rc = batch_sizes(ncases, cases, common, &sizes, &total);
  if (rc) return rc;
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->common = *common;
  auto fail = [&](int code) {
    lbm_batch_destroy(b);
    return code;
  };
  if (cudaGetDevice(&b->dev) != cudaSuccess) return fail(LBM_ERR_CUDA);
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess)
    return fail(LBM_ERR_CUDA);
  if (common->workspace) {
    if (common->workspace_bytes < total || ((uintptr_t)common->workspace % kAlign) != 0) return fail(LBM_ERR_OOM);
    b->ws = common->workspace;
  } else {
    size_t freeb = 0, tot = 0;
    if (cudaMemGetInfo(&freeb, &tot) != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (total > freeb) return fail(LBM_ERR_OOM);
    if (cudaMalloc(&b->ws, total) != cudaSuccess) return fail(LBM_ERR_OOM);
    b->own_ws = true;
  }
  b->ws_bytes = total;
  if (common->stream) {
    b->stream = (cudaStream_t)common->stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LBM_ERR_CUDA);
    b->own_stream = true;
  }
  char *base = (char *)b->ws;
  size_t off = 0;
  for (int c = 0; c < ncases; ++c) {
    lbm_opts o = case_opts(*common, cases[c]);
    o.stream = (void *)b->stream;
    o.workspace = base + off;
    o.workspace_bytes = sizes[c];
    off += sizes[c];
    lbm_ctx *ctx = nullptr;
    rc = lbm_create_ex(&o, cases[c].mask, &ctx);
    if (rc) return fail(rc);
    b->cases.push_back(ctx);
  }
  b->desc = (CaseDesc *)(base + off);
  int kernel = common->kernel, shape = default_batch_shape(common->storage);
  int ctas = common->ctas_per_sm > 0 ? common->ctas_per_sm : default_batch_ctas(common->storage);
  if (common->consumer_warps || common->cells_per_thread || common->stages) {
    shape = -1;
    for (int s = 0; s < kNumTmaShapes; ++s)
      if (kTmaShapes[s].ncw == common->consumer_warps && kTmaShapes[s].cpt == common->cells_per_thread &&
          kTmaShapes[s].stages == common->stages)
        shape = s;
    if (shape < 0) return fail(LBM_ERR_ARG);
  }
  if (kernel == LBM_KERNEL_AUTO) kernel = default_kernel(common->storage);
  rc = configure_batch(b, kernel, shape, ctas);
  if (rc) return fail(rc);
  rc = capture_batch_graph(b);
  if (rc) return fail(rc);
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (lbm_ctx *c : b->cases) lbm_destroy(c);
  if (b->own_ws && b->ws) cudaFree(b->ws);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int lbm_batch_case(lbm_batch *b, int c, lbm_ctx **ctx) {
  if (!valid_case(b, c) || !ctx) return LBM_ERR_ARG;
  *ctx = b->cases[c];
  return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch *b, int c, const double *rho, const double *u, const double *v) {
  if (!valid_case(b, c)) return LBM_ERR_ARG;
  lbm_ctx *ctx = b->cases[c];
  // the batch steps all cases with one parity: bring this case's f*(0) to it
  int rc = lbm_init_fields(ctx, rho, u, v);
  if (rc) return rc;
  if (b->cur != 0) {
    CK(cudaMemcpyAsync(ctx->buf[1], ctx->buf[0], (size_t)9 * ctx->plane * ctx->elem, cudaMemcpyDeviceToDevice,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    ctx->cur = 1;
  }
  return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int64_t n) {
  if (!b || n < 0) return LBM_ERR_ARG;
  for (lbm_ctx *c : b->cases)
    if (!c->inited) return LBM_ERR_STATE;
  CK(cudaSetDevice(b->dev));
  while (n > 0) {
    if (b->graph && b->cur == 0 && n >= b->graph_steps) {
      CK(cudaGraphLaunch(b->graph, b->stream));
      n -= b->graph_steps;
      b->launches += b->graph_steps;
    } else {
      CK(launch_batch(b, b->cur));
      b->cur ^= 1;
      --n;
      ++b->launches;
    }
  }
  for (lbm_ctx *c : b->cases) c->cur = b->cur;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch *b) {
  if (!b) return LBM_ERR_ARG;
  int worst = LBM_OK;
  for (lbm_ctx *c : b->cases) {
    const int rc = lbm_sync(c);
    if (rc == LBM_ERR_TIMEOUT || (rc && worst != LBM_ERR_TIMEOUT)) worst = rc;
  }
  return worst;
}

int lbm_batch_set_kernel(lbm_batch *b, int kernel, int ncw, int cpt, int stages, int ctas_per_sm) {
  if (!b || kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_TMA) return LBM_ERR_ARG;
  CK(cudaSetDevice(b->dev));
  CK(cudaStreamSynchronize(b->stream));
  const int storage = b->common.storage;
  int shape = default_batch_shape(storage);
  int ctas = ctas_per_sm > 0 ? ctas_per_sm : default_batch_ctas(storage);
  if (kernel != LBM_KERNEL_DIRECT && (ncw || cpt || stages)) {
    shape = -1;
    for (int s = 0; s < kNumTmaShapes; ++s)
      if (kTmaShapes[s].ncw == ncw && kTmaShapes[s].cpt == cpt && kTmaShapes[s].stages == stages) shape = s;
    if (shape < 0) return LBM_ERR_ARG;
  } else if (kernel == LBM_KERNEL_AUTO) {
    kernel = default_kernel(storage);
  }
  const int rc = configure_batch(b, kernel, shape, ctas);
  if (rc) return rc;
  return capture_batch_graph(b);
}

int lbm_batch_get_kernel(lbm_batch *b, int *out6) {
  if (!b || !out6) return LBM_ERR_ARG;
  const bool tma = b->kernel != LBM_KERNEL_DIRECT;
  out6[0] = b->kernel;
  out6[1] = tma ? kTmaShapes[b->shape].ncw : kDirectThreads / 32;
  out6[2] = tma ? kTmaShapes[b->shape].cpt : 1;
  out6[3] = tma ? kTmaShapes[b->shape].stages : 0;
  out6[4] = b->ctas;
  out6[5] = b->grid;
  return LBM_OK;
}

int lbm_batch_get_stream(lbm_batch *b, void **stream) {
  if (!b || !stream) return LBM_ERR_ARG;
  *stream = (void *)b->stream;
  return LBM_OK;
}

int lbm_batch_launch_count(lbm_batch *b, int64_t *count) {
  if (!b || !count) return LBM_ERR_ARG;
  *count = b->launches;
  return LBM_OK;
}

int lbm_batch_nodes(lbm_batch *b, int64_t *nodes, double *bytes_per_step) {
  if (!b || !nodes) return LBM_ERR_ARG;
  *nodes = b->nodes;
  if (bytes_per_step) *bytes_per_step = 2.0 * 9.0 * b->cases[0]->elem * (double)b->nodes;
  return LBM_OK;
}

}  // extern "C"
