// lbm_noalloc.cu -- lbm_step_noalloc: one fused step on caller-owned device
// buffers whose scratch memory is a fixed array in the library's device
// image, so the call allocates nothing.
//
// Who needs it: code that runs the solver where it may not call cudaMalloc
// or any allocating routine -- inside a caller's memory pool or arena, in a
// process whose allocator is owned by another runtime, or on a hot path
// that must never touch the allocator.  Such a caller already owns the
// populations (input and output) and the force output; the only memory the
// step needs besides them is its scratch: the per-tile force partials and
// the counters of the fixed-order force reduction.  Here that scratch is
// g_step_scratch below, a file-scope device array of 1 MiB that every GPU
// which loads this library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm_ctx.h"

using namespace gblbm;

namespace {

constexpr size_t kScratchBytes = size_t(1) << 20;  // 1 MiB
constexpr size_t kCtrlBytes = 256;                  // done, err, step counter
constexpr int kSlotsMax = (int)((kScratchBytes - kCtrlBytes) / sizeof(double2));
constexpr int kDirectSeg = 256;                     // tile width of the direct kernel
constexpr int kMaxDevices = 64;

// Device scratch of lbm_step_noalloc.  In host code this name is only a
// host-side stand-in; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Once per device, with that device current: look up the scratch address.
int scratch_for_device(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_step_scratch);
    if (e != cudaSuccess || !ptr) return LBM_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace

namespace gblbm {

// Called by lbm_create_ex with the context's device current: the address
// lookup (which may load the module that holds the array) happens when the
// context is made, so lbm_step_noalloc itself never triggers it.
int noalloc_prepare(int dev) {
  void *ptr = nullptr;
  return scratch_for_device(dev, &ptr);
}

}  // namespace gblbm

extern "C" int lbm_step_noalloc(lbm_ctx *c, const void *f_in, void *f_out, double *force_out) {
  if (!c || !f_in || !f_out || !force_out || f_in == f_out) return LBM_ERR_ARG;
  if (c->qmap) return LBM_ERR_ARG;  // interpolated bounce-back: the step's force needs the next step
  // Force tiles of the direct kernel (rows x 256-node tiles holding links).
  int fy0 = 0, fy1 = 0, fs0 = 0, fs1 = 0;
  const Geometry &g = c->geo;
  if (g.fx1 >= g.fx0) {
    fy0 = g.fy0;
    fy1 = g.fy1;
    fs0 = g.fx0 / kDirectSeg;
    fs1 = g.fx1 / kDirectSeg;
  }
  const long long nslots = (long long)(fy1 - fy0 + 1) * (fs1 - fs0 + 1);
  if (nslots > kSlotsMax) return LBM_ERR_ARG;  // body too large for the static scratch
  if (cudaSetDevice(c->dev) != cudaSuccess) return LBM_ERR_CUDA;
  void *scratch = nullptr;
  const int rc = scratch_for_device(c->dev, &scratch);
  if (rc) return rc;

  StepParams p = c->p;
  p.pitch = c->nx;  // packed [9][ny][nx] buffers
  p.plane = (long long)c->nx * c->ny;
  p.seg = kDirectSeg;
  p.nseg = (c->nx + kDirectSeg - 1) / kDirectSeg;
  p.fy0 = fy0;
  p.fy1 = fy1;
  p.fs0 = fs0;
  p.fs1 = fs1;
  p.nslots = (int)nslots;
  unsigned *ctrl = (unsigned *)scratch;
  p.done = ctrl;
  p.err = ctrl + 1;
  p.step = (unsigned long long *)(ctrl + 2);
  p.slots = (double2 *)((char *)scratch + kCtrlBytes);
  p.hist = force_out;
  p.hist_cap = 1;
  // The array keeps the previous call's contents: the reduction counter and
  // the history index must start at zero.
  if (cudaMemsetAsync(scratch, 0, kCtrlBytes, c->stream) != cudaSuccess) return LBM_ERR_CUDA;
  if (c->ops->direct(f_in, f_out, p, c->stream) != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}
