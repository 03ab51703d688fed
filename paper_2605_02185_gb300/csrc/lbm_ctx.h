// lbm_ctx.h -- the lattice context shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/gblbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace gblbm {

// Host-side geometry: link map over the solid bounding box grown by one
// node, the reference part (sum of 2 r_i c_i) of the Eq. 14 sum, and the
// bounding box of the fluid nodes that own links.
struct Geometry {
  int lx0 = 0, ly0 = 0, lw = 0, lh = 0;
  std::vector<uint16_t> lmap;
  std::vector<float> qmap;  // interpolated bounce-back: [lh][lw][8] fractions per arriving direction
  double fconst_x = 0.0, fconst_y = 0.0;
  int fx0 = 0, fx1 = -1, fy0 = 0, fy1 = -1;  // link-owning fluid nodes
  int solid_rows = 0;
  long long links = 0;
};

}  // namespace gblbm

struct lbm_ctx {
  lbm_opts o{};
  int dev = 0, sms = 0;
  int nx = 0, ny = 0, pitch = 0, elem = 0;
  long long plane = 0;
  const gblbm::KernelOps *ops = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  void *buf[2] = {nullptr, nullptr};
  int cur = 0;  // buf[cur] holds the current f*
  uint16_t *lmap = nullptr;
  float *qmap = nullptr;
  double2 *slots = nullptr;
  int slot_cap = 0;
  double *hist = nullptr;
  long long hist_cap = 0;
  unsigned *ctrl = nullptr;  // [0] done, [1] err, [2..3] step counter
  void *staging = nullptr;
  size_t staging_bytes = 0;
  int band_rows = 1;
  gblbm::Geometry geo;
  double D_ref = 0.0, rho_in = 1.0;
  bool inited = false;
  long long launches = 0;
  // step kernel
  int kernel = LBM_KERNEL_TMA, shape = 0, ctas_per_sm = 1, grid = 0, seg = 0, nseg = 0;
  gblbm::StepParams p{};
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // multi-step kernel: per-row completion counters, the steps they have
  // counted, and the force slots of one launch's steps
  unsigned *wave_rows = nullptr;
  unsigned wave_base = 0;
  double2 *wave_slots = nullptr;
};
