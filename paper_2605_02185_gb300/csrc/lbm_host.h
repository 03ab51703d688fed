// lbm_host.h -- host-side helpers shared by the C ABI translation units:
// storage types, option checks, geometry preprocessing, error mapping and
// the tuned default kernel shapes.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lbm_ctx.h"

namespace gblbm {

inline constexpr size_t kAlign = 256;
inline constexpr int kDirectThreads = 256;
inline constexpr size_t kBandCells = size_t(1) << 20;  // staging band for init / fields

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline const KernelOps *ops_for(int storage) {
  switch (storage) {
    case LBM_F32: return ops_f32();
    case LBM_F16_OFS: return ops_f16();
    case LBM_BF16_OFS: return ops_bf16();
    case LBM_F64: return ops_f64();
    case LBM_F16_SR: return ops_f16sr();
    case LBM_BF16_SR: return ops_bf16sr();
  }
  return nullptr;
}

inline int elem_size(int storage) {
  switch (storage) {
    case LBM_F32: return 4;
    case LBM_F16_OFS: return 2;
    case LBM_BF16_OFS: return 2;
    case LBM_F64: return 8;
    case LBM_F16_SR: return 2;
    case LBM_BF16_SR: return 2;
  }
  return 0;
}


inline int check_opts(const lbm_opts *o) {
  if (!o) return LBM_ERR_ARG;
  if (o->nx < 5 || o->ny < 5) return LBM_ERR_ARG;
  if ((long long)o->nx * o->ny > (1ll << 31) - 1) return LBM_ERR_ARG;
  if (!(o->tau > 0.5) || !std::isfinite(o->tau)) return LBM_ERR_ARG;
  if (!(o->U >= 0.0 && o->U < 0.3)) return LBM_ERR_ARG;
  if (o->bc_top_bottom < LBM_BC_FREESLIP || o->bc_top_bottom > LBM_BC_MOVINGWALL) return LBM_ERR_ARG;
  if (!elem_size(o->storage)) return LBM_ERR_ARG;
  if (o->kernel < LBM_KERNEL_AUTO || o->kernel > LBM_KERNEL_TMA_WAVE) return LBM_ERR_ARG;
  if (o->collision != LBM_COLLIDE_BGK && o->collision != LBM_COLLIDE_MRT) return LBM_ERR_ARG;
  if (o->collision == LBM_COLLIDE_MRT &&
      !(o->s_e > 0.0 && o->s_e < 2.0 && o->s_eps > 0.0 && o->s_eps < 2.0 && o->s_q > 0.0 && o->s_q < 2.0))
    return LBM_ERR_ARG;
  if (o->bounce != LBM_BOUNCE_HALFWAY && o->bounce != LBM_BOUNCE_INTERPOLATED) return LBM_ERR_ARG;
  if (o->bounce == LBM_BOUNCE_INTERPOLATED && !(o->body_r > 0.0 && std::isfinite(o->body_xc) &&
                                                std::isfinite(o->body_yc) && std::isfinite(o->body_r)))
    return LBM_ERR_ARG;
  return LBM_OK;
}

// Fraction q of the link from (x, y) along c_i at which it meets the circle
// (cx, cy, r): the smallest t in (0, 1] with |(x, y) + t c_i - c| = r; 1/2
// where the circle does not cross the link.
inline float circle_fraction(int x, int y, int i, double cx, double cy, double r) {
  const double dx = x - cx, dy = y - cy;
  const double a = (double)(CX(i) * CX(i) + CY(i) * CY(i));
  const double b = dx * CX(i) + dy * CY(i);
  const double c = dx * dx + dy * dy - r * r;
  const double disc = b * b - a * c;
  const double t = disc >= 0.0 ? (-b - std::sqrt(disc)) / a : -1.0;
  return (float)((t > 0.0 && t <= 1.0) ? t : 0.5);
}

inline int build_geometry(const lbm_opts *o, const uint8_t *mask, Geometry *g) {
  const int nx = o->nx, ny = o->ny;
  int x0 = nx, x1 = -1, y0 = ny, y1 = -1;
  if (mask) {
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        if (mask[(size_t)y * nx + x]) {
          if (x < 2 || x > nx - 3 || y < 2 || y > ny - 3) return LBM_ERR_ARG;
          x0 = std::min(x0, x);
          x1 = std::max(x1, x);
          y0 = std::min(y0, y);
          y1 = std::max(y1, y);
        }
  }
  if (x1 < 0) {  // no solid: an empty map
    g->lx0 = g->ly0 = 0;
    g->lw = g->lh = 0;
    return LBM_OK;
  }
  g->solid_rows = y1 - y0 + 1;
  g->lx0 = x0 - 1;
  g->ly0 = y0 - 1;
  g->lw = x1 - x0 + 3;
  g->lh = y1 - y0 + 3;
  g->lmap.assign((size_t)g->lw * g->lh, 0);
  const bool interp = o->bounce == LBM_BOUNCE_INTERPOLATED;
  if (interp) g->qmap.assign((size_t)g->lw * g->lh * 8, 0.5f);
  auto solid = [&](int x, int y) { return mask[(size_t)y * nx + x] != 0; };
  long double fcx = 0.0L, fcy = 0.0L;
  for (int j = 0; j < g->lh; ++j)
    for (int i = 0; i < g->lw; ++i) {
      const int x = g->lx0 + i, y = g->ly0 + j;
      uint16_t m = 0;
      if (solid(x, y)) {
        m = (uint16_t)LM_SOLID;
      } else {
        for (int k = 1; k < 9; ++k) {
          const int sx = x - CX(k), sy = y - CY(k);  // inside by the solid margin
          if (solid(sx, sy)) m |= (uint16_t)(1u << k);
        }
        if (m) {
          g->fx0 = g->fx1 < g->fx0 ? x : std::min(g->fx0, x);
          g->fx1 = std::max(g->fx1, x);
          g->fy0 = g->fy1 < g->fy0 ? y : std::min(g->fy0, y);
          g->fy1 = std::max(g->fy1, y);
          for (int d = 1; d < 9; ++d)
            if (m & (1u << OPP(d))) {  // d points into the solid
              // reference part of the link's momentum exchange: 2 r_d c_d
              // (half-way) or (r_d + r_opp(d)) c_d (interpolated)
              const long double rr = interp ? (long double)ref_pop(d, o->U) + (long double)ref_pop(OPP(d), o->U)
                                            : 2.0L * (long double)ref_pop(d, o->U);
              fcx += rr * CX(d);
              fcy += rr * CY(d);
              ++g->links;
            }
          if (interp) {
            for (int k = 1; k < 9; ++k) {
              if (!(m & (1u << k))) continue;
              // arriving direction k left x along i = opp(k); below q = 1/2
              // the node behind, x + c_k, must be fluid, else half-way
              float q = circle_fraction(x, y, OPP(k), o->body_xc, o->body_yc, o->body_r);
              if (q < 0.5f && solid(x + CX(k), y + CY(k))) q = 0.5f;
              g->qmap[((size_t)j * g->lw + i) * 8 + (k - 1)] = q;
            }
          }
        }
      }
      g->lmap[(size_t)j * g->lw + i] = m;
    }
  g->fconst_x = (double)fcx;
  g->fconst_y = (double)fcy;
  return LBM_OK;
}


inline int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
}

#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// Default TMA shape (an index into GBLBM_TMA_SHAPES) and CTAs per SM of a
// single lattice, from a sweep of every shape at 1 and 2 CTAs/SM on FP32
// cylinder lattices (CUDA events, BGK):
//   >= 16M nodes (16000 x 8000, 8000 x 4000): 12 compute warps x 2 nodes,
//     4 stages (768-node tiles), 1 CTA/SM -- 90.2 and 89.3 GLUPS (the 512-node
//     tile that wastes least on an 8000-node row ran at 59.3);
//   3M .. 16M nodes (3200 x 1600): 16 warps x 1 node, 4 stages (512-node
//     tiles), 2 CTAs/SM -- 77.6 against 73.3 for 640-node tiles at 1 CTA/SM;
//   < 3M nodes (1600 x 800): 10 warps x 2 nodes, 4 stages (640-node tiles),
//     2 CTAs/SM -- 58.7 against 50.6 at 1 CTA/SM.
// 16-bit storage: 12 x 2 x 4 at 2 CTAs/SM (the fastest shape for all four
// 16-bit forms on 16000 x 8000, 0.89 of the copy bandwidth with rounding to
// nearest); double storage: 8 x 2 x 4 at 1 CTA/SM (FP64-ALU bound; it
// runs on the direct kernel by default).  The TMA kernel with interpolated
// bounce-back and the multi-step kernel are built for fewer shapes
// (few_shapes): there float storage takes 12 x 2 x 4 from 16M nodes up and
// 10 x 2 x 4 below, at 1 CTA/SM.
struct DefaultShape {
  int shape, ctas;
};
inline DefaultShape default_shape(int storage, long long nodes, bool few_shapes) {
  if (storage == LBM_F64) return {6, 1};
  if (storage != LBM_F32) return {12, 2};
  if (nodes >= (16ll << 20)) return {12, 1};
  if (few_shapes) return {15, 1};
  if (nodes >= (3ll << 20)) return {11, 2};
  return {15, 2};
}
// Batches of many small lattices: shape 19 (13 compute warps, 2 cells per
// thread, 3 stages: 832-node row tiles, which fit rows of 800-2400 nodes with
// little waste) at 2 CTAs per SM, the autotuner's pick for 64 cases of
// 800-2400 nodes wide (67-68 GLUPS with MRT, 1.48x the same cases run one after
// another as single lattices in their default shapes).
inline int default_batch_shape(int storage) { return storage == LBM_F64 ? 6 : 19; }
inline int default_batch_ctas(int storage) { return storage == LBM_F64 ? 1 : 2; }
inline int default_kernel(int storage) { return storage == LBM_F64 ? LBM_KERNEL_DIRECT : LBM_KERNEL_TMA; }


}  // namespace gblbm
