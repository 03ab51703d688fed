// lbm_internal.h -- interfaces between the C ABI layer and the per-storage
// kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace gblbm {

struct StepParams;
struct CaseDesc;
struct WaveParams;

// Launchers of one storage type.  All launches are asynchronous on `st`.
struct KernelOps {
  int elem;  // bytes per stored population value
  cudaError_t (*direct)(const void *A, void *B, const StepParams &p, cudaStream_t st);
  cudaError_t (*tma)(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st);
  cudaError_t (*prep)(int shape);  // set the dynamic shared memory limit of a TMA shape
  int (*occupancy)(int shape);     // resident CTAs per SM of a TMA shape (0: does not fit)
  size_t (*smem)(int shape);
  cudaError_t (*init)(void *A, const StepParams &p, const double *rho, const double *u, const double *v, int y0,
                      int rows, cudaStream_t st);
  cudaError_t (*force)(const void *A, const StepParams &p, cudaStream_t st);
  cudaError_t (*fields)(const void *A, const StepParams &p, void *rho, void *u, void *v, int dbl, int y0, int rows,
                        cudaStream_t st);
  cudaError_t (*mass_rows)(const void *A, const StepParams &p, double *part, int y0, int rows, cudaStream_t st);
  // batched step over the concatenated row tiles of `ncases` lattices
  cudaError_t (*batch_direct)(const CaseDesc *cases, int ncases, long long nitems, int parity, int mrt,
                              cudaStream_t st);
  cudaError_t (*batch_tma)(int shape, int grid, const CaseDesc *cases, int ncases, long long nitems, int parity,
                           int mrt, cudaStream_t st);
  cudaError_t (*batch_prep)(int shape);
  // initial state from device float fields, optionally with non-equilibrium part
  cudaError_t (*init_device)(void *A, const StepParams &p, const float *rho, const float *u, const float *v,
                             int with_noneq, double tau, cudaStream_t st);
  // the TMA-load + TMA-bulk-store step kernel, shapes of GBLBM_TMA_BULK_SHAPES
  cudaError_t (*tma_bulk)(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st);
  cudaError_t (*bulk_prep)(int shape);
  int (*bulk_occupancy)(int shape);
  size_t (*bulk_smem)(int shape);
  // nodes per thread and chunk of the single-lattice TMA kernel: its row
  // tile is tma_pair * warps * 32 * cells-per-thread nodes wide
  int tma_pair;
  // the TMA kernel with interpolated bounce-back (prep != 0: only set its
  // shared-memory limit); cudaErrorNotSupported for storage types and
  // shapes it is not built for
  cudaError_t (*tma_interp)(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st,
                            int prep);
  // the multi-step TMA kernel (w.steps steps from A, then B, ... in one
  // cooperative launch) and the reduction of its force slots into the
  // history; shapes of GBLBM_WAVE_SHAPES (cudaErrorNotSupported otherwise)
  cudaError_t (*wave)(int shape, int grid, void *A, void *B, const StepParams &p, const WaveParams &w,
                      cudaStream_t st);
  cudaError_t (*wave_prep)(int shape);
  int (*wave_occupancy)(int shape);
};

// Look up (once per device) the address of lbm_step_noalloc's static
// scratch array; lbm_create_ex calls it so that the lookup never happens
// inside a no-allocation step.
int noalloc_prepare(int dev);

const KernelOps *ops_f32();
const KernelOps *ops_f16();
const KernelOps *ops_bf16();
const KernelOps *ops_f64();
const KernelOps *ops_f16sr();
const KernelOps *ops_bf16sr();

// TMA kernel shapes X(id, compute warps, cells per thread, stages).
#define GBLBM_TMA_SHAPES(X) \
  X(0, 8, 4, 4)             \
  X(1, 8, 2, 6)             \
  X(2, 16, 2, 3)            \
  X(3, 16, 1, 6)            \
  X(4, 8, 1, 8)             \
  X(5, 4, 4, 8)             \
  X(6, 8, 2, 4)             \
  X(7, 4, 2, 6)             \
  X(8, 8, 1, 4)             \
  X(9, 4, 2, 4)             \
  X(10, 8, 2, 3)            \
  X(11, 16, 1, 4)           \
  X(12, 12, 2, 4)           \
  X(13, 16, 2, 2)           \
  X(14, 4, 2, 3)            \
  X(15, 10, 2, 4)           \
  X(16, 13, 1, 6)           \
  X(17, 13, 1, 4)           \
  X(18, 10, 1, 6)           \
  X(19, 13, 2, 3)           \
  X(20, 13, 2, 2)

// Shapes (ids and triples of GBLBM_TMA_SHAPES) the multi-step kernel is
// built for: the float defaults by lattice width and the 16-bit default.
#define GBLBM_WAVE_SHAPES(X) \
  X(6, 8, 2, 4)              \
  X(12, 12, 2, 4)            \
  X(15, 10, 2, 4)            \
  X(19, 13, 2, 3)

// Shapes of the TMA-load + TMA-bulk-store kernel X(id, warps, cells/thread, stages).
#define GBLBM_TMA_BULK_SHAPES(X) \
  X(0, 12, 2, 4)                 \
  X(1, 12, 2, 3)                 \
  X(2, 8, 2, 4)                  \
  X(3, 16, 1, 4)                 \
  X(4, 8, 4, 3)

struct TmaShape {
  int ncw, cpt, stages;
};
#define GBLBM_SHAPE_ENTRY(id, a, b, c) {a, b, c},
constexpr TmaShape kTmaShapes[] = {GBLBM_TMA_SHAPES(GBLBM_SHAPE_ENTRY)};
#undef GBLBM_SHAPE_ENTRY
constexpr int kNumTmaShapes = (int)(sizeof(kTmaShapes) / sizeof(kTmaShapes[0]));
#define GBLBM_WAVE_CHECK(id, a, b, c)                                                             \
  static_assert(kTmaShapes[id].ncw == a && kTmaShapes[id].cpt == b && kTmaShapes[id].stages == c, \
                "multi-step shape id does not match the TMA shape list");
GBLBM_WAVE_SHAPES(GBLBM_WAVE_CHECK)
#undef GBLBM_WAVE_CHECK
#define GBLBM_SHAPE_ENTRY(id, a, b, c) {id, a, b, c},
struct WaveShape {
  int id, ncw, cpt, stages;
};
constexpr WaveShape kWaveShapes[] = {GBLBM_WAVE_SHAPES(GBLBM_SHAPE_ENTRY)};
#undef GBLBM_SHAPE_ENTRY
constexpr int kNumWaveShapes = (int)(sizeof(kWaveShapes) / sizeof(kWaveShapes[0]));
// Steps per launch of the multi-step kernel.
constexpr int kWaveSteps = 64;
#define GBLBM_SHAPE_ENTRY(id, a, b, c) {a, b, c},
constexpr TmaShape kTmaBulkShapes[] = {GBLBM_TMA_BULK_SHAPES(GBLBM_SHAPE_ENTRY)};
#undef GBLBM_SHAPE_ENTRY
constexpr int kNumTmaBulkShapes = (int)(sizeof(kTmaBulkShapes) / sizeof(kTmaBulkShapes[0]));

}  // namespace gblbm
