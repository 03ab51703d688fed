// lbm_device.cuh -- device building blocks of the fused D2Q9 step.
//
// Populations are stored as offsets g_i = f_i - w_i (Table 1 weights), in
// the storage type S, in 9 planes [k][ny][pitch].  Arithmetic is float for
// float/half/bfloat16 storage and double for double storage.  Working with
// offsets keeps the stored magnitudes near |c_i.u| w_i instead of w_i, which
// gives the 16-bit forms usable precision and the float form ~16x smaller
// rounding steps; every rule below is linear in f with weight-symmetric
// coefficients, so it reads the same on g.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gblbm {

// ---- D2Q9 lattice, Table 1, k = i - 1 -----------------------------------
__host__ __device__ constexpr int CX(int k) { return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0); }
__host__ __device__ constexpr int CY(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }
__host__ __device__ constexpr int OPP(int k) { return k == 0 ? 0 : (k <= 4 ? ((k + 1) & 3) + 1 : ((k - 3) & 3) + 5); }
__host__ __device__ constexpr double WD(int k) { return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

static_assert(OPP(1) == 3 && OPP(3) == 1 && OPP(2) == 4 && OPP(4) == 2, "opposites");
static_assert(OPP(5) == 7 && OPP(7) == 5 && OPP(6) == 8 && OPP(8) == 6, "opposites");

enum { BC_FREESLIP = 0, BC_PERIODIC = 1, BC_ZOUHE = 2 };

// link-map bits: bit k (1..8) = the pull source x - c_k is solid; bit 15 = solid node
constexpr uint32_t LM_SOLID = 1u << 15;
constexpr uint32_t LM_LINKS = 0x1FEu;

// device error word bits
constexpr unsigned ERR_UNSTABLE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;

// ---- storage conversion --------------------------------------------------
template <class S> struct Store;
template <> struct Store<float> {
  using C = float;
  __device__ static __forceinline__ C ld(float v) { return v; }
  __device__ static __forceinline__ float st(C v) { return v; }
};
template <> struct Store<__half> {
  using C = float;
  __device__ static __forceinline__ C ld(__half v) { return __half2float(v); }
  __device__ static __forceinline__ __half st(C v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  __device__ static __forceinline__ C ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ __nv_bfloat16 st(C v) { return __float2bfloat16_rn(v); }
};
template <> struct Store<double> {
  using C = double;
  __device__ static __forceinline__ C ld(double v) { return v; }
  __device__ static __forceinline__ double st(C v) { return v; }
};

// ---- per-step parameters (passed by value) -------------------------------
struct StepParams {
  int nx, ny, pitch, bc;
  long long plane;         // elements per population plane
  double omega;            // 1 / tau
  double U;                // inlet / wall speed
  // link map over the region [lx0, lx0+lw) x [ly0, ly0+lh)
  const uint16_t *lmap;
  int lx0, ly0, lw, lh;
  // row tiles: item t -> row t / nseg, segment t % nseg of seg cells
  int seg, nseg;
  // force items: rows [fy0, fy1], segments [fs0, fs1]; one slot each
  int fy0, fy1, fs0, fs1;
  int nslots;
  double2 *slots;
  unsigned *done;               // items of this step that posted their slot
  unsigned *err;                // ERR_* bits
  unsigned long long *step;     // history entries written so far
  double *hist;                 // ring [cap][2] of (Fx, Fy)
  long long hist_cap;
  double fconst_x, fconst_y;    // sum over links of 2 w_i c_i (offset part removed)
};

__device__ __forceinline__ uint32_t link_mask(const StepParams &p, int x, int y) {
  unsigned dx = (unsigned)(x - p.lx0), dy = (unsigned)(y - p.ly0);
  if (dx < (unsigned)p.lw && dy < (unsigned)p.lh) return __ldg(p.lmap + (size_t)dy * p.lw + dx);
  return 0u;
}

// Pull (left side of Eq. 2) for the node (xe, y): g[k] = g*_k(xe - c_k).
// A source outside the lattice yields the node's own g*_k (placeholder, later
// overwritten by a boundary rule); a solid source yields the node's own
// g*_opp(k) (half-way bounce-back, reflected within the step).  Regular
// sources come from fetch(k, sx) -- a staged row tile or HBM.
template <class S, class Fetch>
__device__ __forceinline__ void pull(const S *__restrict__ A, const StepParams &p, int xe, int y, uint32_t lm,
                                     Fetch fetch, typename Store<S>::C g[9]) {
  const size_t own = (size_t)y * p.pitch + xe;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int sx = xe - CX(k);
    int sy = y - CY(k);
    bool inside = (unsigned)sx < (unsigned)p.nx;
    if (p.bc == BC_PERIODIC) {
      sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
    } else {
      inside = inside && (unsigned)sy < (unsigned)p.ny;
    }
    if (!inside) {
      g[k] = Store<S>::ld(A[(size_t)k * p.plane + own]);
    } else if (lm & (1u << k)) {
      g[k] = Store<S>::ld(A[(size_t)OPP(k) * p.plane + own]);
    } else {
      g[k] = fetch(k, sx, sy);
    }
  }
}

// Boundary corrections after streaming (Section 2.3), in the order top row,
// bottom row, inlet column.  The outlet (Eq. 13) is realised by computing
// column nx-2 for column nx-1.  Every rule is written on offsets g = f - w;
// the weights cancel because each rule pairs directions of equal weight and
// the weights of each Zou-He density sum to one.
template <class C>
__device__ __forceinline__ void boundaries(C g[9], int xe, int y, const StepParams &p) {
  const C U = (C)p.U;
  if (p.bc != BC_PERIODIC) {
    if (y == p.ny - 1) {
      if (p.bc == BC_FREESLIP) {  // Eq. 7a: f5 = f3, f8 = f7, f9 = f6
        g[4] = g[2];
        g[7] = g[6];
        g[8] = g[5];
      } else {  // Eqs. 9a-c, rho_w = f1 + f2 + f4 + 2 (f3 + f6 + f7)
        const C rho = (C)1 + (g[0] + g[1] + g[3] + (C)2 * (g[2] + g[5] + g[6]));
        const C d = (C)0.5 * (g[1] - g[3]);
        const C m = (C)0.5 * rho * U;
        g[4] = g[2];
        g[7] = g[5] + d - m;
        g[8] = g[6] - d + m;
      }
    } else if (y == 0) {
      if (p.bc == BC_FREESLIP) {  // Eq. 7b: f3 = f5, f7 = f8, f6 = f9
        g[2] = g[4];
        g[6] = g[7];
        g[5] = g[8];
      } else {  // Eqs. 10a-c, rho_w = f1 + f2 + f4 + 2 (f5 + f8 + f9)
        const C rho = (C)1 + (g[0] + g[1] + g[3] + (C)2 * (g[4] + g[7] + g[8]));
        const C d = (C)0.5 * (g[1] - g[3]);
        const C m = (C)0.5 * rho * U;
        g[2] = g[4];
        g[5] = g[7] - d + m;
        g[6] = g[8] + d - m;
      }
    }
  }
  if (xe == 0) {  // Zou-He velocity inlet (U, 0): unknowns f2, f6, f9
    const C rho = ((C)1 + (g[0] + g[2] + g[4] + (C)2 * (g[3] + g[6] + g[7]))) / ((C)1 - U);
    const C ru = rho * U;
    const C h = (C)0.5 * (g[2] - g[4]);
    g[1] = g[3] + ((C)2 / (C)3) * ru;
    g[5] = g[7] - h + ru / (C)6;
    g[8] = g[6] + h + ru / (C)6;
  }
}

// BGK collision (Eq. 2) towards Eq. 3 with the moments of Eq. 4, on offsets:
// delta_rho = sum g, rho u = sum g c, g_eq = w (delta_rho + rho (3 cu +
// 9/2 cu^2 - 3/2 u.u)), g* = g + omega (g_eq - g).  Returns |u|^2.
template <class C>
__device__ __forceinline__ C collide(C g[9], C omega) {
  const C drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const C rho = (C)1 + drho;
  const C jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const C jy = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]);
  const C inv = (C)1 / rho;
  const C ux = jx * inv, uy = jy * inv;
  const C uu = ux * ux + uy * uy;
  const C base = drho - (C)1.5 * rho * uu;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const C cu = (C)CX(k) * ux + (C)CY(k) * uy;
    const C geq = (C)WD(k) * (base + rho * cu * ((C)3 + (C)4.5 * cu));
    g[k] = g[k] + omega * (geq - g[k]);
  }
  return uu;
}

// Offset part of the Eq. 14 link sum for one node: sum over directions i
// pointing into the solid (bit opp(i) of the link mask) of 2 g*_i c_i.
template <class C>
__device__ __forceinline__ void link_force(const C g[9], uint32_t lm, double &fx, double &fy) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (lm & (1u << OPP(i))) {
      const double v = 2.0 * (double)g[i];
      fx += v * CX(i);
      fy += v * CY(i);
    }
  }
}

// Final fixed-order reduction of the per-item force slots into history entry
// step, executed by one full warp after every item of the step has posted.
__device__ __forceinline__ void finish_force(const StepParams &p, int lane) {
  double sx = 0.0, sy = 0.0;
  for (int s = lane; s < p.nslots; s += 32) {
    const double2 v = __ldcg(p.slots + s);
    sx += v.x;
    sy += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    const unsigned long long n = *p.step;
    const long long r = (long long)(n % (unsigned long long)p.hist_cap);
    p.hist[2 * r] = sx + p.fconst_x;
    p.hist[2 * r + 1] = sy + p.fconst_y;
    *p.step = n + 1;
    *p.done = 0u;
    __threadfence();
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- mbarrier / bulk-async copy (TMA engine) PTX -------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: true when the phase with this parity completed; false after
// ~1 s or as soon as *abort is set (then the caller skips its work).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}
// 1-D bulk copy global -> shared, completion counted on an mbarrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void named_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

}  // namespace gblbm
