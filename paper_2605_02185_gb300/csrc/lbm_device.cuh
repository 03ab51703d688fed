// lbm_device.cuh -- device building blocks of the fused D2Q9 step.
//
// Stored state.  Post-collision populations are kept as offsets from the
// free-stream equilibrium, h_i = f_i - r_i with r_i = f_eq_i(rho = 1,
// u = (U, 0)) of Eq. 3, in the storage type S, in 9 planes [k][ny][pitch].
// Arithmetic is float for float/half/bfloat16 storage and double for double
// storage.  In most of the lattice h is orders of magnitude smaller than f,
// so rounding the stored value and every intermediate costs far less; the
// rules below are the paper's rules rewritten on h (r satisfies each of them
// exactly, so only constant corrections remain where a rule is not symmetric
// in r -- the bounce-back of x-moving populations).
//
// Equilibrium in float.  The weights 1/9, 1/36 and the factors 1/3, 1/12 are
// not representable in binary; multiplying by their float roundings biases
// the momentum of f_eq by ~3e-8 of j at every node and step, a systematic
// forcing that accumulates.  collide() therefore computes the diagonal
// equilibria from Eq. 3, the axis pairs' even parts from Eq. 3, and their odd
// parts and the rest population from exact mass and momentum balance --
// identical in exact arithmetic, conservative to a few unbiased roundings in
// float.
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

// Free-stream reference r_k = f_eq_k(1, (U, 0)) (Eq. 3), host and device.
__host__ __device__ inline double ref_pop(int k, double U) {
  const double cu = CX(k) * U;
  return WD(k) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * U * U);
}

enum { BC_FREESLIP = 0, BC_PERIODIC = 1, BC_ZOUHE = 2, BC_MOVINGWALL = 3 };

// link-map bits: bit k (1..8) = the pull source x - c_k is solid; bit 15 = solid node
constexpr uint32_t LM_SOLID = 1u << 15;
constexpr uint32_t LM_LINKS = 0x1FEu;

// device error word bits
constexpr unsigned ERR_UNSTABLE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;

// ---- storage conversion --------------------------------------------------
// C: arithmetic type of one node; ld2/st2 move the values of two adjacent
// nodes (x even, so the 2-element access is aligned) as one float2 -- for the
// 16-bit types one 32-bit word, converted by packed instructions, rounding
// each half to nearest even exactly as st() does.
template <class S> struct Store;
template <> struct Store<float> {
  using C = float;
  __device__ static __forceinline__ C ld(float v) { return v; }
  __device__ static __forceinline__ float st(C v) { return v; }
  __device__ static __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
  __device__ static __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
// IEEE half holds 2^12 h: the small offsets of the far field (density and
// velocity perturbations of 1e-6 .. 1e-5) then stay clear of the binary16
// subnormal range below 6.1e-5, where the step between values is a fixed
// 6e-8; |h| < 1 keeps 2^12 h far below the binary16 maximum 65504, and
// scaling by a power of two is exact.
constexpr float kHalfScale = 4096.f;
constexpr float kHalfInv = 1.f / 4096.f;
template <> struct Store<__half> {
  using C = float;
  __device__ static __forceinline__ C ld(__half v) { return __fmul_rn(__half2float(v), kHalfInv); }
  __device__ static __forceinline__ __half st(C v) { return __float2half_rn(__fmul_rn(v, kHalfScale)); }
  __device__ static __forceinline__ float2 ld2(const __half *p) {
    return __fmul2_rn(__half22float2(*reinterpret_cast<const __half2 *>(p)), make_float2(kHalfInv, kHalfInv));
  }
  __device__ static __forceinline__ void st2(__half *p, float2 v) {
    const float2 s = __fmul2_rn(v, make_float2(kHalfScale, kHalfScale));
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(s.x, s.y);
  }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  __device__ static __forceinline__ C ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ __nv_bfloat16 st(C v) { return __float2bfloat16_rn(v); }
  __device__ static __forceinline__ float2 ld2(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
  }
  __device__ static __forceinline__ void st2(__nv_bfloat16 *p, float2 v) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
  }
};
template <> struct Store<double> {
  using C = double;
  __device__ static __forceinline__ C ld(double v) { return v; }
  __device__ static __forceinline__ double st(C v) { return v; }
};

// ---- 16-bit storage with stochastic rounding ---------------------------------
// Rounding to nearest loses every update smaller than half a step of the
// 16-bit grid: where the flow changes slowly the stored offsets stop moving
// (stagnation) and the error acts like a steady forcing that can suppress
// vortex shedding.  These forms round up with probability equal to the
// fraction of a step the value lies above the grid point below it, so the
// stored value is right on average and small updates accumulate.  The
// "random" bits come from a hash of the node's nine new values and its
// position (one hash per node, then one multiply per direction), so the
// result is deterministic -- identical in every kernel and launch shape --
// and needs no random-number state: values that change from step to step
// draw new bits each time.
struct half_sr { __half v; };
struct bf16_sr { __nv_bfloat16 v; };

// Per-node seed: the bits of the node's nine post-collision offsets folded
// together with its position, then one xorshift-multiply round (the first
// round of the integer finaliser "lowbias32", C. Wellons, hash-prospector,
// 2018); the per-direction multiply in dither() completes the mix.
__device__ __forceinline__ uint32_t dither_seed(uint32_t fold, int x, int y) {
  uint32_t z = fold ^ ((uint32_t)x * 0x9E3779B1u + (uint32_t)y * 0x85EBCA77u);
  z ^= z >> 16;
  return z * 0x7feb352du;
}
__device__ __forceinline__ uint32_t fold9(const float (&h)[9]) {
  uint32_t f = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) f ^= __float_as_uint(h[k]);
  return f;
}
// Odd multipliers spreading one seed over the nine directions.
__device__ __forceinline__ uint32_t dir_mul(int k) {
  return k == 0 ? 0x2545F491u : k == 1 ? 0x9E3779B9u : k == 2 ? 0x85EBCA6Bu : k == 3 ? 0xC2B2AE35u
       : k == 4 ? 0x27D4EB2Fu : k == 5 ? 0x165667B1u : k == 6 ? 0xD3A2646Du : k == 7 ? 0xFD7046C5u : 0xB55A4F09u;
}
// fp32 bits whose DROP low mantissa bits will be discarded, plus a uniform
// offset in [0, 2^DROP): truncating the result rounds stochastically.
template <int DROP>
__device__ __forceinline__ uint32_t dither(uint32_t bits, uint32_t seed, int k) {
  return bits + ((seed * dir_mul(k)) >> (32 - DROP));
}
// The same for binary16 storage of 2^12 h: the scaling by 2^12 is an add to
// the fp32 exponent field (exact for every normal float; zero and float
// subnormals become values far below the binary16 range, which truncate to
// zero as before).
__device__ __forceinline__ uint32_t dither_half(float v, uint32_t seed, int k) {
  return __float_as_uint(v) + (12u << 23) + ((seed * dir_mul(k)) >> 19);
}
__device__ __forceinline__ uint32_t cvt_rz_half2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

template <> struct Store<half_sr> {
  using C = float;
  __device__ static __forceinline__ C ld(half_sr v) { return __fmul_rn(__half2float(v.v), kHalfInv); }
  __device__ static __forceinline__ half_sr st(C v) { return {__float2half_rn(__fmul_rn(v, kHalfScale))}; }
  __device__ static __forceinline__ half_sr st_at(C v, uint32_t seed, int k) {
    return {__float2half_rz(__uint_as_float(dither_half(v, seed, k)))};
  }
  __device__ static __forceinline__ float2 ld2(const half_sr *p) {
    return __fmul2_rn(__half22float2(*reinterpret_cast<const __half2 *>(p)), make_float2(kHalfInv, kHalfInv));
  }
  __device__ static __forceinline__ void st2_at(half_sr *p, float2 v, uint32_t seed0, uint32_t seed1, int k) {
    *reinterpret_cast<uint32_t *>(p) =
        cvt_rz_half2(__uint_as_float(dither_half(v.x, seed0, k)), __uint_as_float(dither_half(v.y, seed1, k)));
  }
};
template <> struct Store<bf16_sr> {
  using C = float;
  __device__ static __forceinline__ C ld(bf16_sr v) { return __bfloat162float(v.v); }
  __device__ static __forceinline__ bf16_sr st(C v) { return {__float2bfloat16_rn(v)}; }
  __device__ static __forceinline__ bf16_sr st_at(C v, uint32_t seed, int k) {
    const uint32_t b = dither<16>(__float_as_uint(v), seed, k);
    return {__ushort_as_bfloat16((unsigned short)(b >> 16))};
  }
  __device__ static __forceinline__ float2 ld2(const bf16_sr *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
  }
  __device__ static __forceinline__ void st2_at(bf16_sr *p, float2 v, uint32_t seed0, uint32_t seed1, int k) {
    const uint32_t b0 = dither<16>(__float_as_uint(v.x), seed0, k), b1 = dither<16>(__float_as_uint(v.y), seed1, k);
    *reinterpret_cast<uint32_t *>(p) = (b0 >> 16) | (b1 & 0xFFFF0000u);
  }
};

// Read-only cached load of one stored value.
template <class S> __device__ __forceinline__ S ldg_s(const S *p) { return __ldg(p); }
template <> __device__ __forceinline__ half_sr ldg_s(const half_sr *p) {
  return {__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p)))};
}
template <> __device__ __forceinline__ bf16_sr ldg_s(const bf16_sr *p) {
  return {__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p)))};
}

// L2-only load (ld.global.cg) of one stored value: for state written earlier
// in the same launch (the multi-step kernel), where the non-coherent
// read-only cache path must not be used.
template <class S> __device__ __forceinline__ S ldcg_s(const S *p) {
  if constexpr (sizeof(S) == 2) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p));
    S v;
    __builtin_memcpy(&v, &b, 2);
    return v;
  } else {
    return __ldcg(p);
  }
}
// A node's own value of the previous step: a plain load, or (COH) ldcg_s.
template <bool COH, class S> __device__ __forceinline__ S own_ld(const S *p) {
  if constexpr (COH) return ldcg_s(p);
  else return *p;
}

// Whether a storage type rounds stochastically (st_at / st2_at) or to
// nearest (st / st2).
template <class S> struct Dithers { static constexpr bool value = false; };
template <> struct Dithers<half_sr> { static constexpr bool value = true; };
template <> struct Dithers<bf16_sr> { static constexpr bool value = true; };

// ---- per-step parameters (passed by value) -------------------------------
// 16-byte aligned and sized so that the batched kernel can stage a case's
// parameters into shared memory with one bulk copy.
struct alignas(16) StepParams {
  int nx, ny, pitch, bc;
  long long plane;         // elements per population plane
  double omega;            // 1 / tau
  double U;                // inlet / wall speed; also the reference velocity of h
  // link map over the region [lx0, lx0+lw) x [ly0, ly0+lh)
  const uint16_t *lmap;
  const float *qmap;            // interpolated bounce-back fractions [lh][lw][8], or null (half-way)
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
  double fconst_x, fconst_y;    // sum over links of 2 r_i c_i (the reference part of Eq. 14)
  int mrt;                      // 0: BGK (Eq. 2); 1: MRT (Eq. 6)
  double s_e, s_eps, s_q;       // MRT rates of e, epsilon and q (the shear rate is omega)
  // collision constants rounded once on the host (fill_coefs), in the order
  // U, -U^2, omega, 1 - omega, omega/36, omega/9, omega/2, omega/4, s_e/36,
  // s_eps/36, s_q/12: float for the float lanes, double for the double lane
  float kf[11];
  double kd[11];
  // Failure-path controls: the limit of every bounded device wait (ns; 0
  // reads as 1 s) and, for tests of that path only, one row tile whose
  // copies the TMA producer announces but does not issue (-1: none), so the
  // waits on it give up and the step reports ERR_TIMEOUT.
  unsigned long long wait_ns;
  int fault_tile;
};

// omega and 1 - omega rounded as a pair that is exact in T and sums to
// exactly 1 (Sterbenz: x - y is exact for y/2 <= x <= 2y), so the BGK update
// (1 - omega) h + omega h_eq carries mass and momentum over without a
// systematic bias from rounding omega.
template <class T>
__host__ __device__ inline void relaxation_pair(double omega, T &om, T &omc) {
  om = (T)omega;
  if (om >= (T)0.5) {
    omc = (T)1 - om;
  } else {
    omc = (T)(1.0 - omega);
    om = (T)1 - omc;
  }
}

// Fill StepParams::kf / kd from omega, U and the MRT rates (host side, once
// per lattice; the kernels only load them).
__host__ __device__ inline void fill_coefs(StepParams &p) {
  float omf, omcf;
  relaxation_pair<float>(p.omega, omf, omcf);
  double omd, omcd;
  relaxation_pair<double>(p.omega, omd, omcd);
  const double of = omf, ocf = omcf;
  const double vf[11] = {p.U, -p.U * p.U, of, ocf, of / 36.0, of / 9.0, 0.5 * of, 0.25 * of,
                         p.s_e / 36.0, p.s_eps / 36.0, p.s_q / 12.0};
  const double vd[11] = {p.U, -p.U * p.U, omd, omcd, omd / 36.0, omd / 9.0, 0.5 * omd, 0.25 * omd,
                         p.s_e / 36.0, p.s_eps / 36.0, p.s_q / 12.0};
  for (int i = 0; i < 11; ++i) {
    p.kf[i] = (float)vf[i];
    p.kd[i] = vd[i];
  }
}

// One lattice of a batch: its parameters, its two population buffers
// (buf[parity] holds f*(n)) and the index of its first row tile in the
// batch-wide tile numbering.
struct CaseDesc {
  StepParams p;  // first: 16-byte aligned in an array of descriptors
  const void *buf[2];
  long long item0;
};

__device__ __forceinline__ uint32_t link_mask(const StepParams &p, int x, int y) {
  unsigned dx = (unsigned)(x - p.lx0), dy = (unsigned)(y - p.ly0);
  if (dx < (unsigned)p.lw && dy < (unsigned)p.lh) return __ldg(p.lmap + (size_t)dy * p.lw + dx);
  return 0u;
}

// True when no node of [xa, xb] in row y needs a boundary rule, a link-map
// lookup or a bounds check: interior row, no inlet/outlet column, no overlap
// with the link region.  Uniform over a warp's node chunk.
__device__ __forceinline__ bool plain_span(const StepParams &p, int xa, int xb, int y) {
  if (y < 1 || y > p.ny - 2 || xa < 1 || xb > p.nx - 2) return false;
  const bool rows = (unsigned)(y - p.ly0) < (unsigned)p.lh;
  const bool cols = xb >= p.lx0 && xa < p.lx0 + p.lw;
  return !(rows && cols);
}

// Pull (left side of Eq. 2) for the node (xe, y): h[k] = h*_k(xe - c_k).
// A source outside the lattice yields the node's own h*_k (placeholder, later
// overwritten by a boundary rule); a solid source yields the node's own
// f*_opp(k), i.e. h*_opp(k) + r_opp(k) - r_k = h*_opp(k) - 6 w_k c_kx U
// (half-way bounce-back, reflected within the step).  With moving walls
// (Eq. 11, wall velocity (U, 0)) a source above the top row or below the
// bottom row yields f*_opp(k) - 2 w rho (c_opp(k) . u_w) / c_s^2 of the node
// itself, on h: h*_opp(k) + 6 w_k c_kx U (rho - 1) with rho the density of the
// node's f*.  Regular sources come from fetch(k, sx, sy) -- a staged row tile
// or HBM.
//
// With INTERP (the direct kernel of a lattice that has link fractions,
// p.qmap) a solid source instead takes the interpolated bounce-back
// (Bouzidi, Firdaouss and Lallemand, linear) of the link's fraction q:
//   q <  1/2:  2q f*_opp(k)(x) + (1 - 2q) f*_opp(k)(x + c_k),
//   q >= 1/2:  f*_opp(k)(x) / (2q) + (1 - 1/(2q)) f*_k(x),
// and, when fxy is given, adds the link's momentum exchange (the population
// that left along c_opp(k) plus the one that returns) to fxy.
template <class S, class Fetch, bool INTERP = false, bool COH = false>
__device__ __forceinline__ void pull(const S *__restrict__ A, const StepParams &p, int xe, int y, uint32_t lm,
                                     Fetch fetch, typename Store<S>::C h[9], double *fxy = nullptr) {
  using C = typename Store<S>::C;
  const size_t own = (size_t)y * p.pitch + xe;
  const C U = (C)p.U;
  C drho_own = (C)0;
  if (p.bc == BC_MOVINGWALL && (y == 0 || y == p.ny - 1)) {
#pragma unroll
    for (int k = 0; k < 9; ++k) drho_own += Store<S>::ld(own_ld<COH>(A + (size_t)k * p.plane + own));
  }
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
      if (CY(k) != 0 && p.bc == BC_MOVINGWALL && (unsigned)sy >= (unsigned)p.ny)
        h[k] = Store<S>::ld(own_ld<COH>(A + (size_t)OPP(k) * p.plane + own)) + (C)(6.0 * WD(k) * CX(k)) * U * drho_own;
      else
        h[k] = Store<S>::ld(own_ld<COH>(A + (size_t)k * p.plane + own));
    } else if (lm & (1u << k)) {
      const C hi = Store<S>::ld(own_ld<COH>(A + (size_t)OPP(k) * p.plane + own));
      if constexpr (!INTERP) {
        h[k] = hi;
        if (CX(k) != 0) h[k] += (C)(-6.0 * WD(k) * CX(k)) * U;
      } else {
        // the weights of the f-form sum to 1, so on h the reference part
        // r_opp(k) - r_k = -6 w_k c_kx U enters with the weight of f*_opp(k)(x)
        const float q = __ldg(p.qmap + ((size_t)(y - p.ly0) * p.lw + (xe - p.lx0)) * 8 + (k - 1));
        C v, wref;
        if (q < 0.5f) {
          const C hb = fetch(OPP(k), xe + CX(k), y + CY(k));  // the node behind, x + c_k
          v = (C)(2.f * q) * hi + (C)(1.f - 2.f * q) * hb;
          wref = (C)1;
        } else {
          const C a = (C)(0.5f / q);
          v = a * hi + ((C)1 - a) * Store<S>::ld(own_ld<COH>(A + (size_t)k * p.plane + own));
          wref = a;
        }
        if (CX(k) != 0) v += (C)(-6.0 * WD(k) * CX(k)) * U * wref;
        h[k] = v;
        if (fxy) {
          const double m = (double)hi + (double)v;
          fxy[0] += m * CX(OPP(k));
          fxy[1] += m * CY(OPP(k));
        }
      }
    } else {
      h[k] = fetch(k, sx, sy);
    }
  }
}

// Boundary corrections after streaming (Section 2.3), in the order top row,
// bottom row, inlet column.  The outlet (Eq. 13) is realised by computing
// column nx-2 for column nx-1.  On h the free-slip and periodic copies are
// unchanged (r is mirror-symmetric in y); in the Zou-He rules the density
// becomes its deviation from 1, because r satisfies each rule with rho = 1.
template <class C>
__device__ __forceinline__ void boundaries(C h[9], int xe, int y, const StepParams &p) {
  const C U = (C)p.U;
  if (p.bc == BC_FREESLIP || p.bc == BC_ZOUHE) {  // periodic and moving walls: done in pull()
    if (y == p.ny - 1) {
      if (p.bc == BC_FREESLIP) {  // Eq. 7a: f5 = f3, f8 = f7, f9 = f6
        h[4] = h[2];
        h[7] = h[6];
        h[8] = h[5];
      } else {  // Eqs. 9a-c, rho_w = f1 + f2 + f4 + 2 (f3 + f6 + f7)
        const C drho = h[0] + h[1] + h[3] + (C)2 * (h[2] + h[5] + h[6]);
        const C d = (C)0.5 * (h[1] - h[3]);
        const C m = (C)0.5 * drho * U;
        h[4] = h[2];
        h[7] = h[5] + d - m;
        h[8] = h[6] - d + m;
      }
    } else if (y == 0) {
      if (p.bc == BC_FREESLIP) {  // Eq. 7b: f3 = f5, f7 = f8, f6 = f9
        h[2] = h[4];
        h[6] = h[7];
        h[5] = h[8];
      } else {  // Eqs. 10a-c, rho_w = f1 + f2 + f4 + 2 (f5 + f8 + f9)
        const C drho = h[0] + h[1] + h[3] + (C)2 * (h[4] + h[7] + h[8]);
        const C d = (C)0.5 * (h[1] - h[3]);
        const C m = (C)0.5 * drho * U;
        h[2] = h[4];
        h[5] = h[7] - d + m;
        h[6] = h[8] + d - m;
      }
    }
  }
  if (xe == 0) {  // Zou-He velocity inlet (U, 0): unknowns f2, f6, f9
    const C drho = (h[0] + h[2] + h[4] + (C)2 * (h[3] + h[6] + h[7])) / ((C)1 - U);
    const C ru = drho * U;
    const C hh = (C)0.5 * (h[2] - h[4]);
    h[1] = h[3] + ((C)2 / (C)3) * ru;
    h[5] = h[7] - hh + ru / (C)6;
    h[8] = h[6] + hh + ru / (C)6;
  }
}

// ---- lane arithmetic -------------------------------------------------------
// The collisions are written once over a lane type: LF (one node, float),
// LD (one node, double) or LF2 (two nodes in packed FP32 instructions,
// FADD2 / FMUL2 / FFMA2).  Every operator rounds on its own and a
// multiply-add happens only where fma() is written, so each node of an LF2
// lane gets bit for bit what the LF lane computes for it: kernels may treat a
// node alone or in a pair and agree exactly.
struct LF { float v; };
struct LD { double v; };
struct LF2 { float2 v; };
template <class C> struct LaneOf;
template <> struct LaneOf<float> { using T = LF; };
template <> struct LaneOf<double> { using T = LD; };
template <class S> using Lane = typename LaneOf<typename Store<S>::C>::T;

__device__ __forceinline__ LF operator+(LF a, LF b) { return {__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ LF operator-(LF a, LF b) { return {__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ LF operator*(LF a, LF b) { return {__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ LF fma(LF a, LF b, LF c) { return {__fmaf_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ LD operator+(LD a, LD b) { return {__dadd_rn(a.v, b.v)}; }
__device__ __forceinline__ LD operator-(LD a, LD b) { return {__dsub_rn(a.v, b.v)}; }
__device__ __forceinline__ LD operator*(LD a, LD b) { return {__dmul_rn(a.v, b.v)}; }
__device__ __forceinline__ LD fma(LD a, LD b, LD c) { return {__fma_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ LF2 operator+(LF2 a, LF2 b) { return {__fadd2_rn(a.v, b.v)}; }
// a - b as b * (-1) + a: the product is exact, so this is the correctly
// rounded difference, the same bits as __fsub_rn.
__device__ __forceinline__ LF2 operator-(LF2 a, LF2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ LF2 operator*(LF2 a, LF2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ LF2 fma(LF2 a, LF2 b, LF2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

// Negated reciprocal -1/x of a density (close to 1).  Float lanes: the
// hardware estimate y of -1/x refined by one Newton-Raphson step,
// e = 1 + x y, y' = y + y e, whose error is below one ulp; the refinement
// runs in lane arithmetic, so a pair reproduces the single lane.  Double: the
// correctly rounded quotient.  The collisions use -1/x so that no lane
// negation is needed.
__device__ __forceinline__ float rcp_estimate(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ LF neg_recip(LF x) {
  const LF y{rcp_estimate(-x.v)};
  const LF e = fma(x, y, LF{1.f});
  return fma(y, e, y);
}
__device__ __forceinline__ LF2 neg_recip(LF2 x) {
  const LF2 y{make_float2(rcp_estimate(-x.v.x), rcp_estimate(-x.v.y))};
  const LF2 e = fma(x, y, LF2{make_float2(1.f, 1.f)});
  return fma(y, e, y);
}
__device__ __forceinline__ LD neg_recip(LD x) { return {-1.0 / x.v}; }

template <class L> __device__ __forceinline__ L splat(double c);
template <> __device__ __forceinline__ LF splat<LF>(double c) { return {(float)c}; }
template <> __device__ __forceinline__ LD splat<LD>(double c) { return {c}; }
template <> __device__ __forceinline__ LF2 splat<LF2>(double c) { return {make_float2((float)c, (float)c)}; }

// |u|^2 <= 0.09 in every node of the lane (false for NaN).
__device__ __forceinline__ bool speed_ok(LF uu) { return uu.v <= 0.09f; }
__device__ __forceinline__ bool speed_ok(LD uu) { return uu.v <= 0.09; }
__device__ __forceinline__ bool speed_ok(LF2 uu) { return (uu.v.x <= 0.09f) & (uu.v.y <= 0.09f); }

// Per-launch constants of the collision (StepParams::kf / kd, rounded once
// on the host by fill_coefs).
template <class L>
struct Coef {
  L U, nUU;                 // U, -U^2
  L om, omc;                // omega, 1 - omega (exact pair)
  L w36, w9, w2, w4;        // omega/36, omega/9, omega/2, omega/4
  L se36, seps36, sq12;     // MRT: s_e/36, s_eps/36, s_q/12
};
template <class L>
__device__ __forceinline__ L coef_at(const StepParams &p, int i);
template <> __device__ __forceinline__ LF coef_at<LF>(const StepParams &p, int i) { return {p.kf[i]}; }
template <> __device__ __forceinline__ LF2 coef_at<LF2>(const StepParams &p, int i) {
  return {make_float2(p.kf[i], p.kf[i])};
}
template <> __device__ __forceinline__ LD coef_at<LD>(const StepParams &p, int i) { return {p.kd[i]}; }
template <class L>
__device__ __forceinline__ Coef<L> make_coef(const StepParams &p) {
  Coef<L> k;
  k.U = coef_at<L>(p, 0);
  k.nUU = coef_at<L>(p, 1);
  k.om = coef_at<L>(p, 2);
  k.omc = coef_at<L>(p, 3);
  k.w36 = coef_at<L>(p, 4);
  k.w9 = coef_at<L>(p, 5);
  k.w2 = coef_at<L>(p, 6);
  k.w4 = coef_at<L>(p, 7);
  k.se36 = coef_at<L>(p, 8);
  k.seps36 = coef_at<L>(p, 9);
  k.sq12 = coef_at<L>(p, 10);
  return k;
}

// The one-node float constants in both lanes of a pair (the same values
// make_coef<LF2> gives).
__device__ __forceinline__ LF2 widen(LF a) { return {make_float2(a.v, a.v)}; }
__device__ __forceinline__ Coef<LF2> widen(const Coef<LF> &c) {
  Coef<LF2> k;
  k.U = widen(c.U);
  k.nUU = widen(c.nUU);
  k.om = widen(c.om);
  k.omc = widen(c.omc);
  k.w36 = widen(c.w36);
  k.w9 = widen(c.w9);
  k.w2 = widen(c.w2);
  k.w4 = widen(c.w4);
  k.se36 = widen(c.se36);
  k.seps36 = widen(c.seps36);
  k.sq12 = widen(c.sq12);
  return k;
}

// BGK collision (Eq. 2) towards Eq. 3 with the moments of Eq. 4, on h.
// delta_rho = sum h, j = (U, 0) + dj with dj = sum h c, and
//   h_eq_k = w_k [delta_rho + 3 c.dj + (9/2 ((c.dj)(c.j + c.U) - delta_rho (c.U)^2)
//            - 3/2 (dj.(j + U) - delta_rho U^2)) / rho],
// which is f_eq_k(rho, j) - r_k written without cancellation.  Opposite
// diagonals share (c.dj)(c.j + c.U).  The relaxation is
// h* = (1 - omega) h + omega h_eq with omega folded into the equilibrium's
// factors.  Returns |u|^2.
template <class L>
__device__ __forceinline__ L collide(L h[9], const Coef<L> &k) {
  const L drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  const L djx = ((h[1] - h[3]) + (h[5] - h[6])) + (h[8] - h[7]);
  const L djy = ((h[2] - h[4]) + (h[5] - h[8])) + (h[6] - h[7]);
  const L jx = k.U + djx, jxU = jx + k.U;
  const L ninv = neg_recip(splat<L>(1.0) + drho);  // -1/rho
  const L nuu2 = drho * k.nUU;
  const L a = djx * jxU, b = djy * djy;
  const L i45 = ninv * splat<L>(-4.5);
  const L dq = fma((a + b) + nuu2, ninv * splat<L>(1.5), drho);
  const L s5 = djx + djy, s6 = djy - djx, t5 = jxU + djy, t6 = djy - jxU;
  const L A5 = fma(fma(s5, t5, nuu2), i45, dq);
  const L A6 = fma(fma(s6, t6, nuu2), i45, dq);
  L o[9];
  o[5] = fma(splat<L>(3.0), s5, A5) * k.w36;
  o[7] = fma(splat<L>(-3.0), s5, A5) * k.w36;
  o[6] = fma(splat<L>(3.0), s6, A6) * k.w36;
  o[8] = fma(splat<L>(-3.0), s6, A6) * k.w36;
  // Axis pairs: even parts from Eq. 3, odd parts and the rest population
  // from exact momentum and mass balance.
  const L ex = fma(a + nuu2, i45, dq) * k.w9;
  const L ey = fma(b, i45, dq) * k.w9;
  const L ox = fma(splat<L>(-0.5), (o[5] - o[6]) + (o[8] - o[7]), djx * k.w2);
  const L oy = fma(splat<L>(-0.5), (o[5] + o[6]) - (o[7] + o[8]), djy * k.w2);
  o[1] = ex + ox;
  o[3] = ex - ox;
  o[2] = ey + oy;
  o[4] = ey - oy;
  o[0] = drho * k.om - (((o[1] + o[3]) + (o[2] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = fma(k.omc, h[i], o[i]);
  return fma(jx, jx, b) * (ninv * ninv);
}

// MRT collision (Eq. 6) on h.  The moments of h use the integer rows of M;
// the deviations d_k = m_k - m_eq_k of the non-conserved moments are formed
// from small quantities only (Q = |j|^2/rho - U^2 without cancellation); the
// update h* = h - M^T diag(s_k / |row_k|^2) d leaves rho and j untouched
// exactly, because the conserved deviations are zero and M is integer.
// Returns |u|^2.
template <class L>
__device__ __forceinline__ L collide_mrt(L h[9], const Coef<L> &k) {
  const L drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  const L d13 = h[1] - h[3], d24 = h[2] - h[4];
  const L d56 = h[5] - h[6], d87 = h[8] - h[7], d58 = h[5] - h[8], d67 = h[6] - h[7];
  const L djx = (d13 + d56) + d87;
  const L djy = (d24 + d58) + d67;
  const L axis = (h[1] + h[2]) + (h[3] + h[4]);
  const L diag = (h[5] + h[6]) + (h[7] + h[8]);
  const L me = fma(splat<L>(-4.0), h[0], diag + diag) - axis;
  const L meps = fma(splat<L>(4.0), h[0], diag) - (axis + axis);
  const L mqx = fma(splat<L>(-2.0), d13, d56 + d87);
  const L mqy = fma(splat<L>(-2.0), d24, (h[5] + h[6]) - (h[7] + h[8]));
  const L mpxx = (h[1] + h[3]) - (h[2] + h[4]);
  const L mpxy = d56 - d87;
  const L jx = k.U + djx;
  const L ninv = neg_recip(splat<L>(1.0) + drho);  // -1/rho
  const L nuu2 = drho * k.nUU;
  const L a = djx * (jx + k.U), b = djy * djy;
  const L nQ = ((a + b) + nuu2) * ninv;  // -Q
  const L ce = fma(splat<L>(3.0), nQ, fma(splat<L>(2.0), drho, me)) * k.se36;
  const L cps = fma(splat<L>(-3.0), nQ, meps - drho) * k.seps36;
  const L cqx = (mqx + djx) * k.sq12;
  const L cqy = (mqy + djy) * k.sq12;
  const L cxx = fma((a - b) + nuu2, ninv, mpxx) * k.w4;
  const L cxy = fma(jx * djy, ninv, mpxy) * k.w4;
  const L ax = fma(splat<L>(2.0), cps, ce);  // common part of the axis directions
  const L dg = fma(splat<L>(2.0), ce, cps);  // common part of the diagonals
  h[0] = fma(splat<L>(-4.0), cps - ce, h[0]);
  h[1] = h[1] - (fma(splat<L>(-2.0), cqx, cxx) - ax);
  h[2] = h[2] + (fma(splat<L>(2.0), cqy, cxx) + ax);
  h[3] = h[3] - (fma(splat<L>(2.0), cqx, cxx) - ax);
  h[4] = h[4] + (fma(splat<L>(-2.0), cqy, cxx) + ax);
  h[5] = h[5] - (dg + ((cqx + cqy) + cxy));
  h[6] = h[6] - (dg + ((cqy - cqx) - cxy));
  h[7] = h[7] - (dg - ((cqx + cqy) - cxy));
  h[8] = h[8] - (dg + ((cqx - cqy) - cxy));
  return fma(jx, jx, b) * (ninv * ninv);
}

// The collision of model MRT (0: BGK, 1: MRT), a compile-time choice so each
// step kernel carries only its own collision.
template <int MRT, class L>
__device__ __forceinline__ L collide_model(L h[9], const Coef<L> &k) {
  if (MRT) return collide_mrt<L>(h, k);
  return collide<L>(h, k);
}

// h part of the Eq. 14 link sum for one node: sum over directions i pointing
// into the solid (bit opp(i) of the link mask) of 2 h*_i c_i.
template <class C>
__device__ __forceinline__ void link_force(const C h[9], uint32_t lm, double &fx, double &fy) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (lm & (1u << OPP(i))) {
      const double v = 2.0 * (double)h[i];
      fx += v * CX(i);
      fy += v * CY(i);
    }
  }
}

// Final fixed-order reduction of the per-item force slots into history entry
// step, executed by one full warp after every item of the step has posted.
// Sum of one step's force slots over a warp in a fixed order (each lane its
// slots in index order, then a butterfly); the result is in every lane.
__device__ __forceinline__ void slot_sum(const double2 *slots, int nslots, int lane, double &sx, double &sy) {
  sx = 0.0;
  sy = 0.0;
  for (int s = lane; s < nslots; s += 32) {
    const double2 v = __ldcg(slots + s);
    sx += v.x;
    sy += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
}

__device__ __forceinline__ void finish_force(const StepParams &p, int lane) {
  double sx, sy;
  slot_sum(p.slots, p.nslots, lane, sx, sy);
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
// Non-blocking test: true when the phase with this parity has completed.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
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
__device__ __forceinline__ unsigned long long wait_limit(unsigned long long ns) {
  return ns ? ns : 1000000000ull;
}
// Bounded wait: true when the phase with this parity completed; false after
// limit_ns (0: 1 s) or as soon as *abort is set (then the caller skips its
// work).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns(), lim = wait_limit(limit_ns);
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > lim) return false;
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

// ---- multi-step kernel: per-row completion counters ------------------------
// rows_done[y] counts the row tiles of row y that finished a step, over the
// launches since the counters were last cleared: when a launch starts, every
// row stands at base * nseg (base = steps run since then); step s of the
// launch is complete for row y once rows_done[y] reaches (base + s + 1) * nseg.
struct WaveParams {
  unsigned *rows_done;  // [ny]
  unsigned base;        // steps run since the counters were cleared
  int steps;            // steps of this launch
  double2 *slots;       // [steps][nslots] force partial of every force tile and step
};

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_relaxed_gpu_add(unsigned *p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_cta_shared(unsigned *p, unsigned v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta_shared(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
// With relaxed loads before it, an acquire; with relaxed writes after it, a
// release (GPU scope).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// Order the generic-proxy writes made visible by an acquire before the bulk
// copies (async proxy) that read them.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

}  // namespace gblbm
