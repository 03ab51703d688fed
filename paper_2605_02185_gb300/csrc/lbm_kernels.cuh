// lbm_kernels.cuh -- the fused D2Q9 step kernels and their helpers, as
// templates over the population storage type.  Each lbm_k_<type>.cu
// instantiates them for one type and exports a KernelOps table.
#pragma once

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace gblbm {

// One row tile's force partial summed over the group in a fixed order (each
// warp's lanes, then the warps in order); the sum is valid in thread 0.
// Called uniformly by all threads of the group; sync() is the group barrier.
template <int NW, class Sync>
__device__ __forceinline__ double2 tile_force(double fx, double fy, int tid, double (&red)[2][NW], Sync sync) {
  const int warp = tid >> 5, lane = tid & 31;
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  if (lane == 0) {
    red[0][warp] = fx;
    red[1][warp] = fy;
  }
  sync();
  double sx = 0.0, sy = 0.0;
  if (tid == 0) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      sx += red[0][w];
      sy += red[1][w];
    }
  }
  return make_double2(sx, sy);
}

__device__ __forceinline__ int force_slot(const StepParams &p, int y, int s) {
  return (y - p.fy0) * (p.fs1 - p.fs0 + 1) + (s - p.fs0);
}

// Post one row tile's force partial to its slot; the tile that posts last in
// the step reduces all slots (fixed order) into the history.
template <int NW, class Sync>
__device__ __forceinline__ void post_force(const StepParams &p, int y, int s, double fx, double fy, int tid,
                                           double (&red)[2][NW], int &s_last, Sync sync) {
  const int warp = tid >> 5, lane = tid & 31;
  const double2 sum = tile_force<NW>(fx, fy, tid, red, sync);
  if (tid == 0) {
    __stcg(p.slots + force_slot(p, y, s), sum);
    __threadfence();
    const unsigned prev = atomicAdd(p.done, 1u);
    s_last = (prev == (unsigned)(p.nslots - 1)) ? 1 : 0;
    if (s_last) __threadfence();
  }
  sync();
  if (s_last && warp == 0) finish_force(p, lane);
}

__device__ __forceinline__ bool is_force_item(const StepParams &p, int y, int s) {
  return y >= p.fy0 && y <= p.fy1 && s >= p.fs0 && s <= p.fs1;
}

// Collision of one node held in C values (Eq. 2 or Eq. 6); false when the
// node's speed left the stable range.  For the 16-bit storage forms, whose
// plain spans are updated two nodes at a time with packed instructions, a
// single node runs the same packed instructions with itself in both lanes:
// inside the step kernels the packed and the one-lane instruction sequences
// were seen to disagree in the last bit on rare nodes, and running one form
// keeps every kernel and shape bit-identical.
template <int MRT>
__device__ __noinline__ bool collide_node_packed(float (&h)[9], const Coef<LF> &cf) {
  const Coef<LF2> c2 = widen(cf);
  LF2 v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = LF2{make_float2(h[k], h[k])};
  const bool ok = speed_ok(collide_model<MRT, LF2>(v, c2));
#pragma unroll
  for (int k = 0; k < 9; ++k) h[k] = v[k].v.x;
  return ok;
}

template <int MRT, class S>
__device__ __forceinline__ bool collide_node(typename Store<S>::C (&h)[9], const Coef<Lane<S>> &cf) {
  using L = Lane<S>;
  if constexpr (sizeof(S) == 2) {
    return collide_node_packed<MRT>(h, cf);
  } else {
    L v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = L{h[k]};
    const bool ok = speed_ok(collide_model<MRT, L>(v, cf));
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = v[k].v;
    return ok;
  }
}

// One node, general form: pull (with bounce-back and placeholders), boundary
// rules, collision into h; adds the node's links to the force.  With INTERP
// (interpolated bounce-back) the links' momentum exchange is that of the
// previous step, taken while pulling: it needs the returning populations.
template <int MRT, class S, class Fetch, bool INTERP = false, bool COH = false>
__device__ __forceinline__ void node_compute(const S *__restrict__ A, const StepParams &p, int x, int y,
                                             const Coef<Lane<S>> &cf, Fetch fetch, double &fx, double &fy,
                                             bool &bad, typename Store<S>::C (&h)[9]) {
  using C = typename Store<S>::C;
  const int xe = (x == p.nx - 1) ? p.nx - 2 : x;  // Eq. 13: outlet = column nx-2
  const uint32_t lm = link_mask(p, xe, y);
  if (lm & LM_SOLID) {
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = (C)0;
  } else if constexpr (INTERP) {
    double fxy[2] = {0.0, 0.0};
    pull<S, Fetch, true, COH>(A, p, xe, y, lm, fetch, h, x == xe ? fxy : nullptr);
    fx += fxy[0];
    fy += fxy[1];
    boundaries<C>(h, xe, y, p);
    bad |= !collide_node<MRT, S>(h, cf);
  } else {
    pull<S, Fetch, false, COH>(A, p, xe, y, lm, fetch, h);
    boundaries<C>(h, xe, y, p);
    bad |= !collide_node<MRT, S>(h, cf);
    if ((lm & LM_LINKS) && x == xe) link_force<C>(h, lm, fx, fy);
  }
}

// One interior fluid node away from every boundary and link (plain_span):
// every source is regular, no rule applies.
template <int MRT, class S, class Fetch>
__device__ __forceinline__ void plain_compute(const StepParams &p, int x, int y, const Coef<Lane<S>> &cf,
                                              Fetch fetch, bool &bad, typename Store<S>::C (&h)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) h[k] = fetch(k, x - CX(k), y - CY(k));
  bad |= !collide_node<MRT, S>(h, cf);
}

template <class S>
__device__ __forceinline__ void store_node(S *__restrict__ B, const StepParams &p, int x, int y,
                                           const typename Store<S>::C (&h)[9]) {
  S *o = B + (size_t)y * p.pitch + x;
  if constexpr (Dithers<S>::value) {
    const uint32_t seed = dither_seed(fold9(h), x, y);
#pragma unroll
    for (int k = 0; k < 9; ++k) o[(size_t)k * p.plane] = Store<S>::st_at(h[k], seed, k);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) o[(size_t)k * p.plane] = Store<S>::st(h[k]);
  }
}

template <int MRT, class S, class Fetch, bool INTERP = false, bool COH = false>
__device__ __forceinline__ void update_node(const S *__restrict__ A, S *__restrict__ B, const StepParams &p, int x,
                                            int y, const Coef<Lane<S>> &cf, Fetch fetch, double &fx, double &fy,
                                            bool &bad) {
  typename Store<S>::C h[9];
  node_compute<MRT, S, Fetch, INTERP, COH>(A, p, x, y, cf, fetch, fx, fy, bad, h);
  store_node<S>(B, p, x, y, h);
}

template <int MRT, class S, class Fetch>
__device__ __forceinline__ void update_plain(S *__restrict__ B, const StepParams &p, int x, int y,
                                             const Coef<Lane<S>> &cf, Fetch fetch, bool &bad) {
  typename Store<S>::C h[9];
  plain_compute<MRT, S>(p, x, y, cf, fetch, bad, h);
  store_node<S>(B, p, x, y, h);
}

// Two adjacent nodes x, x + 1 of a span that needs the general form (pull
// with bounce-back and placeholders, boundary rules, links): each node is
// pulled on its own, the pair collides in the packed form the plain spans
// use, so a node gets the same bits whichever span it falls in.
template <int MRT, class S, class Fetch, bool COH = false>
__device__ __forceinline__ void update_node_pair(const S *__restrict__ A, S *__restrict__ B, const StepParams &p,
                                                 int x, int y, const Coef<LF2> &cf2, Fetch fetch, double &fx,
                                                 double &fy, bool &bad) {
  float h[2][9];
  uint32_t lm[2];
  int xe[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int xn = x + e;
    xe[e] = (xn == p.nx - 1) ? p.nx - 2 : xn;  // Eq. 13: outlet = column nx-2
    lm[e] = xn < p.nx ? link_mask(p, xe[e], y) : LM_SOLID;
    if (lm[e] & LM_SOLID) {
#pragma unroll
      for (int k = 0; k < 9; ++k) h[e][k] = 0.f;
    } else {
      pull<S, Fetch, false, COH>(A, p, xe[e], y, lm[e], fetch, h[e]);
      boundaries<float>(h[e], xe[e], y, p);
    }
  }
  LF2 v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = LF2{make_float2(h[0][k], h[1][k])};
  const LF2 uu = collide_model<MRT, LF2>(v, cf2);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int xn = x + e;
    if (xn >= p.nx) continue;
    if (!(lm[e] & LM_SOLID)) {
      bad |= !((e ? uu.v.y : uu.v.x) <= 0.09f);
#pragma unroll
      for (int k = 0; k < 9; ++k) h[e][k] = e ? v[k].v.y : v[k].v.x;
      if ((lm[e] & LM_LINKS) && xn == xe[e]) link_force<float>(h[e], lm[e], fx, fy);
    }
    store_node<S>(B, p, xn, y, h[e]);
  }
}

// Two adjacent interior nodes (x even) of a plain span, from a staged row
// tile (tile[k * seg + x'] = h*_k at column x' of row y - c_ky): the
// x-aligned planes are read as one pair, the x-shifted ones per node; the
// collision runs on packed FP32 pairs; each plane is stored as one pair.
template <int MRT, class S>
__device__ __forceinline__ void update_pair(S *__restrict__ B, const StepParams &p, int x, int y,
                                            const Coef<LF2> &cf, const S *__restrict__ tile, int seg, bool &bad) {
  LF2 h[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const S *src = tile + k * seg + (x - CX(k));
    if (CX(k) == 0) h[k] = LF2{Store<S>::ld2(src)};
    else h[k] = LF2{make_float2(Store<S>::ld(src[0]), Store<S>::ld(src[1]))};
  }
  bad |= !speed_ok(collide_model<MRT, LF2>(h, cf));
  S *o = B + (size_t)y * p.pitch + x;
  if constexpr (Dithers<S>::value) {
    uint32_t f0 = 0, f1 = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      f0 ^= __float_as_uint(h[k].v.x);
      f1 ^= __float_as_uint(h[k].v.y);
    }
    const uint32_t s0 = dither_seed(f0, x, y), s1 = dither_seed(f1, x + 1, y);
#pragma unroll
    for (int k = 0; k < 9; ++k) Store<S>::st2_at(o + (size_t)k * p.plane, h[k].v, s0, s1, k);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) Store<S>::st2(o + (size_t)k * p.plane, h[k].v);
  }
}

// ---- direct kernel: one CTA per row tile, loads straight from HBM -------
template <class S, int NT, int MRT>
__global__ void __launch_bounds__(NT) step_direct(const S *__restrict__ A, S *__restrict__ B, StepParams p) {
  using C = typename Store<S>::C;
  __shared__ double red[2][NT / 32];
  __shared__ int s_last;
  const int t = blockIdx.x;
  const int y = t / p.nseg, s = t - y * p.nseg;
  const int x0 = s * p.seg;
  const int x1 = min(x0 + p.seg, p.nx);
  const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
  double fx = 0.0, fy = 0.0;
  bool bad = false;
  auto fetch = [&](int k, int sx, int sy) -> C {
    return Store<S>::ld(ldg_s(A + (size_t)k * p.plane + (size_t)sy * p.pitch + sx));
  };
  for (int xw = x0 + (int)(threadIdx.x & ~31u); xw < x1; xw += NT) {
    const int x = xw + (int)(threadIdx.x & 31u);
    if (plain_span(p, xw, xw + 31, y)) {
      update_plain<MRT, S>(B, p, x, y, cf, fetch, bad);
    } else if (x < x1) {
      if (p.qmap)  // interpolated bounce-back is served by this kernel only
        update_node<MRT, S, decltype(fetch), true>(A, B, p, x, y, cf, fetch, fx, fy, bad);
      else
        update_node<MRT, S>(A, B, p, x, y, cf, fetch, fx, fy, bad);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(p.err, ERR_UNSTABLE);
  if (is_force_item(p, y, s))
    post_force<NT / 32>(p, y, s, fx, fy, (int)threadIdx.x, red, s_last, [] { __syncthreads(); });
}

// Nodes per thread and chunk in the plain spans of the TMA kernel: pairs of
// adjacent nodes for the 16-bit storage forms (one 32-bit load and store per
// aligned plane and pair, packed FP32 arithmetic), single nodes otherwise.
template <class S> struct TmaPair { static constexpr int nodes = sizeof(S) == 2 ? 2 : 1; };

// ---- TMA-staged persistent kernel ----------------------------------------
// CTA = NCW compute warps + 1 producer warp.  The producer's elected lane
// walks the CTA's row tiles (grid-stride) and, per tile, issues nine 1-D bulk
// async copies -- for plane k the row y - c_ky, columns [x0 - H, x0 + W + H)
// -- into a STAGES-deep ring of shared-memory tiles, signalling an mbarrier
// with the byte count.  Compute warps wait on it, pull from shared memory
// (any x shift, no bank conflicts: consecutive lanes read consecutive
// elements), apply the boundary rules, collide and store straight to HBM
// with coalesced stores, then release the stage.  Every wait is bounded.
// INTERP: general nodes take the interpolated bounce-back of pull(); the one
// extra population it needs from a neighbour, f*_opp(k)(x + c_k), lies in the
// staged row of plane opp(k), the others are the node's own (read from A).
template <class S, int NCW, int CPT, int STAGES, int MRT, bool INTERP = false>
__global__ void __launch_bounds__((NCW + 1) * 32) step_tma(const S *__restrict__ A, S *__restrict__ B, StepParams p) {
  using C = typename Store<S>::C;
  constexpr int PX = TmaPair<S>::nodes;  // adjacent nodes per thread and chunk
  constexpr int H = 16 / (int)sizeof(S);
  constexpr int NC = NCW * 32;
  constexpr int W = NC * CPT * PX;
  constexpr int SEG = W + 2 * H;
  extern __shared__ __align__(128) unsigned char smem[];
  S *tiles = reinterpret_cast<S *>(smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * 9 * SEG * sizeof(S));
  __shared__ double red[2][NCW];
  __shared__ int s_last;
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = p.ny * p.nseg;
  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(smem_addr(&bars[q]), 1);
      mbar_init(smem_addr(&bars[STAGES + q]), NCW);
    }
    *s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NCW) {  // ---------------- producer
    if (lane == 0) {
      int j = 0;
      for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
        const int st = j % STAGES;
        if (j >= STAGES && !mbar_wait_bounded(smem_addr(&bars[STAGES + st]), ((j / STAGES) - 1) & 1, s_abort, p.wait_ns)) {
          if (!*s_abort) atomicOr(p.err, ERR_TIMEOUT);
          *s_abort = 1;
          break;
        }
        if (*s_abort) break;
        const int y = t / p.nseg, s = t - y * p.nseg;
        const int x0 = s * W;
        const int xs = max(x0 - H, 0), xl = min(x0 + W + H, p.pitch);
        const uint32_t bytes = (uint32_t)(xl - xs) * (uint32_t)sizeof(S);
        int rows[9];
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          int sy = y - CY(k);
          if (p.bc == BC_PERIODIC) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
          rows[k] = ((unsigned)sy < (unsigned)p.ny) ? sy : -1;
          total += rows[k] >= 0 ? bytes : 0u;
        }
        const uint32_t fb = smem_addr(&bars[st]);
        mbar_arrive_expect_tx(fb, total);
        if (t == p.fault_tile) continue;  // failure-path test: announced, never copied
        S *dst = tiles + (size_t)st * 9 * SEG + (xs - (x0 - H));
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (rows[k] >= 0)
            bulk_g2s(smem_addr(dst + (size_t)k * SEG), A + (size_t)k * p.plane + (size_t)rows[k] * p.pitch + xs, bytes,
                     fb);
      }
      // Do not leave while a copy into this CTA's shared memory is in flight.
      for (int q = max(0, j - STAGES); q < j; ++q) {
        const uint32_t fb = smem_addr(&bars[q % STAGES]);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(fb, (q / STAGES) & 1)) {
          if (global_ns() - t0 > wait_limit(p.wait_ns)) {
            atomicOr(p.err, ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    return;
  }

  // ---------------------------------------- compute warps
  const int ctid = threadIdx.x;
  const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
  const Coef<LF2> cf2 = make_coef<LF2>(p);
  bool bad = false;
  int j = 0;
  for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
    const int st = j % STAGES;
    bool ok = false;
    if (!*s_abort) {
      ok = mbar_wait_bounded(smem_addr(&bars[st]), (j / STAGES) & 1, s_abort, p.wait_ns);
      if (!ok && !*s_abort) {
        atomicOr(p.err, ERR_TIMEOUT);
        *s_abort = 1;
      }
    }
    const int y = t / p.nseg, s = t - y * p.nseg;
    const int x0 = s * W;
    double fx = 0.0, fy = 0.0;
    if (ok) {
      const S *tile = tiles + (size_t)st * 9 * SEG + (H - x0);
      auto fetch = [&](int k, int sx, int) -> C { return Store<S>::ld(tile[k * SEG + sx]); };
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int xw = x0 + (c * NC + (ctid & ~31)) * PX;
        if constexpr (PX == 2) {
          const int x = xw + 2 * lane;
          if (plain_span(p, xw, xw + 63, y))
            update_pair<MRT, S>(B, p, x, y, cf2, tile, SEG, bad);
          else if (x < p.nx)
            update_node_pair<MRT, S>(A, B, p, x, y, cf2, fetch, fx, fy, bad);
        } else {
          const int x = xw + lane;
          if (plain_span(p, xw, xw + 31, y))
            update_plain<MRT, S>(B, p, x, y, cf, fetch, bad);
          else if (x < p.nx)
            update_node<MRT, S, decltype(fetch), INTERP>(A, B, p, x, y, cf, fetch, fx, fy, bad);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&bars[STAGES + st]));
    }
    if (is_force_item(p, y, s)) post_force<NCW>(p, y, s, fx, fy, ctid, red, s_last, [] { named_bar(1, NC); });
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, ERR_UNSTABLE);
}

// ---- multi-step TMA kernel ------------------------------------------------
// The TMA kernel above run for w.steps steps in one cooperative launch, with
// the same grid-stride order of row tiles in every step (so the work of the
// boundary rows and of the body is spread over all CTAs as in step_tma).
// The launch boundary between steps is replaced by per-row completion
// counters: the producer loads a tile of row y for step s only after every
// tile of rows y - 1, y, y + 1 has finished step s - 1 (they wrote the rows
// it pulls, and have read the rows it will overwrite).  A CTA can therefore
// start the next step's first rows while other CTAs finish the last rows of
// the step before: no pipeline fill and no tail per step.
// CTA = NCW compute warps, the producer warp, and a publisher warp.  The
// producer sees a tile finished on its stage's "empty" mbarrier (all compute
// warps done with it) -- when it reuses the stage, and by polling the stages
// in flight while it waits on a counter -- and advances a shared-memory count
// of finished tiles (release, CTA scope).  The publisher follows that count
// and adds each finished tile to its row's counter, a batch of tiles per
// GPU-scope fence, off the producer's path.  A producer waiting on a counter
// keeps reporting its finished tiles, so no CTA waits on a completion that
// another wait holds back.  The producer checks the rows of the next WAVE_AHEAD tiles with
// one round of independent loads.
// Per node the arithmetic is that of step_tma, so the results are the same
// bits; the node's own previous values are read through L2 (they were
// written earlier in the launch), and each step's force partials go to a slot
// row of their own, reduced in step order by wave_finish after the launch.
constexpr int WAVE_AHEAD = 8;

// Rows a tile of row y pulls from: y - 1 .. y + 1, wrapped (periodic) or
// clipped to the lattice.
__device__ __forceinline__ void wave_rows(const StepParams &p, int y, int (&r)[3], int &n) {
  n = 0;
  for (int d = -1; d <= 1; ++d) {
    int yy = y + d;
    if (p.bc == BC_PERIODIC) yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
    else if (yy < 0 || yy >= p.ny) continue;
    r[n++] = yy;
  }
}

template <class S, int NCW, int CPT, int STAGES, int MRT>
__global__ void __launch_bounds__((NCW + 2) * 32)
    step_tma_wave(S *buf0, S *buf1, StepParams p, WaveParams w) {
  using C = typename Store<S>::C;
  constexpr int PX = TmaPair<S>::nodes;
  constexpr int H = 16 / (int)sizeof(S);
  constexpr int NC = NCW * 32;
  constexpr int W = NC * CPT * PX;
  constexpr int SEG = W + 2 * H;
  extern __shared__ __align__(128) unsigned char smem[];
  S *tiles = reinterpret_cast<S *>(smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * 9 * SEG * sizeof(S));
  __shared__ unsigned s_finished;  // producer -> publisher: tiles [0, s_finished) finished
  __shared__ double red[2][NCW];
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = p.ny * p.nseg;
  const int G = gridDim.x;
  const int per_step = (nitems - (int)blockIdx.x + G - 1) / G;  // tiles of this CTA in a step (G <= nitems)
  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(smem_addr(&bars[q]), 1);
      mbar_init(smem_addr(&bars[STAGES + q]), NCW);
    }
    s_finished = 0;
    *s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NCW + 1) {  // ---------------- publisher
    if (lane == 0) {
      const unsigned total = (unsigned)per_step * (unsigned)w.steps;
      unsigned q = 0;
      int kk = 0;  // in-step index of tile q
      unsigned long long t0 = global_ns();
      const unsigned long long lim = wait_limit(p.wait_ns);
      while (q < total && !*s_abort) {
        const unsigned c = ld_acquire_cta_shared(&s_finished);
        if (c == q) {
          if (global_ns() - t0 > lim) {
            atomicOr(p.err, ERR_TIMEOUT);
            *s_abort = 1;
            break;
          }
          __nanosleep(64);
          continue;
        }
        fence_acq_rel_gpu();
        for (; q < c; ++q) {
          red_relaxed_gpu_add(w.rows_done + ((int)blockIdx.x + kk * G) / p.nseg, 1u);
          if (++kk == per_step) kk = 0;
        }
        t0 = global_ns();
      }
    }
    return;
  }

  if (warp == NCW) {  // ---------------- producer
    if (lane == 0) {
      int j = 0;     // tiles issued (all steps of this launch)
      int fin = 0;   // tiles [0, fin) finished and reported
      // report the finished prefix of the tiles in flight (non-blocking);
      // a stage is reused only after its tile finished, so each parity test
      // refers to the tile in flight on it
      auto collect = [&]() {
        const int f0 = fin;
        while (fin < j && mbar_test_wait(smem_addr(&bars[STAGES + fin % STAGES]), (fin / STAGES) & 1)) ++fin;
        if (fin != f0) st_release_cta_shared(&s_finished, (unsigned)fin);
      };
      bool stop = false;
      for (int s = 0; s < w.steps && !stop; ++s) {
        const S *A = (s & 1) ? buf1 : buf0;
        const unsigned need = (w.base + (unsigned)s) * (unsigned)p.nseg;  // step s - 1 done
        int ver = s > 0 ? 0 : per_step;  // in-step tiles [0, ver) have their rows checked
        int k = 0;
        for (int t = blockIdx.x; t < nitems; t += G, ++j, ++k) {
          const int st = j % STAGES;
          if (j >= STAGES) {
            if (fin <= j - STAGES &&
                !mbar_wait_bounded(smem_addr(&bars[STAGES + st]), ((j / STAGES) - 1) & 1, s_abort, p.wait_ns)) {
              if (!*s_abort) atomicOr(p.err, ERR_TIMEOUT);
              *s_abort = 1;
              stop = true;
              break;
            }
            collect();
          }
          if (*s_abort) {
            stop = true;
            break;
          }
          if (k >= ver) {  // rows of tiles k .. k + WAVE_AHEAD - 1 of step s - 1
            const unsigned long long t0 = global_ns(), lim = wait_limit(p.wait_ns);
            while (true) {
              unsigned v[WAVE_AHEAD][3];
              int nr[WAVE_AHEAD];
#pragma unroll
              for (int i = 0; i < WAVE_AHEAD; ++i) {
                int r[3];
                nr[i] = 0;
                if (k + i < per_step) wave_rows(p, (t + i * G) / p.nseg, r, nr[i]);
#pragma unroll
                for (int e = 0; e < 3; ++e) v[i][e] = e < nr[i] ? ld_relaxed_gpu(w.rows_done + r[e]) : need;
              }
              int m = 0;
              while (m < WAVE_AHEAD && k + m < per_step && (int)(v[m][0] - need) >= 0 && (int)(v[m][1] - need) >= 0 &&
                     (int)(v[m][2] - need) >= 0)
                ++m;
              if (m > 0) {
                ver = k + m;
                break;
              }
              collect();
              if ((*(volatile const unsigned *)p.err & ERR_TIMEOUT) || global_ns() - t0 > lim) break;
            }
            if (k >= ver) {
              atomicOr(p.err, ERR_TIMEOUT);
              *s_abort = 1;
              stop = true;
              break;
            }
            fence_acq_rel_gpu();  // the loads above become an acquire
            fence_proxy_async_global();
          }
          const int y = t / p.nseg, sg = t - y * p.nseg;
          const int x0 = sg * W;
          const int xs = max(x0 - H, 0), xl = min(x0 + W + H, p.pitch);
          const uint32_t bytes = (uint32_t)(xl - xs) * (uint32_t)sizeof(S);
          int rows[9];
          uint32_t total = 0;
#pragma unroll
          for (int kk = 0; kk < 9; ++kk) {
            int sy = y - CY(kk);
            if (p.bc == BC_PERIODIC) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
            rows[kk] = ((unsigned)sy < (unsigned)p.ny) ? sy : -1;
            total += rows[kk] >= 0 ? bytes : 0u;
          }
          const uint32_t fb = smem_addr(&bars[st]);
          mbar_arrive_expect_tx(fb, total);
          if (t == p.fault_tile) continue;  // failure-path test: announced, never copied
          S *dst = tiles + (size_t)st * 9 * SEG + (xs - (x0 - H));
#pragma unroll
          for (int kk = 0; kk < 9; ++kk)
            if (rows[kk] >= 0)
              bulk_g2s(smem_addr(dst + (size_t)kk * SEG), A + (size_t)kk * p.plane + (size_t)rows[kk] * p.pitch + xs,
                       bytes, fb);
        }
      }
      // Report the last tiles, and do not leave while a copy into this CTA's
      // shared memory is in flight (bounded waits).
      const unsigned long long t0 = global_ns(), lim = wait_limit(p.wait_ns);
      while (fin < j && !*s_abort && global_ns() - t0 <= lim) collect();
      for (int q = max(0, j - STAGES); q < j; ++q) {
        const uint32_t fb = smem_addr(&bars[q % STAGES]);
        while (!mbar_try_wait(fb, (q / STAGES) & 1)) {
          if (global_ns() - t0 > lim) {
            atomicOr(p.err, ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    return;
  }

  // ---------------------------------------- compute warps
  const int ctid = threadIdx.x;
  const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
  const Coef<LF2> cf2 = make_coef<LF2>(p);
  bool bad = false;
  int j = 0;
  for (int s = 0; s < w.steps; ++s) {
    const S *A = (s & 1) ? buf1 : buf0;
    S *B = (s & 1) ? buf0 : buf1;
    double2 *slots = w.slots + (size_t)s * p.nslots;
    for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
      const int st = j % STAGES;
      bool ok = false;
      if (!*s_abort) {
        ok = mbar_wait_bounded(smem_addr(&bars[st]), (j / STAGES) & 1, s_abort, p.wait_ns);
        if (!ok && !*s_abort) {
          atomicOr(p.err, ERR_TIMEOUT);
          *s_abort = 1;
        }
      }
      const int y = t / p.nseg, sg = t - y * p.nseg;
      const int x0 = sg * W;
      double fx = 0.0, fy = 0.0;
      if (ok) {
        const S *tile = tiles + (size_t)st * 9 * SEG + (H - x0);
        auto fetch = [&](int k, int sx, int) -> C { return Store<S>::ld(tile[k * SEG + sx]); };
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int xw = x0 + (c * NC + (ctid & ~31)) * PX;
          if constexpr (PX == 2) {
            const int x = xw + 2 * lane;
            if (plain_span(p, xw, xw + 63, y))
              update_pair<MRT, S>(B, p, x, y, cf2, tile, SEG, bad);
            else if (x < p.nx)
              update_node_pair<MRT, S, decltype(fetch), true>(A, B, p, x, y, cf2, fetch, fx, fy, bad);
          } else {
            const int x = xw + lane;
            if (plain_span(p, xw, xw + 31, y))
              update_plain<MRT, S>(B, p, x, y, cf, fetch, bad);
            else if (x < p.nx)
              update_node<MRT, S, decltype(fetch), false, true>(A, B, p, x, y, cf, fetch, fx, fy, bad);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bars[STAGES + st]));
      }
      if (is_force_item(p, y, sg)) {
        const double2 sum = tile_force<NCW>(fx, fy, ctid, red, [] { named_bar(1, NC); });
        if (ctid == 0) __stcg(slots + force_slot(p, y, sg), sum);
        named_bar(1, NC);
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, ERR_UNSTABLE);
}

// History entries of a multi-step launch: each step's slots reduced as
// finish_force reduces them, written in step order.
template <class S>
__global__ void __launch_bounds__(1024) wave_finish(StepParams p, WaveParams w) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long n0 = *p.step;
  for (int s = warp; s < w.steps; s += 32) {
    double sx, sy;
    slot_sum(w.slots + (size_t)s * p.nslots, p.nslots, lane, sx, sy);
    if (lane == 0) {
      const long long r = (long long)((n0 + (unsigned long long)s) % (unsigned long long)p.hist_cap);
      p.hist[2 * r] = sx + p.fconst_x;
      p.hist[2 * r + 1] = sy + p.fconst_y;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *p.step = n0 + (unsigned long long)w.steps;
}

// Case of batch-wide row tile t: the last case whose first tile is <= t.
__device__ __forceinline__ int case_of(const CaseDesc *__restrict__ cases, int ncases, long long t) {
  int lo = 0, hi = ncases - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&cases[mid].item0) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---- batched direct kernel: one CTA per row tile of any case ------------
template <class S, int NT, int MRT>
__global__ void __launch_bounds__(NT) step_direct_batch(const CaseDesc *__restrict__ cases, int ncases, int parity) {
  using C = typename Store<S>::C;
  __shared__ double red[2][NT / 32];
  __shared__ int s_last;
  const int c = case_of(cases, ncases, blockIdx.x);
  const StepParams &p = cases[c].p;
  const S *__restrict__ A = (const S *)cases[c].buf[parity];
  S *__restrict__ B = (S *)cases[c].buf[parity ^ 1];
  const int t = (int)(blockIdx.x - cases[c].item0);
  const int y = t / p.nseg, s = t - y * p.nseg;
  const int x0 = s * p.seg;
  const int x1 = min(x0 + p.seg, p.nx);
  const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
  double fx = 0.0, fy = 0.0;
  bool bad = false;
  auto fetch = [&](int k, int sx, int sy) -> C {
    return Store<S>::ld(ldg_s(A + (size_t)k * p.plane + (size_t)sy * p.pitch + sx));
  };
  for (int xw = x0 + (int)(threadIdx.x & ~31u); xw < x1; xw += NT) {
    const int x = xw + (int)(threadIdx.x & 31u);
    if (plain_span(p, xw, xw + 31, y))
      update_plain<MRT, S>(B, p, x, y, cf, fetch, bad);
    else if (x < x1)
      update_node<MRT, S>(A, B, p, x, y, cf, fetch, fx, fy, bad);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(p.err, ERR_UNSTABLE);
  if (is_force_item(p, y, s))
    post_force<NT / 32>(p, y, s, fx, fy, (int)threadIdx.x, red, s_last, [] { __syncthreads(); });
}

// ---- batched TMA kernel ---------------------------------------------------
// The single-lattice pipeline over the concatenated row tiles of all cases:
// the producer finds the case of each tile, stages its rows and the case's
// descriptor (step parameters and buffers: one more bulk copy, into the
// stage's descriptor slot) and
// passes (case, row, tile) to the compute warps through a shared-memory slot
// of the stage, all published by the same mbarrier that counts the copied
// bytes.  The compute warps read the parameters from shared memory, not from
// the descriptor array in global memory, and release the stage only when
// they no longer need them.
template <class S, int NCW, int CPT, int STAGES, int MRT>
__global__ void __launch_bounds__((NCW + 1) * 32)
    step_tma_batch(const CaseDesc *__restrict__ cases, int ncases, long long nitems, int parity) {
  using C = typename Store<S>::C;
  constexpr int PX = TmaPair<S>::nodes;
  constexpr int H = 16 / (int)sizeof(S);
  constexpr int NC = NCW * 32;
  constexpr int W = NC * CPT * PX;
  constexpr int SEG = W + 2 * H;
  extern __shared__ __align__(128) unsigned char smem[];
  S *tiles = reinterpret_cast<S *>(smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * 9 * SEG * sizeof(S));
  __shared__ int4 info[STAGES];
  __shared__ CaseDesc sp[STAGES];
  __shared__ double red[2][NCW];
  __shared__ int s_last;
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;
  static_assert(sizeof(CaseDesc) % 16 == 0, "bulk copy of a case descriptor");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(smem_addr(&bars[q]), 1);
      mbar_init(smem_addr(&bars[STAGES + q]), NCW);
    }
    *s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NCW) {  // ---------------- producer
    if (lane == 0) {
      int j = 0;
      for (long long t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
        const int st = j % STAGES;
        if (j >= STAGES && !mbar_wait_bounded(smem_addr(&bars[STAGES + st]), ((j / STAGES) - 1) & 1, s_abort, cases[0].p.wait_ns)) {
          if (!*s_abort) atomicOr(cases[0].p.err, ERR_TIMEOUT);
          *s_abort = 1;
          break;
        }
        if (*s_abort) break;
        const int c = case_of(cases, ncases, t);
        const StepParams &p = cases[c].p;
        const S *A = (const S *)cases[c].buf[parity];
        const int tl = (int)(t - cases[c].item0);
        const int y = tl / p.nseg, s = tl - y * p.nseg;
        const int x0 = s * W;
        const int xs = max(x0 - H, 0), xl = min(x0 + W + H, p.pitch);
        const uint32_t bytes = (uint32_t)(xl - xs) * (uint32_t)sizeof(S);
        int rows[9];
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          int sy = y - CY(k);
          if (p.bc == BC_PERIODIC) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
          rows[k] = ((unsigned)sy < (unsigned)p.ny) ? sy : -1;
          total += rows[k] >= 0 ? bytes : 0u;
        }
        info[st] = make_int4(c, y, s, 0);
        const uint32_t fb = smem_addr(&bars[st]);
        mbar_arrive_expect_tx(fb, total + (uint32_t)sizeof(CaseDesc));
        if (tl == p.fault_tile) continue;  // failure-path test: announced, never copied
        bulk_g2s(smem_addr(&sp[st]), &cases[c], (uint32_t)sizeof(CaseDesc), fb);
        S *dst = tiles + (size_t)st * 9 * SEG + (xs - (x0 - H));
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (rows[k] >= 0)
            bulk_g2s(smem_addr(dst + (size_t)k * SEG), A + (size_t)k * p.plane + (size_t)rows[k] * p.pitch + xs, bytes,
                     fb);
      }
      for (int q = max(0, j - STAGES); q < j; ++q) {
        const uint32_t fb = smem_addr(&bars[q % STAGES]);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(fb, (q / STAGES) & 1)) {
          if (global_ns() - t0 > wait_limit(cases[0].p.wait_ns)) {
            atomicOr(cases[0].p.err, ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    return;
  }

  // ---------------------------------------- compute warps
  const int ctid = threadIdx.x;
  int j = 0;
  for (long long t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
    const int st = j % STAGES;
    bool ok = false;
    if (!*s_abort) {
      ok = mbar_wait_bounded(smem_addr(&bars[st]), (j / STAGES) & 1, s_abort, cases[0].p.wait_ns);
      if (!ok && !*s_abort) {
        atomicOr(cases[0].p.err, ERR_TIMEOUT);
        *s_abort = 1;
      }
    }
    // the tile's case and row: from the stage slot, or (after an abort)
    // recomputed so the force bookkeeping below stays uniform
    int c, y, s;
    if (ok) {
      const int4 in = info[st];
      c = in.x;
      y = in.y;
      s = in.z;
    } else {
      c = case_of(cases, ncases, t);
      const int tl = (int)(t - cases[c].item0);
      y = tl / cases[c].p.nseg;
      s = tl - y * cases[c].p.nseg;
    }
    const int x0 = s * W;
    if (ok) {
      const StepParams &p = sp[st].p;
      const S *__restrict__ A = (const S *)sp[st].buf[parity];
      S *__restrict__ B = (S *)sp[st].buf[parity ^ 1];
      const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
      double fx = 0.0, fy = 0.0;
      bool bad = false;
      const S *tile = tiles + (size_t)st * 9 * SEG + (H - x0);
      auto fetch = [&](int k, int sx, int) -> C { return Store<S>::ld(tile[k * SEG + sx]); };
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) {
        const int xw = x0 + (cc * NC + (ctid & ~31)) * PX;
        if constexpr (PX == 2) {
          const int x = xw + 2 * lane;
          const Coef<LF2> cf2 = widen(cf);
          if (plain_span(p, xw, xw + 63, y))
            update_pair<MRT, S>(B, p, x, y, cf2, tile, SEG, bad);
          else if (x < p.nx)
            update_node_pair<MRT, S>(A, B, p, x, y, cf2, fetch, fx, fy, bad);
        } else {
          const int x = xw + lane;
          if (plain_span(p, xw, xw + 31, y))
            update_plain<MRT, S>(B, p, x, y, cf, fetch, bad);
          else if (x < p.nx)
            update_node<MRT, S>(A, B, p, x, y, cf, fetch, fx, fy, bad);
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, ERR_UNSTABLE);
      if (is_force_item(p, y, s)) post_force<NCW>(p, y, s, fx, fy, ctid, red, s_last, [] { named_bar(1, NC); });
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&bars[STAGES + st]));  // the stage, parameters included, is free
    } else {
      const StepParams &p = cases[c].p;
      if (is_force_item(p, y, s)) post_force<NCW>(p, y, s, 0.0, 0.0, ctid, red, s_last, [] { named_bar(1, NC); });
    }
  }
}

// ---- TMA loads + TMA bulk stores ----------------------------------------
// The single-lattice pipeline of step_tma, but the compute warps write the
// new f* of a row tile into a shared-memory output tile (two, alternating)
// and one thread stores each of its nine plane rows with a bulk async copy
// (cp.async.bulk global <- shared).  A node then costs nine shared-memory
// stores instead of nine global stores with their 64-bit address arithmetic,
// which matters where the step is issue-bound (16-bit storage, MRT).
template <class S, int NCW, int CPT, int STAGES>
constexpr size_t tma_bulk_smem_bytes() {
  return ((size_t)STAGES * 9 * (NCW * 32 * CPT + 2 * (16 / sizeof(S))) * sizeof(S) + 2 * STAGES * sizeof(uint64_t) +
          15) / 16 * 16 +
         (size_t)2 * 9 * NCW * 32 * CPT * sizeof(S);
}

__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <class S, int NCW, int CPT, int STAGES, int MRT>
__global__ void __launch_bounds__((NCW + 1) * 32)
    step_tma_bulk(const S *__restrict__ A, S *__restrict__ B, StepParams p) {
  using C = typename Store<S>::C;
  constexpr int H = 16 / (int)sizeof(S);
  constexpr int NC = NCW * 32;
  constexpr int W = NC * CPT;
  constexpr int SEG = W + 2 * H;
  extern __shared__ __align__(128) unsigned char smem[];
  S *tiles = reinterpret_cast<S *>(smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * 9 * SEG * sizeof(S));
  S *outs = reinterpret_cast<S *>(
      smem + (((size_t)STAGES * 9 * SEG * sizeof(S) + 2 * STAGES * sizeof(uint64_t) + 15) / 16 * 16));
  __shared__ double red[2][NCW];
  __shared__ int s_last;
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = p.ny * p.nseg;
  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(smem_addr(&bars[q]), 1);
      mbar_init(smem_addr(&bars[STAGES + q]), NCW);
    }
    *s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NCW) {  // ---------------- producer (as in step_tma)
    if (lane == 0) {
      int j = 0;
      for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
        const int st = j % STAGES;
        if (j >= STAGES && !mbar_wait_bounded(smem_addr(&bars[STAGES + st]), ((j / STAGES) - 1) & 1, s_abort, p.wait_ns)) {
          if (!*s_abort) atomicOr(p.err, ERR_TIMEOUT);
          *s_abort = 1;
          break;
        }
        if (*s_abort) break;
        const int y = t / p.nseg, s = t - y * p.nseg;
        const int x0 = s * W;
        const int xs = max(x0 - H, 0), xl = min(x0 + W + H, p.pitch);
        const uint32_t bytes = (uint32_t)(xl - xs) * (uint32_t)sizeof(S);
        int rows[9];
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          int sy = y - CY(k);
          if (p.bc == BC_PERIODIC) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
          rows[k] = ((unsigned)sy < (unsigned)p.ny) ? sy : -1;
          total += rows[k] >= 0 ? bytes : 0u;
        }
        const uint32_t fb = smem_addr(&bars[st]);
        mbar_arrive_expect_tx(fb, total);
        if (t == p.fault_tile) continue;  // failure-path test: announced, never copied
        S *dst = tiles + (size_t)st * 9 * SEG + (xs - (x0 - H));
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (rows[k] >= 0)
            bulk_g2s(smem_addr(dst + (size_t)k * SEG), A + (size_t)k * p.plane + (size_t)rows[k] * p.pitch + xs, bytes,
                     fb);
      }
      for (int q = max(0, j - STAGES); q < j; ++q) {
        const uint32_t fb = smem_addr(&bars[q % STAGES]);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(fb, (q / STAGES) & 1)) {
          if (global_ns() - t0 > wait_limit(p.wait_ns)) {
            atomicOr(p.err, ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    return;
  }

  // ---------------------------------------- compute warps
  const int ctid = threadIdx.x;
  const Coef<Lane<S>> cf = make_coef<Lane<S>>(p);
  bool bad = false;
  int j = 0;
  for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
    const int st = j % STAGES;
    bool ok = false;
    if (!*s_abort) {
      ok = mbar_wait_bounded(smem_addr(&bars[st]), (j / STAGES) & 1, s_abort, p.wait_ns);
      if (!ok && !*s_abort) {
        atomicOr(p.err, ERR_TIMEOUT);
        *s_abort = 1;
      }
    }
    const int y = t / p.nseg, s = t - y * p.nseg;
    const int x0 = s * W;
    double fx = 0.0, fy = 0.0;
    S *out = outs + (size_t)(j & 1) * 9 * W;
    if (ok) {
      const S *tile = tiles + (size_t)st * 9 * SEG + (H - x0);
      auto fetch = [&](int k, int sx, int) -> C { return Store<S>::ld(tile[k * SEG + sx]); };
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int xw = x0 + c * NC + (ctid & ~31);
        const int x = xw + lane;
        C h[9];
        if (plain_span(p, xw, xw + 31, y)) {
          plain_compute<MRT, S>(p, x, y, cf, fetch, bad, h);
        } else if (x < p.nx) {
          node_compute<MRT, S>(A, p, x, y, cf, fetch, fx, fy, bad, h);
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) h[k] = (C)0;
        }
#pragma unroll
        if constexpr (Dithers<S>::value) {
          const uint32_t seed = dither_seed(fold9(h), x, y);
#pragma unroll
          for (int k = 0; k < 9; ++k) out[k * W + (x - x0)] = Store<S>::st_at(h[k], seed, k);
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) out[k * W + (x - x0)] = Store<S>::st(h[k]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&bars[STAGES + st]));
    }
    fence_proxy_async_smem();
    // the bulk store that last read the other output tile has finished
    if (ctid == 0) bulk_wait_read0();
    named_bar(2, NC);
    if (ok && ctid == 0) {
      const int xl = min(x0 + W, p.pitch);
      const uint32_t bytes = (uint32_t)(xl - x0) * (uint32_t)sizeof(S);
#pragma unroll
      for (int k = 0; k < 9; ++k)
        bulk_s2g(B + (size_t)k * p.plane + (size_t)y * p.pitch + x0, smem_addr(out + k * W), bytes);
      bulk_commit();
    }
    if (is_force_item(p, y, s)) post_force<NCW>(p, y, s, fx, fy, ctid, red, s_last, [] { named_bar(1, NC); });
  }
  if (ctid == 0) bulk_wait0();
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, ERR_UNSTABLE);
}

// Dynamic shared memory of a TMA kernel whose row tile holds PX * NCW * 32 *
// CPT nodes (PX = TmaPair<S>::nodes for step_tma and step_tma_batch).
template <class S, int NCW, int CPT, int STAGES, int PX = 1>
constexpr size_t tma_smem_bytes() {
  return (size_t)STAGES * 9 * (PX * NCW * 32 * CPT + 2 * (16 / sizeof(S))) * sizeof(S) + 2 * STAGES * sizeof(uint64_t);
}

// ---- initial state: f*(0) = f_eq(rho0, u0), Eq. 3, as offsets ----------
template <class S>
__global__ void init_kernel(S *__restrict__ A, StepParams p, const double *__restrict__ rho,
                            const double *__restrict__ u, const double *__restrict__ v, int y0, int rows) {
  const long long n = (long long)rows * p.nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = y0 + (int)(i / p.nx);
    const uint32_t lm = link_mask(p, x, y);
    const size_t o = (size_t)y * p.pitch + x;
    if (lm & LM_SOLID) {
#pragma unroll
      for (int k = 0; k < 9; ++k) A[(size_t)k * p.plane + o] = Store<S>::st(0);
      continue;
    }
    const double r = rho[i], ux = u[i], uy = v[i];
    const double uu = ux * ux + uy * uy;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double cu = CX(k) * ux + CY(k) * uy;
      const double feq = WD(k) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      A[(size_t)k * p.plane + o] = Store<S>::st((typename Store<S>::C)(feq - ref_pop(k, p.U)));
    }
  }
}

// ---- initial state from DEVICE fields, optionally with the first-order
// Chapman-Enskog non-equilibrium part (BGK, stress relaxation time tau):
//   f_i = f_eq_i(rho, u) - (tau w_i rho / c_s^2) Q_i : grad u,
//   Q_i = c_i c_i - c_s^2 I, c_s^2 = 1/3.
// Velocity gradients: central differences, one-sided where a neighbour is
// outside the lattice or solid, zero where both are.
__device__ __forceinline__ bool fluid_at(const StepParams &p, int x, int y) {
  if ((unsigned)x >= (unsigned)p.nx || (unsigned)y >= (unsigned)p.ny) return false;
  return !(link_mask(p, x, y) & LM_SOLID);
}
__device__ __forceinline__ double diff1(const float *f, const StepParams &p, int x, int y, int ddx, int ddy) {
  const bool lo = fluid_at(p, x - ddx, y - ddy), hi = fluid_at(p, x + ddx, y + ddy);
  const size_t c = (size_t)y * p.nx + x;
  const double fc = f[c];
  const double fl = lo ? (double)f[(size_t)(y - ddy) * p.nx + (x - ddx)] : fc;
  const double fh = hi ? (double)f[(size_t)(y + ddy) * p.nx + (x + ddx)] : fc;
  if (lo && hi) return 0.5 * (fh - fl);
  if (hi) return fh - fc;
  if (lo) return fc - fl;
  return 0.0;
}

template <class S>
__global__ void init_device_kernel(S *__restrict__ A, StepParams p, const float *__restrict__ rho,
                                   const float *__restrict__ u, const float *__restrict__ v, int with_noneq,
                                   double tau) {
  const long long n = (long long)p.nx * p.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = (int)(i / p.nx);
    const uint32_t lm = link_mask(p, x, y);
    const size_t o = (size_t)y * p.pitch + x;
    if (lm & LM_SOLID) {
#pragma unroll
      for (int k = 0; k < 9; ++k) A[(size_t)k * p.plane + o] = Store<S>::st(0);
      continue;
    }
    const double r = rho[i], ux = u[i], uy = v[i];
    const double uu = ux * ux + uy * uy;
    double dudx = 0.0, dudy = 0.0, dvdx = 0.0, dvdy = 0.0;
    if (with_noneq) {
      dudx = diff1(u, p, x, y, 1, 0);
      dudy = diff1(u, p, x, y, 0, 1);
      dvdx = diff1(v, p, x, y, 1, 0);
      dvdy = diff1(v, p, x, y, 0, 1);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double cu = CX(k) * ux + CY(k) * uy;
      double f = WD(k) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      if (with_noneq) {
        // stored state is post-collision: f*_neq = (1 - 1/tau) f_neq, and
        // (1 - 1/tau) (-tau w rho / c_s^2) = -(tau - 1) w rho / c_s^2
        const double qxx = CX(k) * CX(k) - 1.0 / 3.0, qyy = CY(k) * CY(k) - 1.0 / 3.0, qxy = CX(k) * CY(k);
        f -= 3.0 * (tau - 1.0) * WD(k) * r * (qxx * dudx + qyy * dvdy + qxy * (dudy + dvdx));
      }
      A[(size_t)k * p.plane + o] = Store<S>::st((typename Store<S>::C)(f - ref_pop(k, p.U)));
    }
  }
}

// ---- Eq. 14 force of the stored f*, one CTA, fixed order -----------------
template <class S>
__global__ void __launch_bounds__(256) force_kernel(const S *__restrict__ A, StepParams p) {
  __shared__ double rx[256], ry[256];
  double fx = 0.0, fy = 0.0;
  const int n = p.lw * p.lh;
  for (int i = threadIdx.x; i < n; i += 256) {
    const uint32_t lm = p.lmap[i];
    if ((lm & LM_SOLID) || !(lm & LM_LINKS)) continue;
    const int x = p.lx0 + i % p.lw, y = p.ly0 + i / p.lw;
    const size_t o = (size_t)y * p.pitch + x;
#pragma unroll
    for (int d = 1; d < 9; ++d)
      if (lm & (1u << OPP(d))) {
        const double g = (double)Store<S>::ld(A[(size_t)d * p.plane + o]);
        fx += 2.0 * g * CX(d);
        fy += 2.0 * g * CY(d);
      }
  }
  rx[threadIdx.x] = fx;
  ry[threadIdx.x] = fy;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < 256; ++i) {
      sx += rx[i];
      sy += ry[i];
    }
    const unsigned long long s = *p.step;
    const long long r = (long long)(s % (unsigned long long)p.hist_cap);
    p.hist[2 * r] = sx + p.fconst_x;
    p.hist[2 * r + 1] = sy + p.fconst_y;
    *p.step = s + 1;
  }
}

// ---- moments (Eq. 4) of the stored f* for rows [y0, y0 + rows) ---------
template <class S, class O>
__global__ void fields_kernel(const S *__restrict__ A, StepParams p, O *__restrict__ rho, O *__restrict__ u,
                              O *__restrict__ v, int y0, int rows) {
  const long long n = (long long)rows * p.nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = y0 + (int)(i / p.nx);
    const uint32_t lm = link_mask(p, x, y);
    if (lm & LM_SOLID) {
      rho[i] = (O)1;
      u[i] = (O)0;
      v[i] = (O)0;
      continue;
    }
    const size_t o = (size_t)y * p.pitch + x;
    double g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = (double)Store<S>::ld(A[(size_t)k * p.plane + o]);
    const double drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const double r = 1.0 + drho;
    const double jx = p.U + ((g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]));
    const double jy = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]);
    rho[i] = (O)r;
    u[i] = (O)(jx / r);
    v[i] = (O)(jy / r);
  }
}

// ---- per-row double sums of rho over fluid nodes (mass drift) ----------
template <class S>
__global__ void __launch_bounds__(256) mass_rows_kernel(const S *__restrict__ A, StepParams p, double *__restrict__ part,
                                                        int y0) {
  __shared__ double red[256];
  const int y = y0 + blockIdx.x;
  double acc = 0.0;
  for (int x = threadIdx.x; x < p.nx; x += 256) {
    if (link_mask(p, x, y) & LM_SOLID) continue;
    const size_t o = (size_t)y * p.pitch + x;
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) d += (double)Store<S>::ld(A[(size_t)k * p.plane + o]);
    acc += 1.0 + d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- host-side launchers for one storage type ----------------------------
template <class S>
struct Launch {
  static cudaError_t direct(const void *A, void *B, const StepParams &p, cudaStream_t st) {
    const int nitems = p.ny * p.nseg;
    if (p.mrt)
      step_direct<S, 256, 1><<<nitems, 256, 0, st>>>((const S *)A, (S *)B, p);
    else
      step_direct<S, 256, 0><<<nitems, 256, 0, st>>>((const S *)A, (S *)B, p);
    return cudaGetLastError();
  }

  template <int NCW, int CPT, int STAGES>
  static cudaError_t tma_one(int grid, const void *A, void *B, const StepParams &p, cudaStream_t st) {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (p.mrt)
      step_tma<S, NCW, CPT, STAGES, 1><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    else
      step_tma<S, NCW, CPT, STAGES, 0><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    return cudaGetLastError();
  }
  template <int NCW, int CPT, int STAGES>
  static cudaError_t tma_prep() {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(step_tma<S, NCW, CPT, STAGES, 0>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_tma<S, NCW, CPT, STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  template <int NCW, int CPT, int STAGES>
  static int tma_occ() {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return 0;
    int n = 0;
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_tma<S, NCW, CPT, STAGES, 0>, (NCW + 1) * 32, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, step_tma<S, NCW, CPT, STAGES, 1>, (NCW + 1) * 32, smem) !=
            cudaSuccess)
      return 0;
    return n < m ? n : m;
  }

  // Interpolated bounce-back on the TMA kernel: float storage, the shapes
  // the library picks by default for float ((12,2,4), (10,2,4), (8,2,4)).
  template <int NCW, int CPT, int STAGES>
  static cudaError_t tma_interp_one(int grid, const void *A, void *B, const StepParams &p, cudaStream_t st, bool prep) {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (prep) {
      const cudaError_t e = cudaFuncSetAttribute(step_tma<S, NCW, CPT, STAGES, 0, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(step_tma<S, NCW, CPT, STAGES, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    }
    if (p.mrt)
      step_tma<S, NCW, CPT, STAGES, 1, true><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    else
      step_tma<S, NCW, CPT, STAGES, 0, true><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    return cudaGetLastError();
  }
  // prep != 0: only set the shared-memory limit (and so report whether this
  // storage type and shape have the kernel: cudaErrorNotSupported if not)
  static cudaError_t tma_interp(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st,
                                int prep) {
    if constexpr (std::is_same<S, float>::value) {
      switch (shape) {
        case 6: return tma_interp_one<8, 2, 4>(grid, A, B, p, st, prep != 0);
        case 12: return tma_interp_one<12, 2, 4>(grid, A, B, p, st, prep != 0);
        case 15: return tma_interp_one<10, 2, 4>(grid, A, B, p, st, prep != 0);
      }
    }
    return cudaErrorNotSupported;
  }

  // The multi-step kernel (cooperative launch, so that all CTAs are
  // resident at once) followed by the reduction of its force slots.
  template <int NCW, int CPT, int STAGES>
  static cudaError_t wave_one(int grid, void *A, void *B, const StepParams &p, const WaveParams &w, cudaStream_t st,
                              int mode, int *occ) {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto k0 = step_tma_wave<S, NCW, CPT, STAGES, 0>;
    auto k1 = step_tma_wave<S, NCW, CPT, STAGES, 1>;
    if (mode == 1) {  // set the shared-memory limit
      const cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (mode == 2) {  // resident CTAs per SM into *occ
      int n = 0, m = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k0, (NCW + 2) * 32, smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k1, (NCW + 2) * 32, smem) != cudaSuccess)
        return cudaErrorInvalidConfiguration;
      *occ = n < m ? n : m;
      return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((NCW + 2) * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = p.mrt ? cudaLaunchKernelEx(&cfg, k1, (S *)A, (S *)B, p, w)
                                : cudaLaunchKernelEx(&cfg, k0, (S *)A, (S *)B, p, w);
    if (e != cudaSuccess) return e;
    wave_finish<S><<<1, 1024, 0, st>>>(p, w);
    return cudaGetLastError();
  }
  static cudaError_t wave_dispatch(int shape, int grid, void *A, void *B, const StepParams &p, const WaveParams &w,
                                   cudaStream_t st, int mode, int *occ) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return wave_one<a, b, c>(grid, A, B, p, w, st, mode, occ);
      GBLBM_WAVE_SHAPES(X)
#undef X
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t wave(int shape, int grid, void *A, void *B, const StepParams &p, const WaveParams &w,
                          cudaStream_t st) {
    return wave_dispatch(shape, grid, A, B, p, w, st, 0, nullptr);
  }
  static cudaError_t wave_prep(int shape) {
    return wave_dispatch(shape, 0, nullptr, nullptr, StepParams{}, WaveParams{}, nullptr, 1, nullptr);
  }
  static int wave_occupancy(int shape) {
    int n = 0;
    if (wave_dispatch(shape, 0, nullptr, nullptr, StepParams{}, WaveParams{}, nullptr, 2, &n) != cudaSuccess) return 0;
    return n;
  }

  static cudaError_t tma(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return tma_one<a, b, c>(grid, A, B, p, st);
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t prep(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return tma_prep<a, b, c>();
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  static int occupancy(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return tma_occ<a, b, c>();
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return 0;
  }
  static size_t smem(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return tma_smem_bytes<S, a, b, c, TmaPair<S>::nodes>();
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return 0;
  }

  template <int NCW, int CPT, int STAGES>
  static cudaError_t bulk_one(int grid, const void *A, void *B, const StepParams &p, cudaStream_t st) {
    constexpr size_t smem = tma_bulk_smem_bytes<S, NCW, CPT, STAGES>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (p.mrt)
      step_tma_bulk<S, NCW, CPT, STAGES, 1><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    else
      step_tma_bulk<S, NCW, CPT, STAGES, 0><<<grid, (NCW + 1) * 32, smem, st>>>((const S *)A, (S *)B, p);
    return cudaGetLastError();
  }
  template <int NCW, int CPT, int STAGES>
  static cudaError_t bulk_prep_one() {
    constexpr size_t smem = tma_bulk_smem_bytes<S, NCW, CPT, STAGES>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(step_tma_bulk<S, NCW, CPT, STAGES, 0>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_tma_bulk<S, NCW, CPT, STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  template <int NCW, int CPT, int STAGES>
  static int bulk_occ_one() {
    constexpr size_t smem = tma_bulk_smem_bytes<S, NCW, CPT, STAGES>();
    if (smem > 227 * 1024) return 0;
    int n = 0, m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_tma_bulk<S, NCW, CPT, STAGES, 0>, (NCW + 1) * 32,
                                                      smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, step_tma_bulk<S, NCW, CPT, STAGES, 1>, (NCW + 1) * 32,
                                                      smem) != cudaSuccess)
      return 0;
    return n < m ? n : m;
  }
  static cudaError_t tma_bulk(int shape, int grid, const void *A, void *B, const StepParams &p, cudaStream_t st) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return bulk_one<a, b, c>(grid, A, B, p, st);
      GBLBM_TMA_BULK_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t bulk_prep(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return bulk_prep_one<a, b, c>();
      GBLBM_TMA_BULK_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  static int bulk_occupancy(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return bulk_occ_one<a, b, c>();
      GBLBM_TMA_BULK_SHAPES(X)
#undef X
    }
    return 0;
  }
  static size_t bulk_smem(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return tma_bulk_smem_bytes<S, a, b, c>();
      GBLBM_TMA_BULK_SHAPES(X)
#undef X
    }
    return 0;
  }

  static cudaError_t init(void *A, const StepParams &p, const double *r, const double *u, const double *v, int y0,
                          int rows, cudaStream_t st) {
    const long long n = (long long)rows * p.nx;
    const int blocks = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    init_kernel<S><<<blocks > 0 ? blocks : 1, 256, 0, st>>>((S *)A, p, r, u, v, y0, rows);
    return cudaGetLastError();
  }
  static cudaError_t init_device(void *A, const StepParams &p, const float *r, const float *u, const float *v,
                                 int with_noneq, double tau, cudaStream_t st) {
    const long long n = (long long)p.nx * p.ny;
    const int blocks = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    init_device_kernel<S><<<blocks > 0 ? blocks : 1, 256, 0, st>>>((S *)A, p, r, u, v, with_noneq, tau);
    return cudaGetLastError();
  }
  static cudaError_t force(const void *A, const StepParams &p, cudaStream_t st) {
    force_kernel<S><<<1, 256, 0, st>>>((const S *)A, p);
    return cudaGetLastError();
  }
  static cudaError_t fields(const void *A, const StepParams &p, void *r, void *u, void *v, int dbl, int y0, int rows,
                            cudaStream_t st) {
    const long long n = (long long)rows * p.nx;
    const int blocks = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    if (dbl)
      fields_kernel<S, double><<<blocks > 0 ? blocks : 1, 256, 0, st>>>((const S *)A, p, (double *)r, (double *)u,
                                                                        (double *)v, y0, rows);
    else
      fields_kernel<S, float><<<blocks > 0 ? blocks : 1, 256, 0, st>>>((const S *)A, p, (float *)r, (float *)u,
                                                                       (float *)v, y0, rows);
    return cudaGetLastError();
  }
  static cudaError_t mass_rows(const void *A, const StepParams &p, double *part, int y0, int rows, cudaStream_t st) {
    mass_rows_kernel<S><<<rows, 256, 0, st>>>((const S *)A, p, part, y0);
    return cudaGetLastError();
  }

  static cudaError_t batch_direct(const CaseDesc *cases, int ncases, long long nitems, int parity, int mrt,
                                  cudaStream_t st) {
    if (mrt)
      step_direct_batch<S, 256, 1><<<(unsigned)nitems, 256, 0, st>>>(cases, ncases, parity);
    else
      step_direct_batch<S, 256, 0><<<(unsigned)nitems, 256, 0, st>>>(cases, ncases, parity);
    return cudaGetLastError();
  }
  template <int NCW, int CPT, int STAGES>
  static cudaError_t batch_tma_one(int grid, const CaseDesc *cases, int ncases, long long nitems, int parity,
                                   int mrt, cudaStream_t st) {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (mrt)
      step_tma_batch<S, NCW, CPT, STAGES, 1><<<grid, (NCW + 1) * 32, smem, st>>>(cases, ncases, nitems, parity);
    else
      step_tma_batch<S, NCW, CPT, STAGES, 0><<<grid, (NCW + 1) * 32, smem, st>>>(cases, ncases, nitems, parity);
    return cudaGetLastError();
  }
  template <int NCW, int CPT, int STAGES>
  static cudaError_t batch_tma_prep() {
    constexpr size_t smem = tma_smem_bytes<S, NCW, CPT, STAGES, TmaPair<S>::nodes>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(step_tma_batch<S, NCW, CPT, STAGES, 0>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_tma_batch<S, NCW, CPT, STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  static cudaError_t batch_tma(int shape, int grid, const CaseDesc *cases, int ncases, long long nitems, int parity,
                               int mrt, cudaStream_t st) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return batch_tma_one<a, b, c>(grid, cases, ncases, nitems, parity, mrt, st);
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t batch_prep(int shape) {
    switch (shape) {
#define X(id, a, b, c) \
  case id:             \
    return batch_tma_prep<a, b, c>();
      GBLBM_TMA_SHAPES(X)
#undef X
    }
    return cudaErrorInvalidValue;
  }

  static const KernelOps *table() {
    static const KernelOps ops = {(int)sizeof(S), &direct,     &tma,          &prep,     &occupancy,
                                  &smem,          &init,       &force,        &fields,   &mass_rows,
                                  &batch_direct,  &batch_tma,  &batch_prep, &init_device,
                                  &tma_bulk,      &bulk_prep,  &bulk_occupancy, &bulk_smem,
                                  TmaPair<S>::nodes, &tma_interp, &wave,  &wave_prep, &wave_occupancy};
    return &ops;
  }
};

}  // namespace gblbm
