// nn_tc.cu -- the 3x3 convolutions of the warm-start network on the
// Blackwell tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulators in tensor memory), operands staged by the TMA engine
// (cp.async.bulk.tensor) into a multi-stage shared-memory ring guarded by
// mbarriers, and a warp-specialised CTA.
//
// Implicit GEMM.  One CTA computes a tile of 128 output pixels (a segment of
// one image row) x BN output channels:
//   D[m, j] = sum over taps (dy, dx) and input channels c of
//             X[n, h + dy - 1, w0 + m + dx - 1, c] * Wt[o0 + j, dy, dx, c].
// The K loop runs over (tap, chunk of CK input channels).  For each step the
// TMA engine copies the 128 x CK input tile of that tap straight from the
// NHWC activations -- the tap's shift is only a change of the copy's start
// coordinates, and rows or columns outside the image arrive as zeros (the
// convolution's zero padding) -- and the BN x CK weight tile; both land in
// the K-major, 128-byte (CK = 64) or 64-byte (CK = 32) swizzled layout the
// tensor core reads.  No im2col matrix is ever formed.
//
// Warp roles (192 threads): warp 0 issues the TMA copies (one lane) and owns
// the tensor-memory allocation; warp 1 issues the MMAs (one lane) and
// returns each stage to the producer with tcgen05.commit; warps 2-5 read the
// accumulator back (tcgen05.ld, each warp its 32-lane quarter), add the
// bias, apply ReLU or the ReLU-derivative mask and store bfloat16.
//
// Every wait is bounded (2 s); a wait that gives up records the failure in
// g_tc_status, the CTA stops issuing work, waits (bounded) for what it has in
// flight and frees its tensor memory before it returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "nn_tc.h"

namespace gbnn_tc {

typedef __nv_bfloat16 bf16;

__device__ unsigned g_tc_status;  // 1: a bounded wait gave up

constexpr int kThreads = 192;
constexpr int kTileM = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
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
// true when the phase of this parity completed; false after kWaitNs or when
// *abort is set
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void give_up(volatile int *abort) {
  *abort = 1;
  atomicOr(&g_tc_status, 1u);
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (tensor memory) (+)= A (shared) x B (shared)^T, M = 128, N and K = 16 from
// the instruction descriptor; accumulate = 0 overwrites D.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued so far is done.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major, swizzled operand tile whose
// 8-row groups lie sbo bytes apart (tcgen05 descriptor format: start
// address >> 4 in bits 0-13, leading-dimension offset in 16-29 (unused for
// swizzled K-major tiles), stride-dimension offset >> 4 in 32-45, version 1
// in 46-47, swizzle mode in 61-63).
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr, uint32_t sbo, uint32_t swizzle_mode) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swizzle_mode << 61;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

template <int BN> struct TmemCols {
  static constexpr uint32_t value = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

// Resident CTAs per SM whose tensor-memory allocations fit in the SM's 512
// columns, and the dynamic shared memory that keeps any more from being
// placed there (a CTA that cannot allocate would wait for another to free).
__host__ __device__ constexpr int tmem_ctas(uint32_t ncols) { return (int)(512u / ncols); }
__host__ __device__ constexpr int smem_floor(uint32_t ncols) { return 233472 / (tmem_ctas(ncols) + 1) + 1024; }

template <int BN, int CK, int STAGES>
struct TcLayout {
  static constexpr uint32_t ACC_COLS = TmemCols<BN>::value;  // one accumulator
  static constexpr uint32_t NCOLS = 2 * ACC_COLS;            // two, double-buffered
  // taps per stage: with 32-channel chunks a stage carries the three taps of
  // one kernel row, so each pipeline handshake feeds six MMAs instead of two
  static constexpr int TPS = CK == 32 ? 3 : 1;
  static constexpr int A_BYTES = kTileM * CK * 2;  // one tap's input tile
  static constexpr int B_BYTES = BN * CK * 2;      // one tap's weight tile
  static constexpr int A_OFF = 0;
  static constexpr int B_OFF = STAGES * TPS * A_BYTES;
  static constexpr int BAR_OFF = B_OFF + STAGES * TPS * B_BYTES;  // full[S], empty[S], acc_full[2], acc_empty[2], drain
  static constexpr int NBARS = 2 * STAGES + 5;
  static constexpr int BIAS_OFF = BAR_OFF + NBARS * 8 + 16;  // the bias of every output channel
  static constexpr int BYTES = BIAS_OFF + 512 * 4;
  static constexpr int ALLOC = BYTES + 1024 > smem_floor(NCOLS) ? BYTES + 1024 : smem_floor(NCOLS);
  static constexpr uint32_t SBO = 8 * CK * 2;
  static constexpr uint32_t SWZ = CK == 64 ? 2u : 4u;  // 128-byte or 64-byte swizzle
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent: each CTA walks output tiles t = blockIdx.x, += gridDim.x, in
// the order (image, row, 128-pixel segment, channel chunk) so that tiles
// running at the same time share their input rows in L2.  The producer and
// the MMA issuer stream k-blocks across tile boundaries; the accumulator is
// double-buffered in tensor memory, so the epilogue of one tile overlaps the
// main loop of the next.
template <int BN, int CK, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_w,
                   const float *__restrict__ bias, bf16 *__restrict__ y, int ys, const bf16 *__restrict__ mask, int ms,
                   int H, int W, int cin, int nchunks, int relu, int ntiles) {
  using Lay = TcLayout<BN, CK, STAGES>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::BAR_OFF);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lay::BAR_OFF + Lay::NBARS * 8);
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;

  float *sbias = reinterpret_cast<float *>(smem + Lay::BIAS_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TPS = Lay::TPS;
  const int kchunks = cin / CK, kblocks = (9 / TPS) * kchunks;
  const int wtiles = (W + kTileM - 1) / kTileM;
  for (int o = threadIdx.x; o < nchunks * BN; o += blockDim.x) sbias[o] = bias ? bias[o] : 0.f;
  const uint32_t full0 = saddr(&bars[0]), empty0 = saddr(&bars[STAGES]);
  const uint32_t accf0 = saddr(&bars[2 * STAGES]), acce0 = saddr(&bars[2 * STAGES + 2]);
  const uint32_t drain_bar = saddr(&bars[2 * STAGES + 4]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);   // the MMA issuer's commit
      mbar_init(acce0 + 8 * b, 4);   // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&tmap_x);
    prefetch_map(&tmap_w);
  }
  if (warp == 0) {
    tmem_alloc(saddr(tmem_slot), Lay::NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int g = 0;  // k-blocks issued by this CTA
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const int chunk = t % nchunks, r1 = t / nchunks;
        const int wt = r1 % wtiles, r2 = r1 / wtiles;
        const int h = r2 % H, n = r2 / H;
        const int w0 = wt * kTileM, o0 = chunk * BN;
        int tap = 0, c0 = 0;  // first tap of the stage's group, channel chunk
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int s = g % STAGES;
          if (g >= STAGES && !mbar_wait(empty0 + 8 * s, ((g / STAGES) - 1) & 1, s_abort)) {
            if (!*s_abort) give_up(s_abort);
            stop = true;
            break;
          }
          if (*s_abort) {
            stop = true;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, (uint32_t)(TPS * (Lay::A_BYTES + Lay::B_BYTES)));
#pragma unroll
          for (int j = 0; j < TPS; ++j) {
            const int tj = tap + j, dy = tj / 3, dx = tj - 3 * dy;
            tma_load_4d(saddr(smem + Lay::A_OFF + (s * TPS + j) * Lay::A_BYTES), &tmap_x, full0 + 8 * s, c0,
                        w0 + dx - 1, h + dy - 1, n);
            tma_load_2d(saddr(smem + Lay::B_OFF + (s * TPS + j) * Lay::B_BYTES), &tmap_w, full0 + 8 * s,
                        tj * cin + c0, o0);
          }
          c0 += CK;
          if (c0 == cin) {
            c0 = 0;
            tap += TPS;
          }
        }
      }
      // leave no copy in flight into this CTA's shared memory
      for (int q = g - STAGES < 0 ? 0 : g - STAGES; q < g; ++q) {
        const unsigned long long t0 = now_ns();
        while (!mbar_test(full0 + 8 * (q % STAGES), (q / STAGES) & 1)) {
          if (now_ns() - t0 > kWaitNs) {
            give_up(s_abort);
            break;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BN);
      int g = 0, i = 0, issued = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++i) {
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(acce0 + 8 * b, ((i >> 1) - 1) & 1, s_abort)) {  // epilogue done with buffer b
          if (!*s_abort) give_up(s_abort);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * Lay::ACC_COLS);
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int s = g % STAGES;
          if (!mbar_wait(full0 + 8 * s, (g / STAGES) & 1, s_abort)) {
            if (!*s_abort) give_up(s_abort);
            stop = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int j = 0; j < TPS; ++j) {
            const uint64_t ad = kmajor_desc(saddr(smem + Lay::A_OFF + (s * TPS + j) * Lay::A_BYTES), Lay::SBO, Lay::SWZ);
            const uint64_t bd = kmajor_desc(saddr(smem + Lay::B_OFF + (s * TPS + j) * Lay::B_BYTES), Lay::SBO, Lay::SWZ);
#pragma unroll
            for (int kk = 0; kk < CK / 16; ++kk)  // K = 16 per MMA: 32 bytes (2 in the address field) further
              umma_bf16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (kb | j | kk) != 0);
          }
          umma_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
          ++issued;
        }
        if (!stop) umma_commit(accf0 + 8 * b);  // accumulator b is complete
      }
      if (issued > 0) {  // every MMA done before the tensor memory is freed
        umma_commit(drain_bar);
        const unsigned long long t0 = now_ns();
        while (!mbar_test(drain_bar, 0)) {
          if (now_ns() - t0 > kWaitNs) {
            give_up(s_abort);
            break;
          }
        }
      }
    }
  } else {  // ---------------- epilogue warps 2..5
    const int quarter = warp & 3;  // tensor-memory lanes 32 * quarter .. + 31
    const int m = 32 * quarter + lane;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      bool ok = mbar_wait(accf0 + 8 * b, (i >> 1) & 1, s_abort);
      if (!ok && !*s_abort) give_up(s_abort);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective: one decision per warp
      if (!ok) break;
      tc_fence_after();
      const int chunk = t % nchunks, r1 = t / nchunks;
      const int wt = r1 % wtiles, r2 = r1 / wtiles;
      const int h = r2 % H, n = r2 / H;
      const int px = wt * kTileM + m, o0 = chunk * BN;
      const size_t pix = ((size_t)n * H + h) * W + px;
#pragma unroll 1
      for (int j0 = 0; j0 < BN; j0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t)(b * Lay::ACC_COLS) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)j0, r);
        tmem_ld_wait();
        if (px < W) {
          const int o = o0 + j0;
          float v[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]) + sbias[o + q];
          if (relu) {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q], 0.f);
          }
          if (mask) {
            const uint4 *mp = reinterpret_cast<const uint4 *>(mask + pix * ms + o);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint4 mv = __ldg(mp + q);
              const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(&mw[e]);
                if (!(__bfloat162float(mk.x) > 0.f)) v[8 * q + 2 * e] = 0.f;
                if (!(__bfloat162float(mk.y) > 0.f)) v[8 * q + 2 * e + 1] = 0.f;
              }
            }
          }
          uint4 *yp = reinterpret_cast<uint4 *>(y + pix * ys + o);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
              pk[e] = *reinterpret_cast<const uint32_t *>(&b2);
            }
            yp[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        }
      }
      // accumulator b may be overwritten once all four warps have read it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, Lay::NCOLS);
  }
}

// ---- weight gradient ---------------------------------------------------------
// gw[o, tap, c] += sum over pixels p of x[p + shift(tap), c] * gy[p, o].
// GEMM with M = (tap, input channel), N = output channels, K = pixels.  The
// 128 rows of one M tile are four blocks of 32 rows, each block one
// (tap, 32-channel chunk) pair -- so the nine taps of a 32-channel layer
// fill M with little waste -- and N is the whole output-channel count
// (<= 256).  Per K step of 128 pixels (a segment of one image row) the TMA
// engine copies the four shifted 128 x 32 input boxes and the 128 x N output
// gradient; in NHWC both arrive channel-contiguous, i.e. M- and N-major
// (MN-major, 64-byte swizzle: 32-channel atoms 128 x 64 B apart, 8-pixel row
// groups 512 B apart).  Each CTA sums a contiguous range of K steps (split
// K); the epilogue warp of TMEM quarter q owns row block q and adds its
// 32 x N partial sums to gw with coalesced float atomics (order not fixed).
constexpr int kWgPix = 128;                  // pixels per K step
constexpr int kWgBlockBytes = kWgPix * 32 * 2;  // one 128-pixel x 32-channel box

template <int BN, int STAGES>
struct WgLayout {
  static constexpr int A_BYTES = 4 * kWgBlockBytes;
  static constexpr int B_BYTES = (BN / 32) * kWgBlockBytes;
  static constexpr int A_OFF = 0;
  static constexpr int B_OFF = STAGES * A_BYTES;
  static constexpr int BAR_OFF = B_OFF + STAGES * B_BYTES;
  static constexpr int BYTES = BAR_OFF + (2 * STAGES + 2) * 8 + 16;
  static constexpr int ALLOC = BYTES + 1024;
};

// Instruction descriptor, kind::f16, FP32 accumulator, BF16 A and B, both
// MN-major (transpose bits 15 and 16), M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int n) { return idesc_bf16(n) | (1u << 15) | (1u << 16); }

// Descriptor of an MN-major operand made of 32-element (64-byte swizzled)
// atoms lbo bytes apart along M or N, with 8-pixel row groups 512 B apart.
__device__ __forceinline__ uint64_t mnmajor_desc(uint32_t addr, uint32_t lbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;  // 64-byte swizzle
  return d;
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_g,
                    float *__restrict__ gw, int H, int W, int cin, int cout, int nblocks, long long ksteps,
                    long long ksteps_per_cta) {
  using Lay = WgLayout<BN, STAGES>;
  constexpr uint32_t NCOLS = TmemCols<BN>::value;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::BAR_OFF);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lay::BAR_OFF + (2 * STAGES + 2) * 8);
  __shared__ int s_abort_store;
  volatile int *s_abort = &s_abort_store;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mtile = blockIdx.x;  // M tiles of one K range run side by side and share their loads in L2
  const long long k0 = (long long)blockIdx.y * ksteps_per_cta;
  const long long k1 = k0 + ksteps_per_cta < ksteps ? k0 + ksteps_per_cta : ksteps;
  const int nk = k1 > k0 ? (int)(k1 - k0) : 0;
  const int segs = (W + kWgPix - 1) / kWgPix;  // K steps per image row
  const int cchunks = cin / 32;
  const uint32_t full0 = saddr(&bars[0]), empty0 = saddr(&bars[STAGES]);
  const uint32_t acc_bar = saddr(&bars[2 * STAGES]), drain_bar = saddr(&bars[2 * STAGES + 1]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(acc_bar, 1);
    mbar_init(drain_bar, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&tmap_x);
    prefetch_map(&tmap_g);
  }
  if (warp == 0) {
    tmem_alloc(saddr(tmem_slot), NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0 && nk > 0) {  // ---------------- TMA producer
      // row block -> (tap, 32-channel chunk): the channel and the tap's shift
      // of each of the four boxes; blocks past the last one load a box wholly
      // outside the image (zeros)
      int bc[4], bdx[4], bdy[4];
      bool blive[4];
#pragma unroll
      for (int rb = 0; rb < 4; ++rb) {
        const int blk = 4 * mtile + rb;
        const int tap = blk / cchunks, dy = tap / 3;
        blive[rb] = blk < nblocks;
        bc[rb] = blive[rb] ? (blk - tap * cchunks) * 32 : 0;
        bdx[rb] = tap - 3 * dy - 1;
        bdy[rb] = dy - 1;
      }
      // the K step's image row and segment, advanced incrementally
      int seg = (int)(k0 % segs);
      const long long row0 = k0 / segs;
      int h = (int)(row0 % H), n = (int)(row0 / H);
      int kb = 0;
      for (; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, ((kb / STAGES) - 1) & 1, s_abort)) {
          if (!*s_abort) give_up(s_abort);
          break;
        }
        if (*s_abort) break;
        const int w0 = seg * kWgPix;
        mbar_expect_tx(full0 + 8 * s, (uint32_t)(Lay::A_BYTES + Lay::B_BYTES));
        const uint32_t a = saddr(smem + Lay::A_OFF + s * Lay::A_BYTES);
#pragma unroll
        for (int rb = 0; rb < 4; ++rb) {
          tma_load_4d(a + rb * kWgBlockBytes, &tmap_x, full0 + 8 * s, bc[rb], blive[rb] ? w0 + bdx[rb] : W,
                      blive[rb] ? h + bdy[rb] : H, n);
        }
        const uint32_t b = saddr(smem + Lay::B_OFF + s * Lay::B_BYTES);
#pragma unroll
        for (int nb = 0; nb < BN / 32; ++nb) tma_load_4d(b + nb * kWgBlockBytes, &tmap_g, full0 + 8 * s, 32 * nb, w0, h, n);
        if (++seg == segs) {
          seg = 0;
          if (++h == H) {
            h = 0;
            ++n;
          }
        }
      }
      for (int q = kb - STAGES < 0 ? 0 : kb - STAGES; q < kb; ++q) {
        const unsigned long long t0 = now_ns();
        while (!mbar_test(full0 + 8 * (q % STAGES), (q / STAGES) & 1)) {
          if (now_ns() - t0 > kWaitNs) {
            give_up(s_abort);
            break;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && nk > 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16_mn(BN);
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(full0 + 8 * s, (kb / STAGES) & 1, s_abort)) {
          if (!*s_abort) give_up(s_abort);
          break;
        }
        tc_fence_after();
        const uint64_t ad = mnmajor_desc(saddr(smem + Lay::A_OFF + s * Lay::A_BYTES), kWgBlockBytes);
        const uint64_t bd = mnmajor_desc(saddr(smem + Lay::B_OFF + s * Lay::B_BYTES), kWgBlockBytes);
#pragma unroll
        for (int kk = 0; kk < kWgPix / 16; ++kk)  // 16 pixels = two 8-row groups = 1024 B (64 in the field)
          umma_bf16(tmem, ad + 64 * kk, bd + 64 * kk, idesc, (kb | kk) != 0);
        umma_commit(empty0 + 8 * s);
        ++issued;
      }
      if (issued == nk) {
        umma_commit(acc_bar);
      } else if (issued > 0) {
        umma_commit(drain_bar);
        const unsigned long long t0 = now_ns();
        while (!mbar_test(drain_bar, 0)) {
          if (now_ns() - t0 > kWaitNs) break;
        }
      }
    }
  } else if (nk > 0) {  // ---------------- epilogue warps 2..5
    const int quarter = warp & 3;  // row block `quarter` of the M tile
    const int blk = 4 * mtile + quarter;
    bool ok = mbar_wait(acc_bar, 0, s_abort);
    if (!ok && !*s_abort) give_up(s_abort);
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      tc_fence_after();
      const int tap = blk / cchunks, c = (blk - tap * cchunks) * 32 + lane;
#pragma unroll 1
      for (int j0 = 0; j0 < BN; j0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)j0, r);
        tmem_ld_wait();
        if (blk < nblocks) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (j0 + i < cout) atomicAdd(gw + ((size_t)(j0 + i) * 9 + tap) * cin + c, __uint_as_float(r[i]));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOLS);
  }
}

// gb[o] += sum over pixels of gy[p, o]: each block sums a pixel range into
// shared memory, then one atomic per channel.
__global__ void bias_grad_kernel(const bf16 *__restrict__ gy, int gs, float *__restrict__ gb, long long P, int cout,
                                 long long pix_per_block) {
  extern __shared__ float part[];
  for (int i = threadIdx.x; i < cout; i += blockDim.x) part[i] = 0.f;
  __syncthreads();
  const long long p0 = (long long)blockIdx.x * pix_per_block;
  const long long p1 = p0 + pix_per_block < P ? p0 + pix_per_block : P;
  const int lanes = blockDim.x / cout > 0 ? blockDim.x / cout : 1;  // pixels in parallel
  const int o = threadIdx.x % cout, sub = threadIdx.x / cout;
  if (sub < lanes && (int)threadIdx.x < lanes * cout) {
    float acc = 0.f;
    for (long long p = p0 + sub; p < p1; p += lanes) acc += __bfloat162float(gy[p * gs + o]);
    atomicAdd(&part[o], acc);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cout; i += blockDim.x) atomicAdd(gb + i, part[i]);
}

// ---- host side ----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  return sms;
}

template <int BN, int CK, int STAGES>
cudaError_t launch(const CUtensorMap &tx, const CUtensorMap &tw, const float *bias, bf16 *y, int ys, const bf16 *mask,
                   int ms, int N, int H, int W, int cin, int nchunks, int relu, cudaStream_t st) {
  using Lay = TcLayout<BN, CK, STAGES>;
  auto kern = conv_tc_kernel<BN, CK, STAGES>;
  static int per_sm = 0;
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::ALLOC);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per
    // CTA), registers (64K per SM, allocated in units of 8 per thread),
    // threads, and the tensor-memory columns
    const int regs = (fa.numRegs + 7) / 8 * 8;
    int n = 233472 / (Lay::ALLOC + 1024);
    n = n < 65536 / (regs * kThreads) ? n : 65536 / (regs * kThreads);
    n = n < 2048 / kThreads ? n : 2048 / kThreads;
    n = n < tmem_ctas(Lay::NCOLS) ? n : tmem_ctas(Lay::NCOLS);
    if (n < 1) return cudaErrorInvalidConfiguration;
    per_sm = n;
  }
  const long long ntiles = (long long)N * H * ((W + kTileM - 1) / kTileM) * nchunks;
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  const int grid = (int)(ntiles < (long long)per_sm * sm_count() ? ntiles : (long long)per_sm * sm_count());
  kern<<<grid, kThreads, Lay::ALLOC, st>>>(tx, tw, bias, y, ys, mask, ms, H, W, cin, nchunks, relu, (int)ntiles);
  return cudaGetLastError();
}

bool eligible(int cin, int cout, int xs, int ys, const void *x, const void *w, const void *y, const void *mask,
              int ms) {
  if (cin % 32 || cout % 32 || cout > 512 || xs % 8 || ys % 8) return false;
  if (cout > 256 && (cout / 2) % 32) return false;  // two equal chunks of a multiple of 32
  if ((uintptr_t)x % 16 || (uintptr_t)w % 16 || (uintptr_t)y % 16) return false;
  if (mask && ((uintptr_t)mask % 16 || ms % 8)) return false;
  return true;
}

int conv_fwd(const void *x, int xs, const void *w, const float *bias, void *y, int ys, const void *mask, int ms, int N,
             int H, int W, int cin, int cout, int relu, cudaStream_t st) {
  if (!eligible(cin, cout, xs, ys, x, w, y, mask, ms)) return kNotEligible;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return -2;
  const int ck = cin % 64 == 0 ? 64 : 32;
  const int bn = cout <= 256 ? cout : cout / 2;
  const int nchunks = cout / bn;
  CUtensorMap tx, tw;
  const CUtensorMapSwizzle swz = ck == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)xs * 2, (cuuint64_t)W * xs * 2, (cuuint64_t)H * W * xs * 2};
    const cuuint32_t box[4] = {(cuuint32_t)ck, (cuuint32_t)kTileM, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)9 * cin, (cuuint64_t)cout};
    const cuuint64_t strides[1] = {(cuuint64_t)9 * cin * 2};
    const cuuint32_t box[2] = {(cuuint32_t)ck, (cuuint32_t)bn};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(w), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  const bf16 *mb = (const bf16 *)mask;
  bf16 *yb = (bf16 *)y;
  cudaError_t e = cudaErrorInvalidValue;
#define GBNN_TC_CASE(BN_, CK_, ST_)                                                                          \
  if (bn == BN_ && ck == CK_)                                                                                \
    e = launch<BN_, CK_, ST_>(tx, tw, bias, yb, ys, mb, ms, N, H, W, cin, nchunks, relu, st);                \
  else
  GBNN_TC_CASE(32, 32, 3)
  GBNN_TC_CASE(64, 32, 2)
  GBNN_TC_CASE(96, 32, 3)
  GBNN_TC_CASE(128, 32, 3)
  GBNN_TC_CASE(192, 32, 3)
  GBNN_TC_CASE(256, 32, 2)
  GBNN_TC_CASE(32, 64, 4)
  GBNN_TC_CASE(64, 64, 4)
  GBNN_TC_CASE(96, 64, 4)
  GBNN_TC_CASE(128, 64, 4)
  GBNN_TC_CASE(192, 64, 4)
  GBNN_TC_CASE(256, 64, 4)
  return kNotEligible;
#undef GBNN_TC_CASE
  return e == cudaSuccess ? 0 : -2;
}

template <int BN, int STAGES>
cudaError_t launch_wgrad(const CUtensorMap &tx, const CUtensorMap &tg, float *gw, int H, int W, int cin, int cout,
                         int nblocks, int mtiles, long long ksteps, int splits, cudaStream_t st) {
  using Lay = WgLayout<BN, STAGES>;
  auto kern = wgrad_tc_kernel<BN, STAGES>;
  static bool prepared = false;
  if (!prepared) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::ALLOC);
    if (e != cudaSuccess) return e;
    prepared = true;
  }
  const long long per = (ksteps + splits - 1) / splits;
  const int nsplit = (int)((ksteps + per - 1) / per);
  kern<<<dim3(mtiles, nsplit), kThreads, Lay::ALLOC, st>>>(tx, tg, gw, H, W, cin, cout, nblocks, ksteps, per);
  return cudaGetLastError();
}

int conv_wgrad(const void *x, int xs, const void *gy, int gs, float *gw, float *gb, int N, int H, int W, int cin,
               int cout, int splits, cudaStream_t st) {
  if (cin % 32 || xs % 8 || gs % 8 || (uintptr_t)x % 16 || (uintptr_t)gy % 16) return kNotEligible;
  const int bn = cout <= 32 ? 32 : cout <= 64 ? 64 : cout <= 128 ? 128 : cout <= 256 ? 256 : 0;
  if (!bn || cout % 32) return kNotEligible;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return -2;
  CUtensorMap tx, tg;
  const cuuint32_t box[4] = {32, (cuuint32_t)kWgPix, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  {
    const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)xs * 2, (cuuint64_t)W * xs * 2, (cuuint64_t)H * W * xs * 2};
    if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  {
    const cuuint64_t dims[4] = {(cuuint64_t)cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)gs * 2, (cuuint64_t)W * gs * 2, (cuuint64_t)H * W * gs * 2};
    if (enc(&tg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(gy), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  const int nblocks = 9 * (cin / 32);
  const int mtiles = (nblocks + 3) / 4;
  const long long ksteps = (long long)N * H * ((W + kWgPix - 1) / kWgPix);
  if (splits <= 0) {
    // about four CTAs per SM in all, at least 8 K steps each
    int sms = 148;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (4ll * sms + mtiles - 1) / mtiles;
    const long long cap = (ksteps + 7) / 8;
    splits = (int)(want < 1 ? 1 : (want > cap ? (cap < 1 ? 1 : cap) : want));
  }
  if (splits > 65535) splits = 65535;
  cudaError_t e;
  switch (bn) {
    case 32: e = launch_wgrad<32, 5>(tx, tg, gw, H, W, cin, cout, nblocks, mtiles, ksteps, splits, st); break;
    case 64: e = launch_wgrad<64, 4>(tx, tg, gw, H, W, cin, cout, nblocks, mtiles, ksteps, splits, st); break;
    case 128: e = launch_wgrad<128, 3>(tx, tg, gw, H, W, cin, cout, nblocks, mtiles, ksteps, splits, st); break;
    default: e = launch_wgrad<256, 2>(tx, tg, gw, H, W, cin, cout, nblocks, mtiles, ksteps, splits, st); break;
  }
  if (e != cudaSuccess) return -2;
  if (gb) {
    const long long P = (long long)N * H * W;
    const int blocks = 608;
    const long long ppb = (P + blocks - 1) / blocks;
    bias_grad_kernel<<<(int)((P + ppb - 1) / ppb), 256, cout * sizeof(float), st>>>((const bf16 *)gy, gs, gb, P,
                                                                                   cout, ppb);
    if (cudaGetLastError() != cudaSuccess) return -2;
  }
  return 0;
}

int status(int reset) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)) != cudaSuccess) return -2;
  if (reset) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_tc_status, &z, sizeof(z)) != cudaSuccess) return -2;
  }
  return (int)v;
}

}  // namespace gbnn_tc
