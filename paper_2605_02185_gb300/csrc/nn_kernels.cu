// nn_kernels.cu -- BF16 tensor-core kernels of the warm-start network.
//
// Activations are NHWC bfloat16 with an explicit channel stride (so a layer
// can read or write a channel slice of a wider buffer: the decoder's skip
// concatenations cost nothing).  Weights are [Cout][3][3][Cin] bfloat16.
// A 3x3 convolution (zero padding 1) is an implicit GEMM: M = pixels,
// N = output channels, K = 9 * Cin, computed with m16n8k16 BF16 MMAs and
// FP32 accumulation.  The forward kernel stages, per 32-channel chunk, the
// three input rows a 128-pixel tile needs (with its 1-pixel halo) and the
// chunk's weights in shared memory, and forms the nine taps by shifting the
// staged rows -- the im2col matrix is never built.  The input gradient is the
// same kernel on the output gradient with spatially flipped, channel-
// transposed weights; the weight gradient is a second implicit GEMM
// (M = Cout, N = Cin, K = pixels, per tap) with split-K partial sums added
// in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbnn.h"
#include "nn_tc.h"

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- forward / input-gradient convolution ---------------------------------
constexpr int FW_BM = 128;     // pixels per tile (one image row segment)
constexpr int FW_CK = 32;      // input channels per chunk
constexpr int FW_CKP = 40;     // padded chunk stride (bank-conflict-free ldmatrix rows)
constexpr int FW_THREADS = 128;

template <int BN>
struct FwdSmem {
  bf16 strip[3][FW_BM + 2][FW_CKP];
  bf16 wts[9][BN][FW_CKP];
};

// y[n, h, w, o] = act(b[o] + sum_{dy,dx,c} x[n, h+dy-1, w+dx-1, c] wt[o, dy, dx, c])
// act = ReLU if relu; if mask is given the result is zeroed where mask <= 0
// (the ReLU derivative of the layer that produced this layer's input).
template <int BN>
__global__ void __launch_bounds__(FW_THREADS) conv_fwd_kernel(const bf16 *__restrict__ x, int xs, const bf16 *__restrict__ wt,
                                                             const float *__restrict__ bias, bf16 *__restrict__ y, int ys,
                                                             const bf16 *__restrict__ mask, int ms, int N, int H, int W,
                                                             int cin, int cout, int relu) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FwdSmem<BN> &sm = *reinterpret_cast<FwdSmem<BN> *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * FW_BM, row = blockIdx.y;
  const int nchunks = (cout + BN - 1) / BN;
  const int n = blockIdx.z / nchunks, o0 = (blockIdx.z % nchunks) * BN;
  constexpr int NT = BN / 8;
  float acc[2][NT][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  for (int c0 = 0; c0 < cin; c0 += FW_CK) {
    // stage the three input rows of the tile (+halo), 8 channels per vector
    for (int i = tid; i < 3 * (FW_BM + 2) * (FW_CK / 8); i += FW_THREADS) {
      const int v = i % (FW_CK / 8), px = (i / (FW_CK / 8)) % (FW_BM + 2), r = i / ((FW_CK / 8) * (FW_BM + 2));
      const int hh = row + r - 1, ww = x0 + px - 1, cc = c0 + v * 8;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (hh >= 0 && hh < H && ww >= 0 && ww < W && cc < cin)
        val = *reinterpret_cast<const uint4 *>(x + (((size_t)n * H + hh) * W + ww) * xs + cc);
      *reinterpret_cast<uint4 *>(&sm.strip[r][px][v * 8]) = val;
    }
    for (int i = tid; i < 9 * BN * (FW_CK / 8); i += FW_THREADS) {
      const int v = i % (FW_CK / 8), o = (i / (FW_CK / 8)) % BN, tap = i / ((FW_CK / 8) * BN);
      const int cc = c0 + v * 8;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (o0 + o < cout && cc < cin)
        val = *reinterpret_cast<const uint4 *>(wt + ((size_t)(o0 + o) * 9 + tap) * cin + cc);
      *reinterpret_cast<uint4 *>(&sm.wts[tap][o][v * 8]) = val;
    }
    __syncthreads();
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3;
#pragma unroll
      for (int kk = 0; kk < FW_CK; kk += 16) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int q = lane >> 3, r = lane & 7;
          const int pm = warp * 32 + mt * 16 + (q & 1) * 8 + r;
          ldsm_x4(saddr(&sm.strip[dy][pm + dx][kk + (q >> 1) * 8]), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
        }
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          const int q = lane >> 3, r = lane & 7;
          uint32_t b0, b1, b2, b3;
          ldsm_x4(saddr(&sm.wts[tap][np * 16 + (q >> 1) * 8 + r][kk + (q & 1) * 8]), b0, b1, b2, b3);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
            mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
          }
        }
      }
    }
    __syncthreads();
  }
  // epilogue: bias, activation / mask, bf16 store
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int px = x0 + warp * 32 + mt * 16 + hf * 8 + g;
      if (px >= W) continue;
      const size_t pix = ((size_t)n * H + row) * W + px;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int o = o0 + nt * 8 + 2 * t;
        if (o >= cout) continue;
        float v0 = acc[mt][nt][2 * hf], v1 = acc[mt][nt][2 * hf + 1];
        if (bias) {
          v0 += bias[o];
          v1 += bias[o + 1];
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (mask) {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * ms + o);
          if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162 *>(y + pix * ys + o) = __floats2bfloat162_rn(v0, v1);
      }
    }
}

// ---- weight gradient --------------------------------------------------------
constexpr int WG_BK = 32;   // pixels per K step
constexpr int WG_BMN = 64;  // output channels x input channels per tile
constexpr int WG_P = 72;    // padded row stride
constexpr int WG_THREADS = 128;

struct WgSmem {
  bf16 g[WG_BK][WG_P];  // [pixel][cout]
  bf16 xs[WG_BK][WG_P]; // [pixel][cin], shifted by the tap
};

// gw[o, tap, c] += sum over this block's pixels of gy[p, o] x[p + shift(tap), c]
// The blocks of the centre tap and the first input-channel chunk also sum
// gy over their pixels into gb[o] (the bias gradient).
__global__ void __launch_bounds__(WG_THREADS) conv_wgrad_kernel(const bf16 *__restrict__ x, int xs,
                                                               const bf16 *__restrict__ gy, int gs,
                                                               float *__restrict__ gw, float *__restrict__ gb, int N,
                                                               int H, int W, int cin, int cout,
                                                               long long pix_per_block) {
  __shared__ __align__(128) WgSmem sm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tap = blockIdx.y, dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int ncc = (cin + WG_BMN - 1) / WG_BMN;
  const int o0 = (blockIdx.z / ncc) * WG_BMN, c0 = (blockIdx.z % ncc) * WG_BMN;
  const long long P = (long long)N * H * W;
  const long long p_begin = (long long)blockIdx.x * pix_per_block;
  const long long p_end = p_begin + pix_per_block < P ? p_begin + pix_per_block : P;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin (o, c)
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const bool do_bias = gb != nullptr && tap == 4 && c0 == 0;
  float bsum = 0.f;  // thread tid < 64: output channel o0 + tid

  for (long long p0 = p_begin; p0 < p_end; p0 += WG_BK) {
    for (int i = tid; i < WG_BK * (WG_BMN / 8); i += WG_THREADS) {
      const int v = i % (WG_BMN / 8), pr = i / (WG_BMN / 8);
      const long long p = p0 + pr;
      uint4 gv = make_uint4(0, 0, 0, 0), xv = make_uint4(0, 0, 0, 0);
      if (p < p_end) {
        const int ww = (int)(p % W), hh = (int)((p / W) % H), nn = (int)(p / ((long long)W * H));
        if (o0 + v * 8 < cout) gv = *reinterpret_cast<const uint4 *>(gy + p * gs + o0 + v * 8);
        const int h2 = hh + dy, w2 = ww + dx;
        if (c0 + v * 8 < cin && h2 >= 0 && h2 < H && w2 >= 0 && w2 < W)
          xv = *reinterpret_cast<const uint4 *>(x + (((size_t)nn * H + h2) * W + w2) * xs + c0 + v * 8);
      }
      *reinterpret_cast<uint4 *>(&sm.g[pr][v * 8]) = gv;
      *reinterpret_cast<uint4 *>(&sm.xs[pr][v * 8]) = xv;
    }
    __syncthreads();
    if (do_bias && tid < WG_BMN)
      for (int pr = 0; pr < WG_BK; ++pr) bsum += __bfloat162float(sm.g[pr][tid]);
#pragma unroll
    for (int kk = 0; kk < WG_BK; kk += 16) {
      const int q = lane >> 3, r = lane & 7;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)  // A = gy^T: rows o, k = pixels; stored [k][o]
        ldsm_x4_t(saddr(&sm.g[kk + (q >> 1) * 8 + r][wm + mt * 16 + (q & 1) * 8]), a[mt][0], a[mt][1], a[mt][2],
                  a[mt][3]);
#pragma unroll
      for (int np = 0; np < 2; ++np) {  // B = x: k = pixels, n = c; stored [k][c]
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(saddr(&sm.xs[kk + (q & 1) * 8 + r][wn + np * 16 + (q >> 1) * 8]), b0, b1, b2, b3);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
          mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
        }
      }
    }
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int o = o0 + wm + mt * 16 + hf * 8 + g;
      if (o >= cout) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = c0 + wn + nt * 8 + 2 * t;
        if (c >= cin) continue;
        float *dst = gw + ((size_t)o * 9 + tap) * cin + c;
        atomicAdd(dst, acc[mt][nt][2 * hf]);
        atomicAdd(dst + 1, acc[mt][nt][2 * hf + 1]);
      }
    }
  if (do_bias && tid < WG_BMN && o0 + tid < cout) atomicAdd(gb + o0 + tid, bsum);
}

// ---- weight gradient, all nine taps per block (32 x 32 channel tiles) ----
// For the wide, shallow layers (full resolution, <= 32 output channels) the
// per-tap kernel above re-reads every input row nine times.  Here one block
// stages a 64-pixel row segment of gy (32 output channels) and the three
// input rows around it (32 input channels, 1-pixel halo) once, and its nine
// warps -- one per tap -- each accumulate a 32 x 32 tile of that tap's
// gradient from shifted views of the staged rows.
constexpr int W9_PX = 64;
constexpr int W9_CP = 40;  // padded channel stride (conflict-free ldmatrix rows)
constexpr int W9_THREADS = 288;

struct W9Smem {
  bf16 g[W9_PX][W9_CP];              // [pixel][o]
  bf16 xs[3][W9_PX + 2][W9_CP];      // [row][pixel + halo][c]
};

__global__ void __launch_bounds__(W9_THREADS) conv_wgrad9_kernel(const bf16 *__restrict__ x, int xs,
                                                                const bf16 *__restrict__ gy, int gs,
                                                                float *__restrict__ gw, float *__restrict__ gb, int N,
                                                                int H, int W, int cin, int cout,
                                                                long long segs_per_block) {
  __shared__ __align__(128) W9Smem sm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tap = warp, dy = tap / 3, dx = tap % 3;
  const int ncc = (cin + 31) / 32;
  const int o0 = (blockIdx.y / ncc) * 32, c0 = (blockIdx.y % ncc) * 32;
  const int spr = (W + W9_PX - 1) / W9_PX;  // segments per image row
  const long long nsegs = (long long)N * H * spr;
  const long long s_begin = (long long)blockIdx.x * segs_per_block;
  const long long s_end = s_begin + segs_per_block < nsegs ? s_begin + segs_per_block : nsegs;
  const bool do_bias = gb != nullptr && c0 == 0;
  float bsum = 0.f;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  for (long long sg = s_begin; sg < s_end; ++sg) {
    const int w0 = (int)(sg % spr) * W9_PX;
    const long long r = sg / spr;
    const int h = (int)(r % H), n = (int)(r / H);
    for (int i = tid; i < W9_PX * 4; i += W9_THREADS) {  // gy: 64 pixels x 32 channels
      const int v = i & 3, px = i >> 2;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (w0 + px < W && o0 + v * 8 < cout)
        val = *reinterpret_cast<const uint4 *>(gy + (((size_t)n * H + h) * W + w0 + px) * gs + o0 + v * 8);
      *reinterpret_cast<uint4 *>(&sm.g[px][v * 8]) = val;
    }
    for (int i = tid; i < 3 * (W9_PX + 2) * 4; i += W9_THREADS) {  // x: 3 rows x 66 pixels x 32 channels
      const int v = i & 3, px = (i >> 2) % (W9_PX + 2), rr = (i >> 2) / (W9_PX + 2);
      const int hh = h + rr - 1, ww = w0 + px - 1;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (hh >= 0 && hh < H && ww >= 0 && ww < W && c0 + v * 8 < cin)
        val = *reinterpret_cast<const uint4 *>(x + (((size_t)n * H + hh) * W + ww) * xs + c0 + v * 8);
      *reinterpret_cast<uint4 *>(&sm.xs[rr][px][v * 8]) = val;
    }
    __syncthreads();
    if (do_bias && tid < 32)
      for (int px = 0; px < W9_PX; ++px) bsum += __bfloat162float(sm.g[px][tid]);
#pragma unroll
    for (int kk = 0; kk < W9_PX; kk += 16) {
      const int q = lane >> 3, rw = lane & 7;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)  // A = gy^T (m = o, k = pixel), stored [pixel][o]
        ldsm_x4_t(saddr(&sm.g[kk + (q >> 1) * 8 + rw][mt * 16 + (q & 1) * 8]), a[mt][0], a[mt][1], a[mt][2],
                  a[mt][3]);
#pragma unroll
      for (int np = 0; np < 2; ++np) {  // B = shifted x (k = pixel, n = c), stored [pixel][c]
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(saddr(&sm.xs[dy][kk + (q & 1) * 8 + rw + dx][np * 16 + (q >> 1) * 8]), b0, b1, b2, b3);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
          mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
        }
      }
    }
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int o = o0 + mt * 16 + hf * 8 + g;
      if (o >= cout) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = c0 + nt * 8 + 2 * t;
        if (c >= cin) continue;
        float *dst = gw + ((size_t)o * 9 + tap) * cin + c;
        atomicAdd(dst, acc[mt][nt][2 * hf]);
        atomicAdd(dst + 1, acc[mt][nt][2 * hf + 1]);
      }
    }
  if (do_bias && tid < 32 && o0 + tid < cout) atomicAdd(gb + o0 + tid, bsum);
}

// wf[c, dy, dx, o] = w[o, 2-dy, 2-dx, c]
__global__ void flip_weights_kernel(const bf16 *__restrict__ w, bf16 *__restrict__ wf, int cout, int cin) {
  const long long n = (long long)cout * 9 * cin;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % cin), tap = (int)((i / cin) % 9), o = (int)(i / ((long long)cin * 9));
    wf[((size_t)c * 9 + (8 - tap)) * cout + o] = w[i];
  }
}

// ---- elementwise ----------------------------------------------------------
__global__ void avgpool2_kernel(const bf16 *__restrict__ x, int xs, bf16 *__restrict__ y, int ys, int N, int H, int W,
                                int C) {  // H, W of the input
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)N * Ho * Wo * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int wo = (int)(p % Wo), ho = (int)((p / Wo) % Ho), nn = (int)(p / ((long long)Wo * Ho));
    const size_t b = (((size_t)nn * H + 2 * ho) * W + 2 * wo) * xs + c;
    const float s = __bfloat162float(x[b]) + __bfloat162float(x[b + xs]) + __bfloat162float(x[b + (size_t)W * xs]) +
                    __bfloat162float(x[b + (size_t)W * xs + xs]);
    y[p * ys + c] = __float2bfloat16_rn(0.25f * s);
  }
}

// gx (+)= 0.25 gy[parent], zeroed where mask <= 0 if a mask is given
__global__ void avgpool2_bwd_kernel(const bf16 *__restrict__ gy, int gs, bf16 *__restrict__ gx, int gxs,
                                    const bf16 *__restrict__ mask, int ms, int N, int H, int W, int C,
                                    int accumulate) {  // H, W of the input
  const long long n = (long long)N * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), nn = (int)(p / ((long long)W * H));
    const size_t q = (((size_t)nn * (H / 2) + h / 2) * (W / 2) + w / 2) * gs + c;
    float v = 0.25f * __bfloat162float(gy[q]);
    if (mask && !(__bfloat162float(mask[p * ms + c]) > 0.f)) v = 0.f;
    if (accumulate) v += __bfloat162float(gx[p * gxs + c]);
    gx[p * gxs + c] = __float2bfloat16_rn(v);
  }
}

__global__ void upsample2_kernel(const bf16 *__restrict__ x, int xs, bf16 *__restrict__ y, int ys, int N, int H, int W,
                                 int C) {  // H, W of the input
  const long long n = (long long)N * (2 * H) * (2 * W) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int w = (int)(p % (2 * W)), h = (int)((p / (2 * W)) % (2 * H)), nn = (int)(p / (4ll * W * H));
    y[p * ys + c] = x[(((size_t)nn * H + h / 2) * W + w / 2) * xs + c];
  }
}

__global__ void upsample2_bwd_kernel(const bf16 *__restrict__ gy, int gs, bf16 *__restrict__ gx, int gxs, int N, int H,
                                     int W, int C) {  // H, W of the (small) input
  const long long n = (long long)N * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), nn = (int)(p / ((long long)W * H));
    const size_t b = (((size_t)nn * 2 * H + 2 * h) * 2 * W + 2 * w) * gs + c;
    const float s = __bfloat162float(gy[b]) + __bfloat162float(gy[b + gs]) +
                    __bfloat162float(gy[b + (size_t)2 * W * gs]) + __bfloat162float(gy[b + (size_t)2 * W * gs + gs]);
    gx[p * gxs + c] = __float2bfloat16_rn(s);
  }
}

// loss partials: sum over elements of wgt * (pred - target)^2; grad = 2 wgt (pred - target) * scale
__global__ void mse_kernel(const bf16 *__restrict__ pred, int ps, const float *__restrict__ target,
                           const float *__restrict__ weight, bf16 *__restrict__ grad, int gs, long long P, int C,
                           float scale, float *__restrict__ loss_sum) {
  __shared__ float red[256];
  float acc = 0.f;
  const long long n = P * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const float wgt = weight ? weight[p] : 1.f;
    const float d = __bfloat162float(pred[p * ps + c]) - target[i];
    acc += wgt * d * d;
    if (grad) grad[p * gs + c] = __float2bfloat16_rn(2.f * wgt * d * scale);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss_sum, red[0]);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ p16, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

// network input of one sample: [solid, Re feature, sin(phase), cos(phase),
// x/W, y/H, cos(k (x - x0) - phase), sin(k (x - x0) - phase)]; the last two
// are a travelling-wave basis (wavenumber k per node) for the wake
__global__ void encode_input_kernel(const uint8_t *__restrict__ solid, float re_feature, float phase, float k,
                                    float x0, int H, int W, bf16 *__restrict__ x) {
  const long long n = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(i % W), h = (int)(i / W);
    __align__(16) bf16 v[8];
    const float arg = k * ((float)w - x0) - phase;
    v[0] = __float2bfloat16_rn(solid[i] ? 1.f : 0.f);
    v[1] = __float2bfloat16_rn(re_feature);
    v[2] = __float2bfloat16_rn(sinf(phase));
    v[3] = __float2bfloat16_rn(cosf(phase));
    v[4] = __float2bfloat16_rn((float)w / (float)W);
    v[5] = __float2bfloat16_rn((float)h / (float)H);
    v[6] = __float2bfloat16_rn(cosf(arg));
    v[7] = __float2bfloat16_rn(sinf(arg));
    *reinterpret_cast<uint4 *>(x + i * 8) = *reinterpret_cast<const uint4 *>(v);
  }
}

// training target [P][3] = ((rho - 1) / rho_scale, (u - U) / vel_scale,
// v / vel_scale), weight = fluid; the velocity is taken relative to the free
// stream so that the network's bfloat16 output resolves the deviations
__global__ void encode_target_kernel(const float *__restrict__ rho, const float *__restrict__ u,
                                     const float *__restrict__ v, const uint8_t *__restrict__ solid, long long P,
                                     float U, float vel_scale, float rho_scale, float *__restrict__ target,
                                     float *__restrict__ weight) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    target[3 * i] = (rho[i] - 1.f) / rho_scale;
    target[3 * i + 1] = (u[i] - U) / vel_scale;
    target[3 * i + 2] = v[i] / vel_scale;
    if (weight) weight[i] = solid[i] ? 0.f : 1.f;
  }
}

// prediction -> fields (inverse of the target map); solid nodes rest at rho = 1
__global__ void decode_output_kernel(const bf16 *__restrict__ out, int os, const uint8_t *__restrict__ solid,
                                     long long P, float U, float vel_scale, float rho_scale, float *__restrict__ rho,
                                     float *__restrict__ u, float *__restrict__ v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    const bool s = solid[i] != 0;
    rho[i] = s ? 1.f : 1.f + rho_scale * __bfloat162float(out[i * os]);
    u[i] = s ? 0.f : U + vel_scale * __bfloat162float(out[i * os + 1]);
    v[i] = s ? 0.f : vel_scale * __bfloat162float(out[i * os + 2]);
  }
}

int g_conv_impl = GBNN_IMPL_AUTO;

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 * 16 ? 65535 * 16 : b));
}

int err(cudaError_t e) { return e == cudaSuccess ? 0 : -2; }

}  // namespace

extern "C" {

int gbnn_set_conv_impl(int impl) {
  if (impl < GBNN_IMPL_AUTO || impl > GBNN_IMPL_TCGEN05) return -1;
  g_conv_impl = impl;
  return 0;
}

int gbnn_conv_impl(void) { return g_conv_impl; }

int gbnn_status(int reset) { return gbnn_tc::status(reset); }

int gbnn_conv3x3_fwd(const void *x, int x_cstride, const void *w, const float *bias, void *y, int y_cstride,
                     const void *mask, int mask_cstride, int N, int H, int W, int cin, int cout, int relu, void *stream) {
  if (!x || !w || !y || N <= 0 || H <= 0 || W <= 0 || cin <= 0 || cout <= 0) return -1;
  if (cin % 8 || cout % 2 || x_cstride % 8 || y_cstride % 2 || x_cstride < cin || y_cstride < cout) return -1;
  if (mask && (mask_cstride % 2 || mask_cstride < cout)) return -1;
  if ((uintptr_t)x % 16 || (uintptr_t)w % 16) return -1;
  const cudaStream_t st = (cudaStream_t)stream;
  if (g_conv_impl != GBNN_IMPL_MMA_SYNC) {
    const int rc = gbnn_tc::conv_fwd(x, x_cstride, w, bias, y, y_cstride, mask, mask_cstride, N, H, W, cin, cout, relu,
                                     st);
    if (rc != gbnn_tc::kNotEligible) return rc;
    if (g_conv_impl == GBNN_IMPL_TCGEN05) return -1;  // required, but this shape is not taken
  }
  const int bn = cout <= 16 ? 16 : (cout <= 32 ? 32 : 64);
  const int nch = (cout + bn - 1) / bn;
  dim3 grid((W + FW_BM - 1) / FW_BM, H, N * nch);
  if ((long long)N * nch > 65535) return -1;
  const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w, *mb = (const bf16 *)mask;
  bf16 *yb = (bf16 *)y;
  if (bn == 16) {
    cudaFuncSetAttribute(conv_fwd_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem<16>));
    conv_fwd_kernel<16><<<grid, FW_THREADS, sizeof(FwdSmem<16>), st>>>(xb, x_cstride, wb, bias, yb, y_cstride, mb,
                                                                       mask_cstride, N, H, W, cin, cout, relu);
  } else if (bn == 32) {
    cudaFuncSetAttribute(conv_fwd_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem<32>));
    conv_fwd_kernel<32><<<grid, FW_THREADS, sizeof(FwdSmem<32>), st>>>(xb, x_cstride, wb, bias, yb, y_cstride, mb,
                                                                       mask_cstride, N, H, W, cin, cout, relu);
  } else {
    cudaFuncSetAttribute(conv_fwd_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem<64>));
    conv_fwd_kernel<64><<<grid, FW_THREADS, sizeof(FwdSmem<64>), st>>>(xb, x_cstride, wb, bias, yb, y_cstride, mb,
                                                                       mask_cstride, N, H, W, cin, cout, relu);
  }
  return err(cudaGetLastError());
}

int gbnn_flip_weights(const void *w, void *wf, int cout, int cin, void *stream) {
  if (!w || !wf || cout <= 0 || cin <= 0) return -1;
  const long long n = (long long)cout * 9 * cin;
  flip_weights_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)w, (bf16 *)wf, cout, cin);
  return err(cudaGetLastError());
}

int gbnn_conv3x3_dgrad(const void *gy, int gy_cstride, const void *w_flipped, void *gx, int gx_cstride,
                       const void *mask, int mask_cstride, int N, int H, int W, int cin, int cout, void *stream) {
  // input gradient = convolution of gy with the flipped, transposed weights
  return gbnn_conv3x3_fwd(gy, gy_cstride, w_flipped, nullptr, gx, gx_cstride, mask, mask_cstride, N, H, W, cout, cin,
                          0, stream);
}

int gbnn_conv3x3_wgrad(const void *x, int x_cstride, const void *gy, int gy_cstride, float *gw, float *gb, int N, int H,
                       int W, int cin, int cout, int splits, void *stream) {
  if (!x || !gy || !gw || N <= 0 || H <= 0 || W <= 0 || cin % 8 || cout % 8 || x_cstride % 8 || gy_cstride % 8)
    return -1;
  const cudaStream_t st = (cudaStream_t)stream;
  if (g_conv_impl != GBNN_IMPL_MMA_SYNC) {
    const int rc = gbnn_tc::conv_wgrad(x, x_cstride, gy, gy_cstride, gw, gb, N, H, W, cin, cout, splits, st);
    if (rc != gbnn_tc::kNotEligible) return rc;
    if (g_conv_impl == GBNN_IMPL_TCGEN05) return -1;
  }
  const long long P = (long long)N * H * W;
  if (cout <= 32) {  // wide, shallow layer: all nine taps per block
    const long long nsegs = (long long)N * H * ((W + W9_PX - 1) / W9_PX);
    const int blocks = splits > 0 ? splits : 608;
    const long long spb = (nsegs + blocks - 1) / blocks;
    const int nb = (int)((nsegs + spb - 1) / spb);
    const int ny = ((cout + 31) / 32) * ((cin + 31) / 32);
    conv_wgrad9_kernel<<<dim3(nb, ny), W9_THREADS, 0, st>>>((const bf16 *)x, x_cstride, (const bf16 *)gy, gy_cstride,
                                                            gw, gb, N, H, W, cin, cout, spb);
    return err(cudaGetLastError());
  }
  if (splits <= 0) splits = 304;
  long long ppb = (P + splits - 1) / splits;
  ppb = (ppb + WG_BK - 1) / WG_BK * WG_BK;
  const int blocks = (int)((P + ppb - 1) / ppb);
  const int nz = ((cout + WG_BMN - 1) / WG_BMN) * ((cin + WG_BMN - 1) / WG_BMN);
  conv_wgrad_kernel<<<dim3(blocks, 9, nz), WG_THREADS, 0, st>>>((const bf16 *)x, x_cstride, (const bf16 *)gy,
                                                                gy_cstride, gw, gb, N, H, W, cin, cout, ppb);
  return err(cudaGetLastError());
}

int gbnn_avgpool2(const void *x, int x_cstride, void *y, int y_cstride, int N, int H, int W, int C, void *stream) {
  if (H % 2 || W % 2) return -1;
  const long long n = (long long)N * (H / 2) * (W / 2) * C;
  avgpool2_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, (bf16 *)y, y_cstride, N, H,
                                                                  W, C);
  return err(cudaGetLastError());
}

int gbnn_avgpool2_bwd(const void *gy, int gy_cstride, void *gx, int gx_cstride, const void *mask, int mask_cstride,
                      int N, int H, int W, int C, int accumulate, void *stream) {
  if (H % 2 || W % 2) return -1;
  const long long n = (long long)N * H * W * C;
  avgpool2_bwd_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)gy, gy_cstride, (bf16 *)gx,
                                                                      gx_cstride, (const bf16 *)mask, mask_cstride, N,
                                                                      H, W, C, accumulate);
  return err(cudaGetLastError());
}

int gbnn_upsample2(const void *x, int x_cstride, void *y, int y_cstride, int N, int H, int W, int C, void *stream) {
  const long long n = (long long)N * 4 * H * W * C;
  upsample2_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, (bf16 *)y, y_cstride, N,
                                                                   H, W, C);
  return err(cudaGetLastError());
}

int gbnn_upsample2_bwd(const void *gy, int gy_cstride, void *gx, int gx_cstride, int N, int H, int W, int C,
                       void *stream) {
  const long long n = (long long)N * H * W * C;
  upsample2_bwd_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)gy, gy_cstride, (bf16 *)gx,
                                                                       gx_cstride, N, H, W, C);
  return err(cudaGetLastError());
}

int gbnn_mse(const void *pred, int pred_cstride, const float *target, const float *weight, void *grad,
             int grad_cstride, long long P, int C, float scale, float *loss_sum, void *stream) {
  if (!pred || !target || !loss_sum || P <= 0 || C <= 0) return -1;
  const long long n = P * C;
  const int blocks = grid_for(n) < 4096 ? grid_for(n) : 4096;
  mse_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const bf16 *)pred, pred_cstride, target, weight, (bf16 *)grad,
                                                        grad_cstride, P, C, scale, loss_sum);
  return err(cudaGetLastError());
}

int gbnn_encode_input(const uint8_t *solid, float re_feature, float phase, float wave_k, float wave_x0, int H, int W,
                      void *x, void *stream) {
  if (!solid || !x || H <= 0 || W <= 0 || ((uintptr_t)x % 16)) return -1;
  encode_input_kernel<<<grid_for((long long)H * W), 256, 0, (cudaStream_t)stream>>>(
      solid, re_feature, phase, wave_k, wave_x0, H, W, (bf16 *)x);
  return err(cudaGetLastError());
}

int gbnn_encode_target(const float *rho, const float *u, const float *v, const uint8_t *solid, long long P, float U,
                       float vel_scale, float rho_scale, float *target, float *weight, void *stream) {
  if (!rho || !u || !v || !solid || !target || P <= 0 || !(vel_scale > 0.f) || !(rho_scale > 0.f)) return -1;
  encode_target_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(rho, u, v, solid, P, U, vel_scale, rho_scale,
                                                                       target, weight);
  return err(cudaGetLastError());
}

int gbnn_decode_output(const void *out, int out_cstride, const uint8_t *solid, long long P, float U, float vel_scale,
                       float rho_scale, float *rho, float *u, float *v, void *stream) {
  if (!out || !solid || !rho || !u || !v || P <= 0 || out_cstride < 3) return -1;
  decode_output_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>((const bf16 *)out, out_cstride, solid, P, U,
                                                                       vel_scale, rho_scale, rho, u, v);
  return err(cudaGetLastError());
}

int gbnn_fill_zero(void *ptr, size_t bytes, void *stream) {
  if (!ptr) return -1;
  return err(cudaMemsetAsync(ptr, 0, bytes, (cudaStream_t)stream));
}

int gbnn_adam(float *param, const float *grad, float *m, float *v, void *param_bf16, long long n, float lr,
              float beta1, float beta2, float eps, int t, void *stream) {
  if (!param || !grad || !m || !v || n <= 0 || t <= 0) return -1;
  float c1 = 1.f, c2 = 1.f, p1 = 1.f, p2 = 1.f;
  for (int i = 0; i < t && i < 100000; ++i) {
    p1 *= beta1;
    p2 *= beta2;
  }
  c1 = 1.f - p1;
  c2 = 1.f - p2;
  adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, (bf16 *)param_bf16, n, lr, beta1, beta2,
                                                              eps, c1, c2);
  return err(cudaGetLastError());
}

}  // extern "C"
