// ns_cnn.cu -- the learned closure's network: four 3x3 convolutions on a
// periodic 2D grid (channels 1 -> C -> C -> C -> 1, GELU after the first
// three), BF16 activations and weights, FP32 accumulation, with hand-written
// forward, backward and Adam kernels.
//
// Data layout: [batch][channel][y][x], periodic in y and x.  Parameters are
// one flat FP32 array (the Adam master copy) in the order W0 b0 W1 b1 W2 b2
// W3 b3, W_l as [Cout][Cin][3][3]; a BF16 copy of every W_l feeds the
// kernels.  Layer l computes z_l = conv(a_l, W_l) + b_l with
// conv(a, W)[co](p) = sum_ci sum_{dy,dx in -1..1} W[co][ci][dy+1][dx+1] a[ci](p + (dy, dx)),
// a_{l+1} = GELU(z_l) (exact, erf form) for l < 3, output y = z_3.
// Training minimises the mean squared error to a target field.
//
// Kernels: conv_fwd (one block per 16x16 tile and image: the input halo tile
// and all weights in shared memory, one output pixel per thread for every
// output channel); conv_bwd_data (the same kernel on the flipped, transposed
// weights, with the GELU derivative of the layer below fused in);
// conv_bwd_weight (each block sums a 64x64 region in 16x16 sub-tiles and adds
// its partial sums to the FP32 gradient with atomics: order-dependent in the
// last bits, not bitwise reproducible); elementwise MSE and Adam.  The 32 ->
// 32 convolutions of widths that are multiples of 128 (forward, data and
// weight gradients) run on the tensor cores instead (conv32_tc,
// conv32_wgrad_tc below).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_tc.cuh"

namespace {

using bf16 = __nv_bfloat16;
constexpr int TILE = 16;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752440f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752440f)) + z * 0.39894228040143267794f * expf(-0.5f * z * z);
}

template <typename T>
__device__ __forceinline__ float ldf(const T *p) {
  return (float)*p;
}
template <>
__device__ __forceinline__ float ldf<bf16>(const bf16 *p) {
  return __bfloat162float(*p);
}

enum Epi { EPI_LINEAR = 0, EPI_GELU = 1, EPI_GELU_BWD = 2 };

// out[b][co][p] = epi( sum_ci sum_k w[co][ci][k] x[b][ci][p + off(k)] + bias[co] )
//   EPI_LINEAR  : out = acc (float)
//   EPI_GELU    : zout = bf16(acc), out = bf16(GELU(acc))
//   EPI_GELU_BWD: out = acc * GELU'(zin[b][co][p])  (float)
template <int CIN, int COUT, int EPI, typename TIN, typename TOUT>
__global__ void __launch_bounds__(TILE *TILE) conv_fwd(const TIN *__restrict__ x, const bf16 *__restrict__ w,
                                                       const float *__restrict__ bias, const bf16 *__restrict__ zin,
                                                       bf16 *__restrict__ zout, TOUT *__restrict__ out, int H, int W) {
  extern __shared__ float4 csm4[];
  float *csm = reinterpret_cast<float *>(csm4);
  float *sw = csm;                       // [CIN][9][COUT]: the COUT weights of a tap are contiguous
  float *sx = csm + COUT * CIN * 9;      // [CIN][18][18]
  const int b = blockIdx.z;
  const int y0 = blockIdx.y * TILE, x0 = blockIdx.x * TILE;
  for (int i = threadIdx.x; i < COUT * CIN * 9; i += blockDim.x) {
    const int co = i / (CIN * 9), r = i % (CIN * 9);  // r = ci * 9 + k
    sw[r * COUT + co] = __bfloat162float(w[i]);
  }
  const long long img = (long long)H * W;
  for (int i = threadIdx.x; i < CIN * 18 * 18; i += blockDim.x) {
    const int ci = i / 324, r = i % 324, yy = r / 18, xx = r % 18;
    const int gy = (y0 + yy - 1 + H) % H, gx = (x0 + xx - 1 + W) % W;
    sx[i] = ldf(x + ((long long)b * CIN + ci) * img + (long long)gy * W + gx);
  }
  __syncthreads();
  const int ty = threadIdx.x / TILE, tx = threadIdx.x % TILE;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float v = sx[ci * 324 + (ty + k / 3) * 18 + tx + k % 3];
      const float *wk = sw + (ci * 9 + k) * COUT;
      if constexpr (COUT % 4 == 0) {  // one broadcast 16-byte load per four channels
#pragma unroll
        for (int q = 0; q < COUT / 4; ++q) {
          const float4 c4 = reinterpret_cast<const float4 *>(wk)[q];
          acc[4 * q] = fmaf(c4.x, v, acc[4 * q]);
          acc[4 * q + 1] = fmaf(c4.y, v, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(c4.z, v, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(c4.w, v, acc[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wk[co], v, acc[co]);
      }
    }
  }
  const long long p = (long long)(y0 + ty) * W + x0 + tx;
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    const long long o = ((long long)b * COUT + co) * img + p;
    if (EPI == EPI_GELU) {
      zout[o] = __float2bfloat16(acc[co]);
      out[o] = (TOUT)__float2bfloat16(gelu_f(acc[co]));
    } else if (EPI == EPI_GELU_BWD) {
      out[o] = (TOUT)(acc[co] * gelu_d(__bfloat162float(zin[o])));
    } else {
      out[o] = (TOUT)acc[co];
    }
  }
}

// ------------------------------------------- 32 -> 32 on the tensor cores ---
// The same convolution as conv_fwd<32, 32, EPI> as an implicit GEMM on
// tcgen05: per image row segment of 128 pixels, D[pixel][co] = sum over the 9
// taps of A_tap[pixel][ci] B_tap[ci][co] with A_tap(p, ci) = x[ci](p + off(tap))
// and B_tap(ci, co) = w[co][ci][tap]; M = 128 pixels, N = 32, K = 32 per tap
// (two MMAs of K = 16), FP32 accumulation in tensor memory.  BF16 inputs are
// exact operands; FP32 inputs (the data gradient) are split x = hi + lo into
// two BF16 operands and multiplied separately (relative error ~2^-17).
//
// A block owns a strip of 128 columns of one image over a range of rows and
// walks down it: a ring of four input rows lives in shared memory as
// [slot][channel chunk c][pixel q][8 channels] (16 bytes per (c, q), halo
// pixels q = 0 and 129 wrap periodically), so the A operand of a tap is the
// K-major descriptor at slot (y + dy) mod 4, pixel 1 + dx: leading byte
// offset = the chunk stride (along K), stride byte offset = 128 (8 pixels
// along M).  Row y + 1 is loaded while the MMAs of row y run; the tensor
// memory holds two accumulators, so the epilogue of row y - 1 (bias, GELU or
// GELU', planar stores) overlaps the MMAs of row y.  One thread issues the
// MMAs and commits them to the mbarrier of their accumulator; every wait is
// bounded (on expiry the block records code 3 in the error word and leaves).
namespace ctc {
constexpr int kQ = 130;                        // pixels of a ring row (128 + halo)
constexpr unsigned kChunk = kQ * 16;           // bytes of one channel chunk of a row
constexpr unsigned kSlot = 4 * kChunk;         // one ring row: 4 chunks of 8 channels
constexpr unsigned kRing = 4 * kSlot;          // four rows
constexpr unsigned kWB = 9 * 32 * 32 * 2;      // B operands of the 9 taps
constexpr unsigned kIdesc = nsk::tc::idesc_bf16(128, 32, false);
__host__ __device__ constexpr unsigned smem_bytes(bool split) { return kWB + (split ? 2 : 1) * kRing + 128; }
// byte offset of w[co][ci][tap] in the B tiles: K-major [tap][co / 8][ci / 8][co % 8][ci % 8]
__device__ __forceinline__ unsigned woff(int tap, int co, int ci) {
  return (unsigned)(tap * 2048 + (co >> 3) * 512 + (ci >> 3) * 128 + (co & 7) * 16 + (ci & 7) * 2);
}
}  // namespace ctc

constexpr int kConvThreads = 256;  // two threads per tensor-memory lane (pixel)

// One ring row (channels 0..31 at pixels x0 - 1 .. x0 + 128 of row yy, both
// ends wrapped) gathered in two phases, so that the global loads of a row are
// in flight while the block works on earlier rows: issue() loads this
// thread's items (chunk c, pixel q) into registers, store() writes them to the
// ring slot as 16-byte [chunk][pixel][8 channels] units (hi and lo for an
// FP32 input).
template <typename TIN>
struct RowGather {
  static constexpr int kItems = (4 * ctc::kQ + kConvThreads - 1) / kConvThreads;
  float v[kItems][8];
  int yy = 0;
  __device__ __forceinline__ void issue(const TIN *__restrict__ x, int b, int x0, int row, int H, int W) {
    yy = row;
    const int gy = ((row % H) + H) % H;
    const long long img = (long long)H * W;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const int i = threadIdx.x + kConvThreads * it;
      if (i < 4 * ctc::kQ) {
        const int c = i / ctc::kQ, q = i % ctc::kQ;
        int gx = x0 - 1 + q;
        gx = gx < 0 ? gx + W : (gx >= W ? gx - W : gx);
        const TIN *src = x + ((long long)b * 32 + 8 * c) * img + (long long)gy * W + gx;
#pragma unroll
        for (int j = 0; j < 8; ++j) v[it][j] = ldf(src + j * img);
      }
    }
  }
  __device__ __forceinline__ void store(unsigned char *ring) const {
    namespace tc = nsk::tc;
    const int slot = yy & 3;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const int i = threadIdx.x + kConvThreads * it;
      if (i < 4 * ctc::kQ) {
        const int c = i / ctc::kQ, q = i % ctc::kQ;
        const unsigned o = slot * ctc::kSlot + c * ctc::kChunk + q * 16;
        uint4 hi, lo;
        tc::split2(v[it][0], v[it][1], hi.x, lo.x);
        tc::split2(v[it][2], v[it][3], hi.y, lo.y);
        tc::split2(v[it][4], v[it][5], hi.z, lo.z);
        tc::split2(v[it][6], v[it][7], hi.w, lo.w);
        *reinterpret_cast<uint4 *>(ring + o) = hi;  // exact for BF16 inputs (lo = 0)
        if constexpr (sizeof(TIN) == 4) *reinterpret_cast<uint4 *>(ring + ctc::kRing + o) = lo;
      }
    }
  }
};

template <int EPI, typename TIN, typename TOUT>
__global__ void __launch_bounds__(kConvThreads) conv32_tc(const TIN *__restrict__ x, const bf16 *__restrict__ w,
                                                          const float *__restrict__ bias,
                                                          const bf16 *__restrict__ zin, bf16 *__restrict__ zout,
                                                          TOUT *__restrict__ out, int H, int W, int rows_per_block,
                                                          int *err) {
  using namespace ctc;
  namespace tc = nsk::tc;
  constexpr bool SPLIT = sizeof(TIN) == 4;
  extern __shared__ __align__(128) unsigned char csmb[];
  unsigned char *wb = csmb, *ring = csmb + kWB;  // ring hi, then ring lo (SPLIT)
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int strips = W / 128, segs = (H + rows_per_block - 1) / rows_per_block;
  const int b = blockIdx.x / (strips * segs), rem = blockIdx.x % (strips * segs);
  const int x0 = (rem / segs) * 128, y0 = (rem % segs) * rows_per_block;
  const int y1 = min(H, y0 + rows_per_block);
  const long long img = (long long)H * W;
  const unsigned sbase = nsk::smem_addr(csmb);
  for (int i = tid; i < 9 * 32 * 32; i += kConvThreads) {
    const int co = i / 288, r = i % 288, ci = r / 9, tap = r % 9;  // w[co][ci][tap]
    *reinterpret_cast<bf16 *>(wb + woff(tap, co, ci)) = w[i];
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 64);
  if (tid == 0) {
    nsk::mbar_init(&bars[0], 1);
    nsk::mbar_init(&bars[1], 1);
  }
  // epilogue of output row yy from accumulator buf: this thread = pixel
  // x0 + tid % 128 (tensor-memory lane), output channels 16 (tid / 128) + 0..15
  auto epilogue = [&](int yy, int buf) {
    const int px = tid & 127, c0 = (tid >> 7) * 16;
    float acc[16];
    tc::tmem_ld<16>(tslot + ((unsigned)((warp & 3) * 32) << 16) + buf * 32 + c0, acc);
    tc::tmem_wait_ld();
    const long long p = (long long)yy * W + x0 + px;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int co = c0 + j;
      const long long o = ((long long)b * 32 + co) * img + p;
      if (EPI == EPI_GELU) {
        const float v = acc[j] + (bias ? bias[co] : 0.0f);
        zout[o] = __float2bfloat16(v);
        out[o] = (TOUT)__float2bfloat16(gelu_f(v));
      } else if (EPI == EPI_GELU_BWD) {
        out[o] = (TOUT)(acc[j] * gelu_d(__bfloat162float(zin[o])));
      } else {
        out[o] = (TOUT)(acc[j] + (bias ? bias[co] : 0.0f));
      }
    }
  };
  RowGather<TIN> g;
  g.issue(x, b, x0, y0 - 1, H, W);
  g.store(ring);
  g.issue(x, b, x0, y0, H, W);
  g.store(ring);
  g.issue(x, b, x0, y0 + 1, H, W);
  unsigned ph[2] = {0u, 0u};
  bool bad = false;
  for (int y = y0; y < y1; ++y) {
    g.store(ring);  // row y + 1; its slot was last read by the MMAs of row y - 3, long completed
    if (y + 2 <= y1) g.issue(x, b, x0, y + 2, H, W);  // in flight during this row's MMAs and epilogue
    tc::fence_async_smem();
    tc::fence_before();
    if (__syncthreads_or(bad)) break;  // ring rows visible; epilogue reads of this accumulator done
    tc::fence_after();
    const int buf = y & 1;
    if (tid == 0) {
      const unsigned d = tslot + buf * 32;
      int n = 0;
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const unsigned a0 = sbase + kWB + ((y + dy) & 3) * kSlot + (1 + dx) * 16;
#pragma unroll
        for (int part = 0; part < (SPLIT ? 2 : 1); ++part)
#pragma unroll
          for (int kh = 0; kh < 2; ++kh) {
            const unsigned a = a0 + part * kRing + kh * 2 * kChunk;
            const unsigned bo = sbase + tap * 2048 + kh * 256;
            tc::mma(d, tc::sdesc(a, kChunk, 128), tc::sdesc(bo, 128, 512), kIdesc, n++ != 0);
          }
      }
      tc::commit(&bars[buf]);
    }
    if (y > y0) {
      const int pb = (y - 1) & 1;
      bad |= !nsk::mbar_wait_bounded(&bars[pb], ph[pb]);
      ph[pb] ^= 1u;
      tc::fence_after();
      if (!bad) epilogue(y - 1, pb);
    }
  }
  // the last row
  if (!bad && y1 > y0) {
    const int pb = (y1 - 1) & 1;
    bad |= !nsk::mbar_wait_bounded(&bars[pb], ph[pb]);
    tc::fence_after();
    if (!bad) epilogue(y1 - 1, pb);
  }
  if (bad) {
    if (tid == 0) atomicExch(err, 3);
    // MMAs still in flight may write the accumulators: a last bounded wait on both
    nsk::mbar_wait_bounded(&bars[0], ph[0]);
    nsk::mbar_wait_bounded(&bars[1], ph[1]);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tslot, 64);
}

// Weight gradient of a 32 -> 32 layer on the tensor cores:
//   dw[co][ci][tap] += sum_p dz[co](p) a[ci](p + off(tap)),  db[co] += sum_p dz[co](p)
// per tap a GEMM D_tap[co][ci] = sum over pixels (K) of A[co][p] B_tap[p][ci],
// both operands MN-major (8 channels contiguous per pixel): A from the
// split dz row ([co chunk][pixel][8 co], hi and lo), B_tap from the ring of
// input rows at slot (y + dy) mod 4, pixel 1 + dx (the layout of conv32_tc).
// M = 128 is the smallest MMA height here: rows 0..31 of D are the 32 output
// channels, rows 32..127 read other (in-bounds) shared memory and are
// discarded (a row of D depends only on its own row of A).  The nine
// 32-column accumulators (288 tensor-memory columns) sum over all rows of the
// block's strip; the next row's loads overlap the MMAs of the current one.
namespace ctc {
constexpr unsigned kDz = 128 * 16 * 4;                      // one split part of a dz row: 4 chunks x 128 pixels
constexpr unsigned kWgSmem = 4 * kDz + kRing + 128;         // dz hi / lo, two buffers each, then the ring
constexpr unsigned kIdescW = nsk::tc::idesc_bf16(128, 32, true) | (1u << 16);  // A and B MN-major
}  // namespace ctc

__global__ void __launch_bounds__(kConvThreads) conv32_wgrad_tc(const bf16 *__restrict__ a,
                                                                const float *__restrict__ dz, float *__restrict__ dw,
                                                                float *__restrict__ db, int H, int W,
                                                                int rows_per_block, int *err) {
  using namespace ctc;
  namespace tc = nsk::tc;
  extern __shared__ __align__(128) unsigned char csmb[];
  unsigned char *dzs = csmb, *ring = csmb + 4 * kDz;  // dzs: [buffer][part][chunk][pixel][8]
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int px = tid & 127, c0 = (tid >> 7) * 16;  // this thread's pixel and dz channels c0 .. c0 + 15
  const int strips = W / 128, segs = (H + rows_per_block - 1) / rows_per_block;
  const int b = blockIdx.x / (strips * segs), rem = blockIdx.x % (strips * segs);
  const int x0 = (rem / segs) * 128, y0 = (rem % segs) * rows_per_block;
  const int y1 = min(H, y0 + rows_per_block);
  const long long img = (long long)H * W;
  const unsigned sbase = nsk::smem_addr(csmb);
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (tid == 0) nsk::mbar_init(&bar, 1);
  float bacc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) bacc[i] = 0.0f;
  // dz row yy: issued into registers, stored (split) into buffer yy & 1
  float dv[16];
  int dyy = 0;
  auto issue_dz = [&](int yy) {
    dyy = yy;
    const float *src = dz + ((long long)b * 32 + c0) * img + (long long)yy * W + x0 + px;
#pragma unroll
    for (int j = 0; j < 16; ++j) dv[j] = src[j * img];
  };
  auto store_dz = [&]() {
    unsigned char *base = dzs + (dyy & 1) * 2 * kDz;
#pragma unroll
    for (int j = 0; j < 16; ++j) bacc[j] += dv[j];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float *v = dv + 8 * h;
      uint4 hi, lo;
      tc::split2(v[0], v[1], hi.x, lo.x);
      tc::split2(v[2], v[3], hi.y, lo.y);
      tc::split2(v[4], v[5], hi.z, lo.z);
      tc::split2(v[6], v[7], hi.w, lo.w);
      const int c = (c0 >> 3) + h;
      *reinterpret_cast<uint4 *>(base + c * 2048 + px * 16) = hi;
      *reinterpret_cast<uint4 *>(base + kDz + c * 2048 + px * 16) = lo;
    }
  };
  RowGather<bf16> g;
  g.issue(a, b, x0, y0 - 1, H, W);
  g.store(ring);
  g.issue(a, b, x0, y0, H, W);
  g.store(ring);
  g.issue(a, b, x0, y0 + 1, H, W);
  g.store(ring);
  issue_dz(y0);
  store_dz();
  if (y0 + 1 < y1) {
    g.issue(a, b, x0, y0 + 2, H, W);
    issue_dz(y0 + 1);
  }
  unsigned ph = 0;
  bool bad = false;
  for (int y = y0; y < y1; ++y) {
    tc::fence_async_smem();
    tc::fence_before();
    if (__syncthreads_or(bad)) break;  // rows y - 1 .. y + 1 and dz row y in place; the MMAs of row y - 1 done
    tc::fence_after();
    if (tid == 0) {
      // consecutive MMAs go to different accumulators (tap innermost), so
      // that no MMA waits for the one before it
      const unsigned abase = sbase + (y & 1) * 2 * kDz;
#pragma unroll 1
      for (int step = 0; step < 16; ++step) {
        const int part = step >> 3, kk = step & 7;
        const unsigned long long adesc = tc::sdesc(abase + part * kDz + kk * 256, 128, 2048);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          const unsigned bd = sbase + 4 * kDz + ((y + dy) & 3) * kSlot + (1 + dx) * 16 + kk * 256;
          tc::mma(tslot + tap * 32, adesc, tc::sdesc(bd, 128, kChunk), kIdescW, (y > y0 || step) ? 1u : 0u);
        }
      }
      tc::commit(&bar);
    }
    // the next rows go into the slot / buffer the MMAs of row y - 1 read
    // (completed), while the MMAs of row y run; the loads after them are in
    // flight until the next iteration
    if (y + 1 < y1) {
      g.store(ring);  // row y + 2
      store_dz();     // dz row y + 1
      if (y + 2 < y1) {
        g.issue(a, b, x0, y + 3, H, W);
        issue_dz(y + 2);
      }
    }
    bad |= !nsk::mbar_wait_bounded(&bar, ph);
    ph ^= 1u;
    tc::fence_after();
  }
  if (bad) {
    if (tid == 0) atomicExch(err, 3);
    nsk::mbar_wait_bounded(&bar, ph);  // an MMA group in flight may still write the accumulators
  }
  // bias: sum over the block's pixels of the per-channel sums
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float v = bacc[j];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0 && !bad) atomicAdd(db + c0 + j, v);
  }
  // weights: warp 0's lanes are the 32 output channels
  if (warp == 0 && !bad) {
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      float v[32];
      tc::tmem_ld<32>(tslot + tap * 32, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int ci = 0; ci < 32; ++ci) atomicAdd(dw + (lane * 32 + ci) * 9 + tap, v[ci]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tslot, 512);
}

// dw[co][ci][k] += sum_b sum_p dz[b][co][p] a[b][ci][p + off(k)];  db[co] += sum dz[b][co][p]
// One block per (image, 64x64 region), walking its 16 sub-tiles.
template <int CIN, int COUT, typename TA>
__global__ void __launch_bounds__(256) conv_bwd_weight(const TA *__restrict__ a, const float *__restrict__ dz,
                                                       float *__restrict__ dw, float *__restrict__ db, int H, int W) {
  extern __shared__ float csm[];
  constexpr int AS = 325;                // channel strides: odd, so lanes on consecutive channels hit distinct banks
  constexpr int DS = TILE * TILE + 1;
  float *sdz = csm;                      // [COUT][DS] holding 16 x 16
  float *sa = csm + COUT * DS;           // [CIN][AS] holding 18 x 18
  const int b = blockIdx.z;
  const long long img = (long long)H * W;
  constexpr int PAIRS = COUT * CIN;
  constexpr int PPT = (PAIRS + 255) / 256;  // pairs per thread
  float acc[PPT][9];
  float accb[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    accb[q] = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[q][k] = 0.0f;
  }
  for (int sub = 0; sub < 16; ++sub) {
    const int y0 = blockIdx.y * 64 + (sub / 4) * TILE, x0 = blockIdx.x * 64 + (sub % 4) * TILE;
    __syncthreads();
    for (int i = threadIdx.x; i < COUT * TILE * TILE; i += blockDim.x) {
      const int co = i / (TILE * TILE), r = i % (TILE * TILE);
      sdz[co * DS + r] = dz[((long long)b * COUT + co) * img + (long long)(y0 + r / TILE) * W + x0 + r % TILE];
    }
    for (int i = threadIdx.x; i < CIN * 324; i += blockDim.x) {
      const int ci = i / 324, r = i % 324, yy = r / 18, xx = r % 18;
      const int gy = (y0 + yy - 1 + H) % H, gx = (x0 + xx - 1 + W) % W;
      sa[ci * AS + r] = ldf(a + ((long long)b * CIN + ci) * img + (long long)gy * W + gx);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int pr = threadIdx.x + 256 * q;
      if (pr >= PAIRS) break;
      const int co = pr / CIN, ci = pr % CIN;
      for (int py = 0; py < TILE; ++py)
        for (int px = 0; px < TILE; ++px) {
          const float g = sdz[co * DS + py * TILE + px];
          if (ci == 0) accb[q] += g;
#pragma unroll
          for (int k = 0; k < 9; ++k) acc[q][k] = fmaf(g, sa[ci * AS + (py + k / 3) * 18 + px + k % 3], acc[q][k]);
        }
    }
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int pr = threadIdx.x + 256 * q;
    if (pr >= PAIRS) break;
    const int co = pr / CIN, ci = pr % CIN;
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(dw + (co * CIN + ci) * 9 + k, acc[q][k]);
    if (ci == 0) atomicAdd(db + co, accb[q]);
  }
}

// Weight gradient of the layers with one input or one output channel (32
// channel pairs): one thread per (pair, tap), 288 threads, each summing the
// 1024 pixels of a 32x32 region (four 16x16 sub-tiles staged in shared
// memory); one atomic add per (pair, tap) and block, the bias from the tap-0
// threads of input channel 0.
template <int CIN, int COUT, typename TA>
__global__ void __launch_bounds__(CIN * COUT * 9) conv_bwd_weight_small(const TA *__restrict__ a,
                                                                       const float *__restrict__ dz,
                                                                       float *__restrict__ dw,
                                                                       float *__restrict__ db, int H, int W) {
  static_assert(CIN * COUT == 32, "32 channel pairs");
  __shared__ float sdz[COUT][TILE * TILE];
  __shared__ float sa[CIN][18 * 18];
  const int b = blockIdx.z;
  const long long img = (long long)H * W;
  const int u = threadIdx.x, pr = u / 9, tap = u % 9, co = pr / CIN, ci = pr % CIN;
  const int ky = tap / 3, kx = tap % 3;
  float acc = 0.0f, accb = 0.0f;
  for (int sub = 0; sub < 4; ++sub) {
    const int y0 = blockIdx.y * 32 + (sub / 2) * TILE, x0 = blockIdx.x * 32 + (sub % 2) * TILE;
    __syncthreads();
    for (int i = threadIdx.x; i < COUT * TILE * TILE; i += blockDim.x) {
      const int c = i / (TILE * TILE), r = i % (TILE * TILE);
      sdz[c][r] = dz[((long long)b * COUT + c) * img + (long long)(y0 + r / TILE) * W + x0 + r % TILE];
    }
    for (int i = threadIdx.x; i < CIN * 324; i += blockDim.x) {
      const int c = i / 324, r = i % 324, yy = r / 18, xx = r % 18;
      const int gy = (y0 + yy - 1 + H) % H, gx = (x0 + xx - 1 + W) % W;
      sa[c][r] = ldf(a + ((long long)b * CIN + c) * img + (long long)gy * W + gx);
    }
    __syncthreads();
#pragma unroll 4
    for (int p = 0; p < TILE * TILE; ++p) {
      const float g = sdz[co][p];
      acc = fmaf(g, sa[ci][(p / TILE + ky) * 18 + p % TILE + kx], acc);
      accb += g;
    }
  }
  atomicAdd(dw + pr * 9 + tap, acc);
  if (ci == 0 && tap == 0) atomicAdd(db + co, accb);
}

// flipped, transposed weights for the data gradient: wt[ci][co][8-k] = w[co][ci][k]
__global__ void flip_weights(const bf16 *__restrict__ w, bf16 *__restrict__ wt, int cin, int cout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cin * cout * 9) return;
  const int co = i / (cin * 9), r = i % (cin * 9), ci = r / 9, k = r % 9;
  wt[(ci * cout + co) * 9 + (8 - k)] = w[i];
}

// dy = 2 (y - t) / count, loss += sum (y - t)^2 / count
__global__ void mse_grad(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                         float *__restrict__ loss, long long n) {
  __shared__ float part[256];
  float s = 0.0f;
  const float inv = 1.0f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d * inv;
    s += d * d * inv;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, part[0]);
}

__global__ void adam_update(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16(const float *__restrict__ src, bf16 *__restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

__global__ void f64_to_f32_scaled(const double *__restrict__ src, float *__restrict__ dst, long long n, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)(src[i] * scale);
}

__global__ void f32_scaled_add_f64(const float *__restrict__ src, const double *__restrict__ base,
                                   double *__restrict__ dst, long long n, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (base ? base[i] : 0.0) + scale * (double)src[i];
}

// splitmix64 stream -> standard normals (Box-Muller) for the weight init
uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
double unif(uint64_t seed, uint64_t i) { return ((sm64(seed ^ sm64(i)) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

thread_local std::string g_cnn_error;

}  // namespace

struct ns_cnn {
  int C = 32, H = 0, W = 0, maxb = 0;
  int cin[4], cout[4];
  long long woff[4], boff[4];
  int nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grad, Adam moments
  bf16 *wb[4] = {nullptr, nullptr, nullptr, nullptr};             // BF16 weights
  bf16 *wt[4] = {nullptr, nullptr, nullptr, nullptr};             // flipped weights
  bf16 *z[3] = {nullptr, nullptr, nullptr}, *a[3] = {nullptr, nullptr, nullptr};
  float *y = nullptr, *dy = nullptr, *dza = nullptr, *dzb = nullptr, *loss = nullptr;
  int *errw = nullptr;  // device error word of the tensor-core convolutions (bounded waits)
  int nsm = 1;
  int step = 0;
  std::string err;
};

namespace {

int cfail(ns_cnn *c, int code, const std::string &m) {
  if (c)
    c->err = m;
  else
    g_cnn_error = m;
  return code;
}

#define CNN_CK(c, call)                                                                              \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return cfail((c), NS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t fwd_smem(int cin, int cout) { return sizeof(float) * (cout * cin * 9 + cin * 324); }
size_t bww_smem(int cin, int cout) { return sizeof(float) * (cout * (TILE * TILE + 1) + cin * 325); }

// Launches carry no attribute calls, so they can be captured into a CUDA
// graph; set_attributes() raises the dynamic shared-memory limits once.
template <int CIN, int COUT, int EPI, typename TIN, typename TOUT>
int launch_fwd(const TIN *x, const bf16 *w, const float *bias, const bf16 *zin, bf16 *zout, TOUT *out, int B, int H,
               int W, cudaStream_t s) {
  conv_fwd<CIN, COUT, EPI, TIN, TOUT><<<dim3(W / TILE, H / TILE, B), TILE * TILE, fwd_smem(CIN, COUT), s>>>(
      x, w, bias, zin, zout, out, H, W);
  return (int)cudaGetLastError();
}

// the 32 -> 32 convolution on the tensor cores when the width is a multiple
// of 128 (row segments of 128 pixels), else conv_fwd on the CUDA cores; rows
// per block chosen so that about two blocks per SM are launched
template <int EPI, typename TIN, typename TOUT>
int launch_c32(const ns_cnn *c, const TIN *x, const bf16 *w, const float *bias, const bf16 *zin, bf16 *zout, TOUT *out,
               int B, int H, int W, cudaStream_t s) {
  if (W % 128 != 0) return launch_fwd<32, 32, EPI, TIN, TOUT>(x, w, bias, zin, zout, out, B, H, W, s);
  const int strips = W / 128;
  const int segs = std::max(1, std::min(H, (2 * c->nsm + B * strips - 1) / (B * strips)));
  const int rows = (H + segs - 1) / segs;
  const int blocks = B * strips * ((H + rows - 1) / rows);
  conv32_tc<EPI, TIN, TOUT><<<blocks, kConvThreads, ctc::smem_bytes(sizeof(TIN) == 4), s>>>(x, w, bias, zin, zout, out, H, W,
                                                                                   rows, c->errw);
  return (int)cudaGetLastError();
}

// weight gradient of a 32 -> 32 layer: the tensor cores when the width is a
// multiple of 128, about one block per SM (each holds all of the SM's tensor
// memory), else conv_bwd_weight
int launch_w32(const ns_cnn *c, const bf16 *a, const float *dz, float *dw, float *db, int B, int H, int W,
               cudaStream_t s);

template <int CIN, int COUT, typename TA>
int launch_bww(const TA *a, const float *dz, float *dw, float *db, int B, int H, int W, cudaStream_t s) {
  conv_bwd_weight<CIN, COUT, TA><<<dim3(W / 64, H / 64, B), 256, bww_smem(CIN, COUT), s>>>(a, dz, dw, db, H, W);
  return (int)cudaGetLastError();
}

template <int CIN, int COUT, int EPI, typename TIN, typename TOUT>
void fwd_attr() {
  cudaFuncSetAttribute(conv_fwd<CIN, COUT, EPI, TIN, TOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fwd_smem(CIN, COUT));
}
template <int CIN, int COUT, typename TA>
void bww_attr() {
  cudaFuncSetAttribute(conv_bwd_weight<CIN, COUT, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bww_smem(CIN, COUT));
}

int launch_w32(const ns_cnn *c, const bf16 *a, const float *dz, float *dw, float *db, int B, int H, int W,
               cudaStream_t s) {
  if (W % 128 != 0) return launch_bww<32, 32, bf16>(a, dz, dw, db, B, H, W, s);
  const int strips = W / 128;
  const int segs = std::max(1, std::min(H, c->nsm / (B * strips)));  // at most one wave
  const int rows = (H + segs - 1) / segs;
  const int blocks = B * strips * ((H + rows - 1) / rows);
  conv32_wgrad_tc<<<blocks, kConvThreads, ctc::kWgSmem, s>>>(a, dz, dw, db, H, W, rows, c->errw);
  return (int)cudaGetLastError();
}

// every kernel instance that forward() and backward() launch
void set_attributes() {
  fwd_attr<1, 32, EPI_GELU, float, bf16>();
  fwd_attr<32, 32, EPI_GELU, bf16, bf16>();
  fwd_attr<32, 1, EPI_LINEAR, bf16, float>();
  fwd_attr<1, 32, EPI_GELU_BWD, float, float>();
  fwd_attr<32, 32, EPI_GELU_BWD, float, float>();
  bww_attr<32, 32, bf16>();
  cudaFuncSetAttribute(conv32_tc<EPI_GELU, bf16, bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ctc::smem_bytes(false));
  cudaFuncSetAttribute(conv32_tc<EPI_GELU_BWD, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ctc::smem_bytes(true));
  cudaFuncSetAttribute(conv32_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctc::kWgSmem);
}

// forward pass through all layers; keeps z_l, a_l for the backward pass
int forward(ns_cnn *c, const float *x, int B, cudaStream_t s) {
  const int H = c->H, W = c->W;
  int rc;
  const float *p = c->p;
  if ((rc = launch_fwd<1, 32, EPI_GELU, float, bf16>(x, c->wb[0], p + c->boff[0], nullptr, c->z[0], c->a[0], B, H, W,
                                                      s)))
    return rc;
  if ((rc = launch_c32<EPI_GELU, bf16, bf16>(c, c->a[0], c->wb[1], p + c->boff[1], nullptr, c->z[1], c->a[1], B, H,
                                              W, s)))
    return rc;
  if ((rc = launch_c32<EPI_GELU, bf16, bf16>(c, c->a[1], c->wb[2], p + c->boff[2], nullptr, c->z[2], c->a[2], B, H,
                                              W, s)))
    return rc;
  return launch_fwd<32, 1, EPI_LINEAR, bf16, float>(c->a[2], c->wb[3], p + c->boff[3], nullptr, nullptr, c->y, B, H,
                                                    W, s);
}

// gradients of the mean squared error into c->g (zeroed here)
int backward(ns_cnn *c, const float *x, const float *t, int B, cudaStream_t s) {
  const int H = c->H, W = c->W;
  const long long n = (long long)B * H * W;
  int rc;
  CNN_CK(c, cudaMemsetAsync(c->g, 0, sizeof(float) * c->nparams, s));
  CNN_CK(c, cudaMemsetAsync(c->loss, 0, sizeof(float), s));
  mse_grad<<<(unsigned)std::min<long long>((n + 255) / 256, 2048), 256, 0, s>>>(c->y, t, c->dy, c->loss, n);
  for (int l = 0; l < 4; ++l)
    flip_weights<<<(c->cin[l] * c->cout[l] * 9 + 255) / 256, 256, 0, s>>>(c->wb[l], c->wt[l], c->cin[l], c->cout[l]);
  float *g = c->g;
  // layer 3: dz3 = dy
  conv_bwd_weight_small<32, 1, bf16><<<dim3(W / 32, H / 32, B), 288, 0, s>>>(c->a[2], c->dy, g + c->woff[3],
                                                                             g + c->boff[3], H, W);
  if ((rc = (int)cudaGetLastError())) return rc;
  if ((rc = launch_fwd<1, 32, EPI_GELU_BWD, float, float>(c->dy, c->wt[3], nullptr, c->z[2], nullptr, c->dza, B, H, W,
                                                          s)))
    return rc;  // dz2
  if ((rc = launch_w32(c, c->a[1], c->dza, g + c->woff[2], g + c->boff[2], B, H, W, s))) return rc;
  if ((rc = launch_c32<EPI_GELU_BWD, float, float>(c, c->dza, c->wt[2], nullptr, c->z[1], nullptr, c->dzb, B, H, W,
                                                    s)))
    return rc;  // dz1
  if ((rc = launch_w32(c, c->a[0], c->dzb, g + c->woff[1], g + c->boff[1], B, H, W, s))) return rc;
  if ((rc = launch_c32<EPI_GELU_BWD, float, float>(c, c->dzb, c->wt[1], nullptr, c->z[0], nullptr, c->dza, B, H, W,
                                                    s)))
    return rc;  // dz0
  conv_bwd_weight_small<1, 32, float><<<dim3(W / 32, H / 32, B), 288, 0, s>>>(x, c->dza, g + c->woff[0],
                                                                              g + c->boff[0], H, W);
  return (int)cudaGetLastError();
}

// the device error word (a tensor-core convolution whose bounded wait expired
// wrote a nonzero code): NS_ETIMEOUT once, then cleared
int check_err(ns_cnn *c) {
  int e = 0;
  CNN_CK(c, cudaMemcpy(&e, c->errw, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == 0) return NS_OK;
  cudaMemset(c->errw, 0, sizeof(int));
  return cfail(c, NS_ETIMEOUT, "tensor-core convolution: a bounded wait expired");
}

int refresh_bf16(ns_cnn *c, cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    const int n = c->cin[l] * c->cout[l] * 9;
    to_bf16<<<(n + 255) / 256, 256, 0, s>>>(c->p + c->woff[l], c->wb[l], n);
  }
  return (int)cudaGetLastError();
}

}  // namespace

extern "C" {

int ns_cnn_init(ns_cnn **out, int height, int width, int max_batch, unsigned long long seed) {
  if (!out) return cfail(nullptr, NS_EINVAL, "ns_cnn_init: out is null");
  *out = nullptr;
  if (height < TILE * 4 || width < TILE * 4 || height % 64 || width % 64 || max_batch < 1)
    return cfail(nullptr, NS_EINVAL, "ns_cnn_init: height and width must be multiples of 64, batch >= 1");
  ns_cnn *c = new ns_cnn();
  c->H = height;
  c->W = width;
  c->maxb = max_batch;
  const int ci[4] = {1, 32, 32, 32}, co[4] = {32, 32, 32, 1};
  long long off = 0;
  for (int l = 0; l < 4; ++l) {
    c->cin[l] = ci[l];
    c->cout[l] = co[l];
    c->woff[l] = off;
    off += (long long)ci[l] * co[l] * 9;
    c->boff[l] = off;
    off += co[l];
  }
  c->nparams = (int)off;
  std::vector<float> init(c->nparams, 0.0f);
  for (int l = 0; l < 4; ++l) {  // He-normal weights, zero biases
    const double sd = std::sqrt(2.0 / (9.0 * ci[l]));
    for (long long i = 0; i < (long long)ci[l] * co[l] * 9; ++i) {
      const double u1 = unif(seed, 2 * (c->woff[l] + i)), u2 = unif(seed, 2 * (c->woff[l] + i) + 1);
      init[c->woff[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  auto bail = [&](const char *what) {
    g_cnn_error = std::string("ns_cnn_init: ") + what;
    ns_cnn_destroy(c);
    return NS_ENOMEM;
  };
  const size_t img = (size_t)height * width * max_batch;
  if (cudaMalloc(&c->p, sizeof(float) * c->nparams) || cudaMalloc(&c->g, sizeof(float) * c->nparams) ||
      cudaMalloc(&c->m, sizeof(float) * c->nparams) || cudaMalloc(&c->v, sizeof(float) * c->nparams) ||
      cudaMalloc(&c->y, sizeof(float) * img) || cudaMalloc(&c->dy, sizeof(float) * img) ||
      cudaMalloc(&c->dza, sizeof(float) * img * 32) || cudaMalloc(&c->dzb, sizeof(float) * img * 32) ||
      cudaMalloc(&c->loss, sizeof(float)) || cudaMalloc(&c->errw, sizeof(int)) ||
      cudaMemset(c->errw, 0, sizeof(int)))
    return bail("allocation failed");
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (c->nsm < 1) c->nsm = 1;
  }
  for (int l = 0; l < 4; ++l)
    if (cudaMalloc(&c->wb[l], sizeof(bf16) * ci[l] * co[l] * 9) || cudaMalloc(&c->wt[l], sizeof(bf16) * ci[l] * co[l] * 9))
      return bail("allocation failed");
  for (int l = 0; l < 3; ++l)
    if (cudaMalloc(&c->z[l], sizeof(bf16) * img * 32) || cudaMalloc(&c->a[l], sizeof(bf16) * img * 32))
      return bail("allocation failed");
  set_attributes();
  if (cudaMemcpy(c->p, init.data(), sizeof(float) * c->nparams, cudaMemcpyHostToDevice) ||
      cudaMemset(c->m, 0, sizeof(float) * c->nparams) || cudaMemset(c->v, 0, sizeof(float) * c->nparams) ||
      refresh_bf16(c, 0) || cudaDeviceSynchronize())
    return bail("initialisation failed");
  *out = c;
  return NS_OK;
}

int ns_cnn_num_params(const ns_cnn *c) { return c ? c->nparams : -1; }

int ns_cnn_get_params(ns_cnn *c, float *host) {
  if (!c || !host) return NS_EINVAL;
  CNN_CK(c, cudaMemcpy(host, c->p, sizeof(float) * c->nparams, cudaMemcpyDeviceToHost));
  return NS_OK;
}

int ns_cnn_set_params(ns_cnn *c, const float *host) {
  if (!c || !host) return NS_EINVAL;
  CNN_CK(c, cudaMemcpy(c->p, host, sizeof(float) * c->nparams, cudaMemcpyHostToDevice));
  int rc = refresh_bf16(c, 0);
  if (rc) return cfail(c, NS_ECUDA, cudaGetErrorString((cudaError_t)rc));
  CNN_CK(c, cudaDeviceSynchronize());
  return NS_OK;
}

int ns_cnn_forward(ns_cnn *c, const float *x_dev, float *y_dev, int batch, void *stream) {
  if (!c || !x_dev || !y_dev || batch < 1 || batch > c->maxb) return c ? cfail(c, NS_EINVAL, "ns_cnn_forward: args") : NS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(c, x_dev, batch, s);
  if (rc) return cfail(c, NS_ECUDA, cudaGetErrorString((cudaError_t)rc));
  CNN_CK(c, cudaMemcpyAsync(y_dev, c->y, sizeof(float) * (size_t)batch * c->H * c->W, cudaMemcpyDeviceToDevice, s));
  return NS_OK;
}

int ns_cnn_gradients(ns_cnn *c, const float *x_dev, const float *t_dev, int batch, float *grad_host, float *loss) {
  if (!c || !x_dev || !t_dev || !grad_host || !loss || batch < 1 || batch > c->maxb)
    return c ? cfail(c, NS_EINVAL, "ns_cnn_gradients: args") : NS_EINVAL;
  int rc = forward(c, x_dev, batch, 0);
  if (!rc) rc = backward(c, x_dev, t_dev, batch, 0);
  if (rc) return cfail(c, NS_ECUDA, "ns_cnn_gradients: launch failed");
  CNN_CK(c, cudaMemcpy(grad_host, c->g, sizeof(float) * c->nparams, cudaMemcpyDeviceToHost));
  CNN_CK(c, cudaMemcpy(loss, c->loss, sizeof(float), cudaMemcpyDeviceToHost));
  return check_err(c);
}

int ns_cnn_train_step(ns_cnn *c, const float *x_dev, const float *t_dev, int batch, float lr, float *loss_out,
                      void *stream) {
  if (!c || !x_dev || !t_dev || batch < 1 || batch > c->maxb || !(lr > 0))
    return c ? cfail(c, NS_EINVAL, "ns_cnn_train_step: args") : NS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(c, x_dev, batch, s);
  if (!rc) rc = backward(c, x_dev, t_dev, batch, s);
  if (rc) return cfail(c, NS_ECUDA, "ns_cnn_train_step: launch failed");
  c->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)c->step), c2 = 1.0f - std::pow(b2, (float)c->step);
  adam_update<<<(c->nparams + 255) / 256, 256, 0, s>>>(c->p, c->g, c->m, c->v, c->nparams, lr, b1, b2, 1e-8f, c1, c2);
  rc = refresh_bf16(c, s);
  if (rc) return cfail(c, NS_ECUDA, "ns_cnn_train_step: update failed");
  if (loss_out) {
    CNN_CK(c, cudaMemcpyAsync(loss_out, c->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CNN_CK(c, cudaStreamSynchronize(s));
    return check_err(c);
  }
  return NS_OK;
}

int ns_f64_to_f32(const double *src_dev, float *dst_dev, long long n, double scale, void *stream) {
  if (!src_dev || !dst_dev || n < 0) return NS_EINVAL;
  f64_to_f32_scaled<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(
      src_dev, dst_dev, n, scale);
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ECUDA;
}

int ns_f32_axpy_f64(const float *src_dev, const double *base_dev, double *dst_dev, long long n, double scale,
                    void *stream) {
  if (!src_dev || !dst_dev || n < 0) return NS_EINVAL;
  f32_scaled_add_f64<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(
      src_dev, base_dev, dst_dev, n, scale);
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ECUDA;
}

void ns_cnn_destroy(ns_cnn *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  void *ptrs[] = {c->p, c->g, c->m, c->v, c->y, c->dy, c->dza, c->dzb, c->loss, c->errw};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < 4; ++l) {
    if (c->wb[l]) cudaFree(c->wb[l]);
    if (c->wt[l]) cudaFree(c->wt[l]);
  }
  for (int l = 0; l < 3; ++l) {
    if (c->z[l]) cudaFree(c->z[l]);
    if (c->a[l]) cudaFree(c->a[l]);
  }
  delete c;
}

const char *ns_cnn_last_error(const ns_cnn *c) { return c ? c->err.c_str() : g_cnn_error.c_str(); }

}  // extern "C"
