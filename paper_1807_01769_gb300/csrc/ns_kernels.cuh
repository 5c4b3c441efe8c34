// ns_kernels.cuh -- the pass kernels of the right-hand side and time step.
//
// One RK stage of the 3D solver is four launches (all names refer to the
// axis transformed):
//   inv2   (y)  : 6 fields, ky -> y, zero-padded from the c retained rows
//   xpass  (x)  : per (z, y) line: 6 c2r, n = u x omega, 3 r2c, keep kx <= kc
//   fwd2   (y)  : 3 fields, y -> ky, keep the c retained rows
//   fwd1   (z)  : 3 fields, z -> kz, keep retained rows, divide by N^3,
//                 project, add forcing, RK stage update, then (fused) the
//                 curl and z -> kz inverse of the next stage input (6 fields)
// and the first inverse axis of a call (inv1: curl + z inverse from the state)
// runs once per ns_step call.  The 2D solver is two launches per stage: xpass
// (4 c2r, n = -(u . grad w), 1 r2c) and fwd1 (y forward, dealias, RK, then
// velocity / vorticity-gradient forms and y inverse of the next stage).
//
// Physical fields never touch global memory: they exist only in registers
// inside xpass, packed two real points per complex number (z[m] = x[2m] +
// i x[2m+1]) so the c2r and r2c of length N are complex FFTs of length N/2 with
// a pre/post-processing step, and the pointwise product acts on the packed
// pairs directly.  The operators follow the FluidSim paper's list ("The
// simulation object": FFT, IFFT, dealiasing, divergence, curl; "Tri-dimensional
// simulations": FFT, RK4, curl, vector product, projection).
#pragma once
#include <cuda.h>  // CUtensorMap (a kernel parameter type; no driver calls here)

#include "ns_fft.cuh"
#include "ns_internal.h"

namespace nsk {

template <typename R>
__host__ __device__ constexpr int wmax() {
  return sizeof(R) == 4 ? 16 : 8;  // 128 bytes of complex per tile row
}
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
// columns per tile: light kernels (one field live per thread) and the fused
// fwd1 (three fields live per thread)
template <typename R, int N>
__host__ __device__ constexpr int w_light() {
  return cmin(wmax<R>(), cmax(1, 1024 / (N / 8)));
}
template <typename R, int N>
__host__ __device__ constexpr int w_heavy() {
  return cmin(wmax<R>(), cmax(1, (sizeof(R) == 4 ? 512 : 256) / (N / 8)));
}
// columns per tile of the y passes (rules in ns_internal.h)
template <typename R, int N>
__host__ __device__ constexpr int w_yinv() {
  return y_inv_columns((int)sizeof(R) * 2, N);
}
template <typename R, int N>
__host__ __device__ constexpr int w_yfwd() {
  return y_fwd_columns((int)sizeof(R) * 2, N);
}
// lines per block of the x kernels (N/16 threads per line); lines longer
// than a warp in FP32: one line per block, whose barriers then span only that
// line's warps (measured at 1024^3: x pass 18.6 ms with 4 lines per block,
// 16.7 ms with 2, 16.4 ms with 1)
template <typename R, int N>
__host__ __device__ constexpr int x_lines() {
  return cmin(N, cmax(1, (sizeof(R) == 4 ? (N / 16 > 32 ? 64 : 256) : 128) / (N / 16)));
}
__host__ __device__ constexpr int pitch_of(int W, int csize) { return (W * csize < 128) ? W + 1 : W; }

// Shared memory of a column kernel: the exchange tile [N][pitch], doubled when
// two copies plus `extra` bytes fit in one block's shared memory.
constexpr size_t kSmemMax = 232448;
__host__ __device__ constexpr size_t col_tile_bytes(int N, int W, int csize) {
  return (size_t)N * pitch_of(W, csize) * csize;
}
__host__ __device__ constexpr bool col_db(int N, int W, int csize, size_t extra) {
  return 2 * col_tile_bytes(N, W, csize) + extra <= kSmemMax;
}
__host__ __device__ constexpr size_t col_smem(int N, int W, int csize, size_t extra) {
  return (col_db(N, W, csize, extra) ? 2 : 1) * col_tile_bytes(N, W, csize) + extra;
}

// dynamic shared memory, 128-byte aligned (TMA destinations need it)
template <typename C>
__device__ __forceinline__ C *dyn_smem() {
  extern __shared__ __align__(128) unsigned char ns_dyn_smem[];
  return reinterpret_cast<C *>(ns_dyn_smem);
}
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Loads of data read exactly once (pass inputs): kept out of L1 so that the
// reused twiddle and factor tables stay there.
template <typename C>
__device__ __forceinline__ C ld_stream(const C *p) {
  return __ldcg(p);
}

// Asynchronous global -> shared copies of BYTES (4, 8 or 16); a false
// predicate zero-fills the destination without reading the source.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst_smem)), "l"(src), "n"(BYTES),
               "r"(pred ? BYTES : 0)
               : "memory");
}
// 16 bytes, cached in L2 only (streamed operands that would evict L1 data).
__device__ __forceinline__ void cp_async_cg16(void *dst_smem, const void *src, bool pred) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst_smem)), "l"(src),
               "r"(pred ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ bool retained(int n, int N, int kc) { return n <= kc || n >= N - kc; }
__device__ __forceinline__ int compact_of(int n, int N, int kc, int c) { return n <= kc ? n : n - (N - c); }
__device__ __forceinline__ int kfull_of(int n, int N, int kc) { return n <= kc ? n : n - N; }
__device__ __forceinline__ int ktr_of(int i, int kc, int c) { return i <= kc ? i : i - c; }

// componentwise product of packed real pairs
template <typename C>
__device__ __forceinline__ C pmul(C a, C b) {
  return C{a.x * b.x, a.y * b.y};
}
template <typename C>
__device__ __forceinline__ C pfma(C a, C b, C acc) {
  return C{fma(a.x, b.x, acc.x), fma(a.y, b.y, acc.y)};
}
template <typename C>
__device__ __forceinline__ C pfms(C a, C b, C acc) {  // acc - a*b
  return C{fma(-a.x, b.x, acc.x), fma(-a.y, b.y, acc.y)};
}

// ----------------------------------------------- x-line helper routines ---
// Stage the half spectrum X[0..h-1] of L lines (row stride hs) into shared
// lines of length H (zero above h).
template <typename C, int H, int L>
__device__ __forceinline__ void stage_lines(C *S, const C *__restrict__ src, long long line0, int h, int hs) {
  constexpr int SL = smline_len(H);
  for (int idx = threadIdx.x; idx < L * H; idx += blockDim.x) {
    const int ll = idx / H, k = idx % H;
    S[ll * SL + k + (k >> 3)] = k < h ? ld_stream(src + (line0 + ll) * hs + k) : czero<C>();
  }
}

// c2r pre-processing: Z[k] = (X[k] + conj X[H-k]) + i e^{+2 pi i k/N} (X[k] - conj X[H-k]),
// X[H] = 0 (never retained), imaginary part of X[0] dropped (real part of the
// self-conjugate term, as the inverse c2r of a Hermitian spectrum).
template <typename C, int N>
__device__ __forceinline__ C c2r_pre(const C *Sl, int k, const C *__restrict__ tw) {
  constexpr int H = N / 2;
  C xk = Sl[k + (k >> 3)];
  C xm;
  if (k == 0) {
    xk.y = 0;
    xm = czero<C>();
  } else {
    const int j = H - k;
    xm = Sl[j + (j >> 3)];
  }
  const C a = cadd(xk, cconj(xm));
  const C b = csub(xk, cconj(xm));
  const C e = cconj(__ldg(tw + k));
  return cadd(a, cmuli(cmul(e, b)));
}

// r2c post-processing: X[k] = (Z[k] + conj Z[H-k])/2 - i/2 e^{-2 pi i k/N} (Z[k] - conj Z[H-k]).
template <typename C, int N>
__device__ __forceinline__ C r2c_post(const C *Sl, int k, const C *__restrict__ tw) {
  constexpr int H = N / 2;
  using R = decltype(C{}.x);
  const int j = (H - k) & (H - 1);
  const C zk = Sl[k + (k >> 3)], zm = Sl[j + (j >> 3)];
  const C a = cadd(zk, cconj(zm));
  const C b = csub(zk, cconj(zm));
  const C e = __ldg(tw + k);
  const C r = csub(a, cmuli(cmul(e, b)));
  return C{(R)0.5 * r.x, (R)0.5 * r.y};
}

// Write the forward-transformed line (v[m] = Z[t + TX m]) to shared memory and
// emit X[0..h-1] of all L lines to dst (row stride hs), coalesced.
template <typename C, int N, int L>
__device__ __forceinline__ void emit_r2c(C (&v)[8], int t, int l, C *S, C *__restrict__ dst, long long line0, int h,
                                         int hs, const C *__restrict__ tw) {
  constexpr int H = N / 2, TX = H / 8, SL = smline_len(H);
  __syncthreads();  // last FFT stage finished reading S
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k = t + TX * m;
    S[l * SL + k + (k >> 3)] = v[m];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < L * h; idx += blockDim.x) {
    const int ll = idx / h, k = idx % h;
    dst[(line0 + ll) * hs + k] = r2c_post<C, N>(S + ll * SL, k, tw);
  }
}

// ------------------------------------- warp-per-line x helpers (TX <= 32) ---
// Lane t of a line (TX lanes) holds slot m = index k = t + TX m of a length-H
// line.  Returns the value at index (H - k) mod H: lane (TX - t) mod TX holds
// it in slot 7 - m (t > 0) or slot (8 - m) mod 8 (t = 0).  All lanes of the
// warp must call it with the same m.
template <int TX, typename C>
__device__ __forceinline__ C shfl_partner(const C (&x)[8], int m, int t) {
  const C send = (t == 0) ? x[(8 - m) & 7] : x[7 - m];
  if (TX == 1) return send;
  const int src = (TX - t) & (TX - 1);
  return C{__shfl_sync(0xffffffffu, send.x, src, TX), __shfl_sync(0xffffffffu, send.y, src, TX)};
}

// exp(-2 pi i m / 16), m = 0..7: with TX = N/16 lanes per line,
// exp(-2 pi i (t + TX m) / N) = exp(-2 pi i t / N) * exp(-2 pi i m / 16).
template <typename C>
__device__ __forceinline__ C w16(int m) {
  using R = decltype(C{}.x);
  const R c1 = (R)0.92387953251128675612818318939678828682;  // cos(pi/8)
  const R s1 = (R)0.38268343236508977172845998403039886676;  // sin(pi/8)
  const R h = (R)0.70710678118654752440084436210484903928;   // cos(pi/4)
  switch (m) {
    case 0: return C{(R)1, (R)0};
    case 1: return C{c1, -s1};
    case 2: return C{h, -h};
    case 3: return C{s1, -c1};
    case 4: return C{(R)0, (R)-1};
    case 5: return C{-s1, -c1};
    case 6: return C{-h, -h};
    default: return C{-c1, -s1};
  }
}

// c2r pre-processing from registers (see c2r_pre); x[m] = X[t + TX m];
// wt = exp(-2 pi i t / N).
template <typename C, int N, int TX>
__device__ __forceinline__ C c2r_pre_reg(const C (&x)[8], int m, int t, C wt) {
  const int k = t + TX * m;
  C xk = x[m];
  C xm = shfl_partner<TX>(x, m, t);
  if (k == 0) {
    xk.y = 0;
    xm = czero<C>();
  }
  const C a = cadd(xk, cconj(xm));
  const C b = csub(xk, cconj(xm));
  const C e = cconj(cmul(wt, w16<C>(m)));
  return cadd(a, cmuli(cmul(e, b)));
}

// r2c post-processing from registers (see r2c_post); z[m] = Z[t + TX m];
// wt = exp(-2 pi i t / N).
template <typename C, int N, int TX>
__device__ __forceinline__ C r2c_post_reg(const C (&z)[8], int m, int t, C wt) {
  using R = decltype(C{}.x);
  const C zk = z[m];
  const C zm = shfl_partner<TX>(z, m, t);
  const C a = cadd(zk, cconj(zm));
  const C b = csub(zk, cconj(zm));
  const C e = cmul(wt, w16<C>(m));
  const C r = csub(a, cmuli(cmul(e, b)));
  return C{(R)0.5 * r.x, (R)0.5 * r.y};
}

template <typename C, int TX>
__device__ __forceinline__ void load_line(C (&x)[8], const C *__restrict__ src, int t, int h) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k = t + TX * m;
    x[m] = k < h ? ld_stream(src + k) : czero<C>();
  }
}

template <int N, bool MULTI>
__host__ __device__ constexpr int xw_line_len() {
  return smline_len(N / 2) + (MULTI ? 2 : 0);
}

// ================================================================== 3D ====
// inv1: z inverse from a state-shaped array.  CURL: six fields (u, i k x u);
// otherwise three fields (u).  One block = a tile of W kx columns at one ky.
template <typename R, int N, int W, bool CURL>
__global__ void __launch_bounds__((N / 8) * W) k3_inv1(Geo g, const typename CplxOf<R>::T *__restrict__ src,
                                                        typename CplxOf<R>::T *__restrict__ zb,
                                                        const typename CplxOf<R>::T *__restrict__ tw, int wz) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr size_t EXTRA_SMEM = 0;
  C *sm = dyn_smem<C>();
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int nkt = g.hs / W;
  const int iy = blockIdx.x / nkt;
  const int kx = (blockIdx.x % nkt) * W + w;
  const bool valid = kx < g.h;
  const R kxr = (R)kx, kyr = (R)ktr_of(iy, g.kc, g.c);
  const long long plane = (long long)g.c * g.hs;
  const long long col = (long long)iy * g.hs + kx;
  constexpr bool DB = col_db(N, W, sizeof(C), EXTRA_SMEM);
  const SmCol<C, DB> view{sm + w, P, N * P};
  const long long st = g.st_comp;
  // five transforms for six fields: omega_z = i (kx u_y - ky u_x) has no kz,
  // so its z inverse is formed from the inverses of u_x and u_y
  constexpr int NF = CURL ? 5 : 3;
  C zx[8];
  for (int f = 0; f < NF; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int n = t + T * m;
      C x = czero<C>();
      if (valid && retained(n, N, g.kc)) {
        const long long idx = (long long)compact_of(n, N, g.kc, g.c) * plane + col;
        if (f < 3) {
          x = src[f * st + idx];
        } else {
          const R kzr = (R)kfull_of(n, N, g.kc);
          C a, b;
          R ka, kb;
          if (f == 3) {  // i (ky uz - kz uy)
            a = src[2 * st + idx];
            b = src[st + idx];
            ka = kyr;
            kb = kzr;
          } else {  // i (kz ux - kx uz)
            a = src[idx];
            b = src[2 * st + idx];
            ka = kzr;
            kb = kxr;
          }
          x = cmuli(C{ka * a.x - kb * b.x, ka * a.y - kb * b.y});
        }
      }
      v[m] = x;
    }
    fft_line<N, +1>(v, t, tw + N, view);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 8; ++m) zb[f * g.zb_f + (long long)(t + T * m) * plane + col] = v[m];
    }
    if (CURL && f == 0) {
#pragma unroll
      for (int m = 0; m < 8; ++m) zx[m] = v[m];
    } else if (CURL && f == 1 && valid && !wz) {
#pragma unroll
      for (int m = 0; m < 8; ++m)
        zb[5 * g.zb_f + (long long)(t + T * m) * plane + col] =
            cmuli(C{kxr * v[m].x - kyr * zx[m].x, kxr * v[m].y - kyr * zx[m].y});
    }
  }
}

// inv2: y inverse of fields 0..nf-1 at plane z = blockIdx.y; the next field's
// loads are issued before the current field is transformed.
template <typename R, int N, int W>
__global__ void __launch_bounds__((N / 8) * W) k3_inv2(Geo g, int nf, int z0, const typename CplxOf<R>::T *__restrict__ zb,
                                                        typename CplxOf<R>::T *__restrict__ yb,
                                                        const typename CplxOf<R>::T *__restrict__ tw) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  C *sm = dyn_smem<C>();
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = blockIdx.x * W + w;
  const bool valid = kx < g.h;
  const int z = z0 + blockIdx.y;
  const C *in = zb + (long long)z * g.c * g.hs + kx;
  C *out = yb + (long long)z * N * g.hs + kx;
  int row[8];
  bool live[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int n = t + T * m;
    live[m] = valid && retained(n, N, g.kc);
    row[m] = compact_of(n, N, g.kc, g.c);
  }
  C xn[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) xn[m] = live[m] ? ld_stream(in + (long long)row[m] * g.hs) : czero<C>();
#pragma unroll 1
  for (int f = 0; f < nf; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = xn[m];
    if (f + 1 < nf) {
      const C *nin = in + (f + 1) * g.zb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) xn[m] = live[m] ? ld_stream(nin + (long long)row[m] * g.hs) : czero<C>();
    }
    fft_line<N, +1>(v, t, tw + N, SmCol<C, col_db(N, W, sizeof(C), 0)>{sm + w, P, N * P});
    if (valid) {
      C *o = out + f * g.yb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) o[(long long)(t + T * m) * g.hs] = v[m];
    }
  }
}

// Largest |value| of the packed real pairs v[0..7] over the warp, merged into
// *slot by an atomic maximum on the bit pattern (non-negative doubles order
// like their bits read as unsigned integers).  The lanes of a block narrower
// than a warp are lanes 0 .. blockDim.x - 1 (a power of two).
template <typename C>
__device__ __forceinline__ void umax_merge(const C (&v)[8], unsigned long long *slot) {
  double m = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) m = fmax(m, fmax(fabs((double)v[i].x), fabs((double)v[i].y)));
  const int width = blockDim.x < 32 ? (int)blockDim.x : 32;
  const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
  for (int off = 16; off > 0; off >>= 1)
    if (off < width) m = fmax(m, __shfl_xor_sync(mask, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, (unsigned long long)__double_as_longlong(m));
}

// xpass (3D): lines (z, y); fields u_x, u_y, u_z, w_x, w_y, w_z in, n = u x w out
// (written over fields 0..2 of the same lines).
// Lines longer than a warp (N/16 > 32 lanes): the Hermitian partners come
// through shared memory, so the exchanges synchronise the block.  As in the
// warp-per-line kernel the three velocity fields are parked in thread-private
// shared slots [field][m][thread], which keeps the kernel at 128 registers
// (FP32) and two 256-thread blocks per SM.
template <typename R>
__host__ __device__ constexpr int xpass_blocks_min(int threads) {
  return sizeof(R) == 4 ? cmax(1, 512 / threads) : 1;
}
template <typename R, int N, int L>
__global__ void __launch_bounds__((N / 16) * L, xpass_blocks_min<R>((N / 16) * L))
    k3_xpass(Geo g, long long line_base, typename CplxOf<R>::T *__restrict__ yb,
             const typename CplxOf<R>::T *__restrict__ tw, unsigned long long *__restrict__ umax) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, SL = smline_len(H), NTH = TX * L;
  C *S = dyn_smem<C>();
  C *park = S + L * SL + threadIdx.x;  // park[(f * 8 + m) * NTH]
  const int t = threadIdx.x % TX, l = threadIdx.x / TX;
  const long long line0 = line_base + (long long)blockIdx.x * L;
  const SmLine<C> view{S + l * SL};
  C nx[8], ny[8], nz[8];
  // the block's L lines of a field are L * H = 8 NTH entries: thread entry j
  // is idx = threadIdx.x + NTH j (line idx / H, index idx % H); the next
  // field's entries are loaded into xn while the current field is transformed
  static_assert(L * H == 8 * NTH, "staging map");
  C xn[8];
  auto load_field = [&](const C *src) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int idx = threadIdx.x + NTH * j, ll = idx / H, k = idx % H;
      xn[j] = k < g.h ? ld_stream(src + (line0 + ll) * g.hs + k) : czero<C>();
    }
  };
  load_field(yb);
#pragma unroll 1
  for (int f = 0; f < 6; ++f) {
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int idx = threadIdx.x + NTH * j, ll = idx / H, k = idx % H;
      S[ll * SL + k + (k >> 3)] = xn[j];
    }
    if (f < 5) load_field(yb + (f + 1) * g.yb_f);
    __syncthreads();
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = c2r_pre<C, N>(S + l * SL, t + TX * m, tw);
    fft_line<H, +1>(v, t, tw + N + stage_tw_len(N), view);
    if (umax != nullptr && f < 3) umax_merge(v, umax + f * kUmaxSlots + blockIdx.x % kUmaxSlots);
    if (f < 3) {
#pragma unroll
      for (int m = 0; m < 8; ++m) park[(f * 8 + m) * NTH] = v[m];
    } else if (f == 3) {  // w_x:  n_y = u_z w_x,  n_z = -u_y w_x
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C uy = park[(8 + m) * NTH], uz = park[(16 + m) * NTH];
        ny[m] = pmul(uz, v[m]);
        nz[m] = pmul(C{-uy.x, -uy.y}, v[m]);
      }
    } else if (f == 4) {  // w_y:  n_x = -u_z w_y, n_z += u_x w_y
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C ux = park[m * NTH], uz = park[(16 + m) * NTH];
        nx[m] = pmul(C{-uz.x, -uz.y}, v[m]);
        nz[m] = pfma(ux, v[m], nz[m]);
      }
    } else {  // w_z: n_x += u_y w_z, n_y -= u_x w_z
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C ux = park[m * NTH], uy = park[(8 + m) * NTH];
        nx[m] = pfma(uy, v[m], nx[m]);
        ny[m] = pfms(ux, v[m], ny[m]);
      }
    }
  }
  for (int gg = 0; gg < 3; ++gg) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = gg == 0 ? nx[m] : (gg == 1 ? ny[m] : nz[m]);
    fft_line<H, -1>(v, t, tw + N + stage_tw_len(N), view);
    emit_r2c<C, N, L>(v, t, l, S, yb + gg * g.yb_f, line0, g.h, g.hs, tw);
  }
}

// xpass (3D), one warp per line group: lines (z, y), TX = N/16 <= 32 lanes per
// line, warp-level exchanges only.  Same arithmetic as k3_xpass.  The three
// velocity fields are parked in a thread-private shared slot [field][m][lane]
// (each thread reads back only what it wrote) so that the product accumulators
// and the prefetched next field fit in 128 registers.
template <typename R, int N, int WPB>
__global__ void __launch_bounds__(32 * WPB, 16 / WPB) k3_xpass_w(Geo g, long long line_base,
                                                                  typename CplxOf<R>::T *__restrict__ yb,
                                                                  const typename CplxOf<R>::T *__restrict__ tw,
                                                                  unsigned long long *__restrict__ umax) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, LPW = 32 / TX;
  constexpr int SL = xw_line_len<N, (LPW > 1)>();
  constexpr int WSM = LPW * SL + 3 * 8 * 32;  // per-warp shared elements
  C *S = dyn_smem<C>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane % TX, sub = lane / TX;
  const long long line = line_base + ((long long)blockIdx.x * WPB + warp) * LPW + sub;
  C *wsm = S + warp * WSM;
  const SmLine<C, N / 2> view{wsm + sub * SL};
  C *park = wsm + LPW * SL + lane;  // park[(a * 8 + m) * 32]
  const C *src = yb + line * g.hs;
  const C wt = __ldg(tw + t);
  C xn[8];
  load_line<C, TX>(xn, src, t, g.h);
  C nx[8], ny[8], nz[8];
#pragma unroll 1
  for (int f = 0; f < 6; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = c2r_pre_reg<C, N, TX>(xn, m, t, wt);
    if (f < 5) load_line<C, TX>(xn, src + (f + 1) * g.yb_f, t, g.h);  // prefetch the next field
    fft_line<H, +1, C, SmLine<C, N / 2>, SYNC_WARP>(v, t, tw + N + stage_tw_len(N), view);
    if (f < 3) {
      if (umax != nullptr) umax_merge(v, umax + f * kUmaxSlots + blockIdx.x % kUmaxSlots);
#pragma unroll
      for (int m = 0; m < 8; ++m) park[(f * 8 + m) * 32] = v[m];
    } else if (f == 3) {  // w_x:  n_y = u_z w_x,  n_z = -u_y w_x
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C uy = park[(8 + m) * 32], uz = park[(16 + m) * 32];
        ny[m] = pmul(uz, v[m]);
        nz[m] = pmul(C{-uy.x, -uy.y}, v[m]);
      }
    } else if (f == 4) {  // w_y:  n_x = -u_z w_y, n_z += u_x w_y
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C ux = park[m * 32], uz = park[(16 + m) * 32];
        nx[m] = pmul(C{-uz.x, -uz.y}, v[m]);
        nz[m] = pfma(ux, v[m], nz[m]);
      }
    } else {  // w_z: n_x += u_y w_z, n_y -= u_x w_z
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const C ux = park[m * 32], uy = park[(8 + m) * 32];
        nx[m] = pfma(uy, v[m], nx[m]);
        ny[m] = pfms(ux, v[m], ny[m]);
      }
    }
  }
#pragma unroll 1
  for (int gg = 0; gg < 3; ++gg) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = gg == 0 ? nx[m] : (gg == 1 ? ny[m] : nz[m]);
    fft_line<H, -1, C, SmLine<C, N / 2>, SYNC_WARP>(v, t, tw + N + stage_tw_len(N), view);
    C *dst = yb + gg * g.yb_f + line * g.hs;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const C x = r2c_post_reg<C, N, TX>(v, m, t, wt);
      const int k = t + TX * m;
      if (k < g.h) dst[k] = x;
    }
  }
}

// ---------------------------------------- paired-field x pass (FP32) ---
// Two real fields travel as one complex line z = x_a + i x_b, so each c2r or
// r2c of length N is half of one complex FFT of length N with no half-length
// pre- or post-processing.  A group of T = N/8 threads owns two lines A, B.
// The roundoff of a paired transform scales with the larger of its two
// fields, so only fields of like size share one: velocity with velocity,
// vorticity with vorticity (|w| is about |k| |u|, up to kc |u|).  Inverse:
// (u_z[A], u_z[B]), (w_z[A], w_z[B]), then per line (u_x, u_y), (w_x, w_y)
// and the product n = u x w at the line's 8 points per thread; forward:
// n_x + i n_y per line, and n_z[A] + i n_z[B] at the end.  The physical
// fields stay in registers.
//
// Slots: thread t holds index k = t + T m.  k is retained (k <= kc or
// k >= N - kc) only for m in {0, 1, 2, 5, 6, 7} (kc < 3N/8), so slots 3 and 4
// are zero on input and never needed on output.
__host__ __device__ constexpr int xp_sync(int T) { return T >= 64 ? T : SYNC_WARP; }
// per group: the double-buffered exchange line, the partner region (3T) and
// two staging buffers of the two input rows of a pair ([2][2][xp_row(N)])
__host__ __device__ constexpr int xp_row(int N) { return ((N - 1) / 3 + 2) / 2 * 2; }
// exchange line: swizzled and unpadded for 512 points (SmLineX), padded otherwise
__host__ __device__ constexpr int xp_line(int N) { return N == 512 ? N : smline_len(N); }
template <int N>
struct XpView {
  using T = SmLine<float2, N, true>;
};
template <>
struct XpView<512> {
  using T = SmLineX<float2, true>;
};
__host__ __device__ constexpr size_t xp_group_elems(int N) {
  return 2 * (size_t)xp_line(N) + 3 * (N / 8) + 4 * (size_t)xp_row(N);
}

// Copy the retained part of the rows X_a, X_b of one pair (h complex each,
// rounded up to whole 16-byte chunks; the row padding holds the extra
// column) into a staging buffer [2][xp_row(N)], 16 bytes per cp.async.
template <int N>
__device__ __forceinline__ void xp_stage(float2 *st, const float2 *__restrict__ ra, const float2 *__restrict__ rb,
                                         int t) {
  constexpr int T = N / 8, RW = xp_row(N), CH = RW / 2;  // chunks per row
  for (int c = t; c < 2 * CH; c += T) {
    const int r = c / CH, q = c % CH;
    cp_async_cg16(st + r * RW + 2 * q, (r ? rb : ra) + 2 * q, true);
  }
  cp_async_commit();
}
// z(k) = X_a(k) + i X_b(k) for k <= kc, conj X_a(N - k) + i conj X_b(N - k) for
// k >= N - kc, zero elsewhere; at k = 0 the real parts (the real part of the
// self-conjugate term, as the c2r of a Hermitian spectrum keeps).
template <int N>
__device__ __forceinline__ void xp_build(float2 (&v)[8], const float2 *st, int t, int kc) {
  constexpr int T = N / 8, RW = xp_row(N);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int m = j < 3 ? j : j + 2, k = t + T * m;
    const bool ok = j < 3 ? k <= kc : k >= N - kc;
    const int idx = j < 3 ? k : N - k;
    float2 z = czero<float2>();
    if (ok) {
      const float2 a = st[idx], b = st[RW + idx];
      z = j < 3 ? float2{a.x - b.y, a.y + b.x} : float2{a.x + b.y, b.x - a.y};
      if (k == 0) z = float2{a.x, b.x};
    }
    v[m] = z;
  }
  v[3] = v[4] = czero<float2>();
}
// Split the forward transform Z of z = x_a + i x_b (v[m] = Z(t + T m)) into
// X_a(k) = (Z(k) + conj Z(N-k))/2 and X_b(k) = (Z(k) - conj Z(N-k))/(2i) for
// k <= kc, written to da[k], db[k].  The partners Z(N - k) (slots 5..7 of
// other threads) go through the group's region P of 3T entries.
template <int N, int SY>
__device__ __forceinline__ void xp_emit(const float2 (&v)[8], int t, float2 *P, float2 *__restrict__ da,
                                        float2 *__restrict__ db, int kc) {
  constexpr int T = N / 8;
#pragma unroll
  for (int m = 5; m < 8; ++m) P[t + T * (m - 5)] = v[m];
  fft_sync<SY>();
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int k = t + T * m;
    if (k <= kc) {
      const float2 zk = v[m], zm = k == 0 ? v[0] : P[3 * T - k];
      da[k] = float2{0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)};
      db[k] = float2{0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x)};
    }
  }
}
// largest |x| over the warp merged into *slot (atomic maximum on the bits of a
// non-negative double)
__device__ __forceinline__ void umax_merge1(float m, unsigned long long *slot) {
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, (unsigned long long)__double_as_longlong((double)m));
}

template <int N>
__host__ __device__ constexpr int xp_groups() {
  return N >= 512 ? 2 : (N == 256 ? 4 : 8);
}
// resident blocks per SM the launch bounds ask for (512 threads per SM at
// most 128 registers a thread)
template <int N>
__host__ __device__ constexpr int xp_min_blocks() {
  return cmax(1, 512 / ((N / 8) * xp_groups<N>()));
}
template <int N, int GPB>
__global__ void __launch_bounds__((N / 8) * GPB, xp_min_blocks<N>())
    k3_xpass_p(Geo g, long long line_base, float2 *__restrict__ yb, const float2 *__restrict__ tw,
               unsigned long long *__restrict__ umax) {
  constexpr int T = N / 8, SY = xp_sync(T), RW = xp_row(N);
  static_assert(GPB <= 15 || SY == SYNC_WARP, "named barriers 1..15");
  float2 *S = dyn_smem<float2>();
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  float2 *gs = S + grp * xp_group_elems(N);
  using View = typename XpView<N>::T;
  const View view{gs, xp_line(N)};
  float2 *P = gs + 2 * xp_line(N);
  float2 *stage = P + 3 * T;  // [2 buffers][2 rows][RW]
  const float2 *stw = tw + N;  // stage tables of the length-N transform
  const long long lineA = line_base + ((long long)blockIdx.x * GPB + grp) * 2;
  const long long fs = g.yb_f, hs = g.hs;
  const int kc = g.kc;
  // the six input pairs (field, line) in order:
  //   0: (u_z A, u_z B)  1: (w_z A, w_z B)  2: (u_x A, u_y A)  3: (w_x A, w_y A)  4, 5: as 2, 3 for B
  auto src = [&](int i, int r) {
    const int f = i < 2 ? 2 + 3 * i : (i % 2 == 0 ? 0 : 3) + r;
    const long long ln = i < 2 ? lineA + r : lineA + (i - 2) / 2;
    return yb + f * fs + ln * hs;
  };
  xp_stage<N>(stage, src(0, 0), src(0, 1), t);
  float2 uz[8], wz[8], v[8];
  float nzA[8];
  // the next pair lands in the other buffer while this one is transformed
  // (that buffer was last read before the previous transform's barriers)
  auto next_pair = [&](int i) {
    if (i < 5) {
      xp_stage<N>(stage + ((i + 1) & 1) * 2 * RW, src(i + 1, 0), src(i + 1, 1), t);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    fft_sync<SY>();  // every thread's copies of pair i are visible
    xp_build<N>(v, stage + (i & 1) * 2 * RW, t, kc);
    fft_line<N, +1, float2, View, SY>(v, t, stw, view);
  };
  next_pair(0);
#pragma unroll
  for (int m = 0; m < 8; ++m) uz[m] = v[m];
  next_pair(1);
#pragma unroll
  for (int m = 0; m < 8; ++m) wz[m] = v[m];
  if (umax != nullptr) {
    float mz = 0.f;
#pragma unroll
    for (int m = 0; m < 8; ++m) mz = fmaxf(mz, fmaxf(fabsf(uz[m].x), fabsf(uz[m].y)));
    umax_merge1(mz, umax + 2 * kUmaxSlots + blockIdx.x % kUmaxSlots);
  }
#pragma unroll
  for (int ln = 0; ln < 2; ++ln) {
    const long long line = lineA + ln;
    next_pair(2 + 2 * ln);
    float2 uxy[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) uxy[m] = v[m];
    if (umax != nullptr) {
      float mx = 0.f, my = 0.f;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        mx = fmaxf(mx, fabsf(uxy[m].x));
        my = fmaxf(my, fabsf(uxy[m].y));
      }
      umax_merge1(mx, umax + 0 * kUmaxSlots + blockIdx.x % kUmaxSlots);
      umax_merge1(my, umax + 1 * kUmaxSlots + blockIdx.x % kUmaxSlots);
    }
    next_pair(3 + 2 * ln);
    // u = (uxy.x, uxy.y, uz), w = (v.x, v.y, wz) of this line: n = u x w
    float2 nxy[8];
    float nz[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float ux = uxy[m].x, uy = uxy[m].y, uzl = ln ? uz[m].y : uz[m].x;
      const float wx = v[m].x, wy = v[m].y, wzl = ln ? wz[m].y : wz[m].x;
      nxy[m] = float2{fmaf(uy, wzl, -uzl * wy), fmaf(uzl, wx, -ux * wzl)};
      nz[m] = fmaf(ux, wy, -uy * wx);
    }
    fft_line<N, -1, float2, View, SY>(nxy, t, stw, view);
    xp_emit<N, SY>(nxy, t, P, yb + line * hs, yb + fs + line * hs, kc);
    if (ln == 0) {
#pragma unroll
      for (int m = 0; m < 8; ++m) nzA[m] = nz[m];
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = float2{nzA[m], nz[m]};
      fft_line<N, -1, float2, View, SY>(v, t, stw, view);
      xp_emit<N, SY>(v, t, P, yb + 2 * fs + lineA * hs, yb + 2 * fs + line * hs, kc);
    }
  }
}

// fwd2: y forward of fields 0..nf-1 at plane z = blockIdx.y, keep retained ky;
// the next field's loads are issued before the current field is transformed.
template <typename R, int N, int W>
__global__ void __launch_bounds__((N / 8) * W) k3_fwd2(Geo g, int nf, int z0, const typename CplxOf<R>::T *__restrict__ yb,
                                                        typename CplxOf<R>::T *__restrict__ zb,
                                                        const typename CplxOf<R>::T *__restrict__ tw) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  C *sm = dyn_smem<C>();
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = blockIdx.x * W + w;
  const bool valid = kx < g.h;
  const int z = z0 + blockIdx.y;
  const C *in = yb + (long long)z * N * g.hs + kx;
  C *out = zb + (long long)z * g.c * g.hs + kx;
  C xn[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) xn[m] = valid ? ld_stream(in + (long long)(t + T * m) * g.hs) : czero<C>();
#pragma unroll 1
  for (int f = 0; f < nf; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = xn[m];
    if (f + 1 < nf) {
      const C *nin = in + (f + 1) * g.yb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) xn[m] = valid ? ld_stream(nin + (long long)(t + T * m) * g.hs) : czero<C>();
    }
    fft_line<N, -1>(v, t, tw + N, SmCol<C, col_db(N, W, sizeof(C), 0)>{sm + w, P, N * P});
    if (valid) {
      C *o = out + f * g.zb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int n = t + T * m;
        if (retained(n, N, g.kc)) o[(long long)compact_of(n, N, g.kc, g.c) * g.hs] = v[m];
      }
    }
  }
}

// ------------------------------------------------ TMA column-tile loads ---
// One mbarrier per block tracks the bytes of the tile in flight.  Waits are
// bounded: after kWaitSpins failed polls the waiting thread gives up and the
// block leaves the kernel together, with a nonzero code in the error word.
constexpr long long kWaitSpins = 1LL << 22;
enum ErrCode { ERR_TMA_TIMEOUT = 1 };

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
  for (long long i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// order this thread's earlier generic-proxy shared accesses before later
// async-proxy (TMA) accesses of the same shared memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// box at (x, y) of a 2D tensor map into shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// box at (x, y, z) of a 3D tensor map into shared memory, completing on bar
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// the same boxes into L2 only (no shared memory, no barrier)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *tm, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n" ::"l"(
                   reinterpret_cast<unsigned long long>(tm)),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *tm, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(
                   reinterpret_cast<unsigned long long>(tm)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}
// Linear index of the block launched `ahead` blocks after this one, or -1.
__device__ __forceinline__ long long block_ahead(int ahead) {
  const long long nb = (long long)blockIdx.y * gridDim.x + blockIdx.x + ahead;
  return (ahead > 0 && nb < (long long)gridDim.x * gridDim.y) ? nb : -1;
}

// inv2 with TMA loads: the same arithmetic as k3_inv2.  Field f's input
// column tile (the c retained ky rows of plane (f, z), W columns) lands in a
// dense [rows][W] shared tile from a 3D tensor map over zb (kx, ky, f N + z);
// the last box reaches past row c, where the tensor ends, so those rows are
// zero-filled without any memory traffic.  Same hand-off as k3_fwd2_tma.
//
// WZ (nf = 6, the curl fields): omega_z = i (kx u_y - ky u_x) is pointwise in
// (z, ky, kx), so it is not read from zb (its producer does not store it) but
// formed here from the landed tiles of u_x and u_y.  Two landing tiles;
// fields in the order u_x, u_y, omega_z, u_z, omega_x, omega_y: tile A takes
// u_x, u_z, omega_y and tile B u_y, omega_x, each refilled as soon as every
// thread has read it.  The same values and operations as a stored omega_z,
// so the results are bit for bit those of the six-field form.
//
// pf = 8 ahead + at (0: off): while item `at` is transformed, thread 0 sends
// the first tile(s) of the block launched `ahead` blocks later (one wave on,
// the block likely to follow on this SM) to L2, so that block's first wait
// ends on an L2 hit.
template <typename R, int N, int W, bool WZ = false>
__global__ void __launch_bounds__((N / 8) * W) k3_inv2_tma(Geo g, int nf, int z0, const __grid_constant__ CUtensorMap tm,
                                                            typename CplxOf<R>::T *__restrict__ yb,
                                                            const typename CplxOf<R>::T *__restrict__ tw, int *err,
                                                            int pf = 0) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr int CR = trunc_rows(N), BOXR = tma_box_rows(CR), NBOX = tma_boxes(CR);
  constexpr int LROWS = NBOX * BOXR;
  constexpr size_t LAND = (size_t)LROWS * W * sizeof(C);
  constexpr int NLAND = WZ ? 2 : 1;
  constexpr bool DB = col_db(N, W, sizeof(C), NLAND * LAND + 32);
  C *sm = dyn_smem<C>();
  C *land = sm + (DB ? 2 : 1) * N * P;  // [NLAND][LROWS][W]
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(land + NLAND * LROWS * W);  // one per tile
  int &s_ok = *reinterpret_cast<int *>(bar + 2);
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = blockIdx.x * W + w;
  const bool valid = kx < g.h;
  const int z = z0 + blockIdx.y;
  const int x8 = blockIdx.x * W * (int)(sizeof(C) / 8);
  // field f into landing tile q
  auto issue = [&](int q, int f) {
    mbar_expect_tx(bar + q, (unsigned)LAND);
#pragma unroll
    for (int b = 0; b < NBOX; ++b)
      tma_load_3d(land + (q * LROWS + b * BOXR) * W, &tm, x8, b * BOXR, f * N + z, bar + q);
  };
  // pf = 8 ahead + at: at item `at`, the first field(s) of the block launched
  // `ahead` blocks later go to L2
  auto prefetch_ahead = [&](int item) {
    if (threadIdx.x != 0 || pf < 8 || item != (pf & 7)) return;
    const long long nb = block_ahead(pf >> 3);
    if (nb < 0) return;
    const int bx = (int)(nb % gridDim.x), zz = z0 + (int)(nb / gridDim.x);
#pragma unroll
    for (int f = 0; f < (WZ ? 2 : 1); ++f)
#pragma unroll
      for (int b = 0; b < NBOX; ++b) tma_prefetch_3d(&tm, bx * W * (int)(sizeof(C) / 8), b * BOXR, f * N + zz);
  };
  int row[8];
  bool live[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int n = t + T * m;
    live[m] = valid && retained(n, N, g.kc);
    row[m] = compact_of(n, N, g.kc, g.c);
  }
  C *out = yb + (long long)z * N * g.hs + kx;
  // wait (bounded) for tile q's phase ph; false: the block leaves
  auto landed = [&](int q, unsigned ph) {
    if (threadIdx.x == 0) {
      bool ok = mbar_wait_bounded(bar + q, ph);
      if (!ok) {
        atomicExch(err, ERR_TMA_TIMEOUT);
        mbar_wait_bounded(bar + q, ph);  // give the copy in flight a last chance to land
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    mbar_try_wait(bar + q, ph);  // completed: acquires the tile for this thread
    return true;
  };
  auto transform_store = [&](C (&v)[8], int f) {
    fft_line<N, +1>(v, t, tw + N, SmCol<C, DB>{sm + w, P, N * P});
    if (valid) {
      C *o = out + f * g.yb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) o[(long long)(t + T * m) * g.hs] = v[m];
    }
  };
  if constexpr (!WZ) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      if (nf > 0) issue(0, 0);  // no copy may outlive the block
    }
    for (int f = 0; f < nf; ++f) {
      if (!landed(0, f & 1)) return;  // the whole block leaves together
      C v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = live[m] ? land[row[m] * W + w] : czero<C>();
      __syncthreads();  // every thread has its values: the tile may be refilled
      if (threadIdx.x == 0 && f + 1 < nf) {
        fence_proxy_async_smem();
        issue(0, f + 1);
      }
      prefetch_ahead(f);
      transform_store(v, f);
    }
  } else {
    const C *la = land, *lb = land + LROWS * W;
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
      issue(0, 0);  // u_x
      issue(1, 1);  // u_y
    }
    C v[8];
    // u_x (tile A stays: omega_z needs it)
    if (!landed(0, 0)) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = live[m] ? la[row[m] * W + w] : czero<C>();
    prefetch_ahead(0);
    transform_store(v, 0);
    // u_y (tile B stays)
    if (!landed(1, 0)) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = live[m] ? lb[row[m] * W + w] : czero<C>();
    prefetch_ahead(1);
    transform_store(v, 1);
    // omega_z = i (kx u_y - ky u_x); then both tiles are refilled
    {
      const R kxr = (R)kx;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        if (live[m]) {
          const R kyr = (R)ktr_of(row[m], g.kc, g.c);
          const C ux = la[row[m] * W + w], uy = lb[row[m] * W + w];
          v[m] = cmuli(C{kxr * uy.x - kyr * ux.x, kxr * uy.y - kyr * ux.y});
        } else {
          v[m] = czero<C>();
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        issue(0, 2);  // u_z
        issue(1, 3);  // omega_x
      }
      prefetch_ahead(2);
      transform_store(v, 5);
    }
    // u_z from tile A, which then takes omega_y
    if (!landed(0, 1)) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = live[m] ? la[row[m] * W + w] : czero<C>();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      issue(0, 4);
    }
    prefetch_ahead(3);
    transform_store(v, 2);
    // omega_x from tile B
    if (!landed(1, 1)) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = live[m] ? lb[row[m] * W + w] : czero<C>();
    prefetch_ahead(4);
    transform_store(v, 3);
    // omega_y from tile A
    if (!landed(0, 0)) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = live[m] ? la[row[m] * W + w] : czero<C>();
    prefetch_ahead(5);
    transform_store(v, 4);
  }
}

// fwd2 with TMA loads: the same arithmetic as k3_fwd2.  Field f's column tile
// (N rows of W columns, rows (f N + z) N .. + N - 1 of yb viewed as a 2D array
// of 8-byte elements) lands in a dense [N][W] shared tile, issued by thread 0
// one field ahead (boxes of at most 256 rows); thread 0 waits for it (bounded),
// the block barrier hands it to every thread, and each thread reads its eight
// values t + T m of column w from the tile.  pf: as in k3_inv2_tma, field 0
// of the block one wave later goes to L2 while field `at` is transformed.
template <typename R, int N, int W>
__global__ void __launch_bounds__((N / 8) * W) k3_fwd2_tma(Geo g, int nf, int z0, const __grid_constant__ CUtensorMap tm,
                                                            typename CplxOf<R>::T *__restrict__ zb,
                                                            const typename CplxOf<R>::T *__restrict__ tw, int *err,
                                                            int pf = 0) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr bool DB = col_db(N, W, sizeof(C), (size_t)N * W * sizeof(C) + 16);
  constexpr int BOXR = N < 256 ? N : 256;
  constexpr unsigned TILE_BYTES = (unsigned)(N * W * sizeof(C));
  static_assert(W * sizeof(C) == 128, "128-byte tile rows");
  C *sm = dyn_smem<C>();
  C *land = sm + (DB ? 2 : 1) * N * P;  // [N][W]
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(land + N * W);
  int &s_ok = *reinterpret_cast<int *>(bar + 1);
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = blockIdx.x * W + w;
  const bool valid = kx < g.h;
  const int z = z0 + blockIdx.y;
  const int x8 = blockIdx.x * W * (int)(sizeof(C) / 8);
  auto issue = [&](int f) {
    mbar_expect_tx(bar, TILE_BYTES);
    const int row0 = (f * N + z) * N;
#pragma unroll
    for (int r = 0; r < N; r += BOXR) tma_load_2d(land + r * W, &tm, x8, row0 + r, bar);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    if (nf > 0) issue(0);  // no copy may outlive the block
  }
  C *out = zb + (long long)z * g.c * g.hs + kx;
  for (int f = 0; f < nf; ++f) {
    if (threadIdx.x == 0) {
      bool ok = mbar_wait_bounded(bar, f & 1);
      if (!ok) {
        atomicExch(err, ERR_TMA_TIMEOUT);
        mbar_wait_bounded(bar, f & 1);  // give the copy in flight a last chance to land
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;  // the whole block leaves together
    mbar_try_wait(bar, f & 1);  // completed: acquires the tile for this thread
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = land[(t + T * m) * W + w];
    __syncthreads();  // every thread has its values: the tile may be refilled
    if (threadIdx.x == 0 && f + 1 < nf) {
      fence_proxy_async_smem();
      issue(f + 1);
    }
    // pf = 8 ahead + at: at field `at`, field 0 of the block launched `ahead`
    // blocks later goes to L2
    if (threadIdx.x == 0 && pf >= 8 && f == (pf & 7)) {
      const long long nb = block_ahead(pf >> 3);
      if (nb >= 0) {
        const int row0 = (z0 + (int)(nb / gridDim.x)) * N;
        for (int r = 0; r < N; r += BOXR) tma_prefetch_2d(&tm, (int)(nb % gridDim.x) * W * (int)(sizeof(C) / 8), row0 + r);
      }
    }
    fft_line<N, -1>(v, t, tw + N, SmCol<C, DB>{sm + w, P, N * P});
    if (valid) {
      C *o = out + f * g.zb_f;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int n = t + T * m;
        if (retained(n, N, g.kc)) o[(long long)compact_of(n, N, g.kc, g.c) * g.hs] = v[m];
      }
    }
  }
}

template <typename R>
struct StepBufs {
  using C = typename CplxOf<R>::T;
  const C *tw;
  const R *ef, *ef2;
  C *u, *acc;
  const C *F;
  C *zb;
  C *yb;
  C *dst;
  R dt;
  const double *dtp;  // time step in device memory (CFL stepping), nullable
  // hyper-viscous states: E, E2 indexed by |k|^2 (the operator does not
  // factor over the axes); null = the per-axis tables ef, ef2
  const R *ek2, *ek22;
  int wz;  // 1: the next inverse leaves omega_z (zb field 5) to the y pass
};

// The time step of a stage update: read from device memory at each use when
// it lives there (CFL stepping; a volatile load, so that no register holds it
// across the kernel), else the launch argument.
template <typename R>
__device__ __forceinline__ R stage_dt(const StepBufs<R> &b) {
  if (b.dtp == nullptr) return b.dt;
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(b.dtp));
  return (R)v;
}



// Integrating factors of a mode from the per-axis tables: exp(-nu |k|^2 dt)
// = prod_i exp(-nu k_i^2 dt) (tables indexed by |k_i| = 0 .. kc, computed in
// FP64 on the host and rounded to the state precision).
template <typename R>
__device__ __forceinline__ R axis_factor(const R *__restrict__ t, int k) {
  return __ldg(t + (k < 0 ? -k : k));
}

// Lawson IF-RK stage update for one mode with its operands already loaded
// (uu = state, a = accumulator); writes acc / u / dst at gi and returns the
// next stage input.  RK4 (stages RK1..RK4, k_s = N of the stage input):
//   RK1: acc = E u + dt/6 E k1,     next = E2 (u + dt/2 k1)
//   RK2: acc += dt/3 E2 k2,         next = E2 u + dt/2 k2
//   RK3: acc += dt/3 E2 k3,         next = E u + dt E2 k3
//   RK4: u = acc + dt/6 k4,         next = u
// RK2 midpoint (M1, M2): next = E2 (u + dt/2 k1);  u = E u + dt E2 k2.
template <int MODE, typename C, typename R>
__device__ __forceinline__ C rk_stage(C nv, C uu, C a, R e, R e2, const StepBufs<R> &b, long long gi) {
  const R dt = (MODE == MODE_RHS || MODE == MODE_PROJ) ? (R)0 : stage_dt(b);
  if (MODE == MODE_RK1) {
    const R c1 = dt * e / (R)6;
    b.acc[gi] = C{e * uu.x + c1 * nv.x, e * uu.y + c1 * nv.y};
    const R h = dt / (R)2;
    return C{e2 * (uu.x + h * nv.x), e2 * (uu.y + h * nv.y)};
  } else if (MODE == MODE_RK2) {
    const R c2 = dt * e2 / (R)3;
    b.acc[gi] = C{a.x + c2 * nv.x, a.y + c2 * nv.y};
    const R h = dt / (R)2;
    return C{e2 * uu.x + h * nv.x, e2 * uu.y + h * nv.y};
  } else if (MODE == MODE_RK3) {
    const R c2 = dt * e2 / (R)3;
    b.acc[gi] = C{a.x + c2 * nv.x, a.y + c2 * nv.y};
    const R c3 = dt * e2;
    return C{e * uu.x + c3 * nv.x, e * uu.y + c3 * nv.y};
  } else if (MODE == MODE_RK4) {
    const R c4 = dt / (R)6;
    const C un = C{a.x + c4 * nv.x, a.y + c4 * nv.y};
    b.u[gi] = un;
    return un;
  } else if (MODE == MODE_M1) {  // RK2 midpoint, stage 1: next = E2 (u + dt/2 N)
    const R h = dt / (R)2;
    return C{e2 * (uu.x + h * nv.x), e2 * (uu.y + h * nv.y)};
  } else if (MODE == MODE_M2) {  // RK2 stage 2: u <- E u + dt E2 N
    const R c = dt * e2;
    const C un = C{e * uu.x + c * nv.x, e * uu.y + c * nv.y};
    b.u[gi] = un;
    return un;
  } else {
    b.dst[gi] = nv;
    return czero<C>();
  }
}

// Lawson IF-RK stage update for one mode (see ns.h), loading its operands;
// e = E, e2 = E2 of the mode; returns the next stage input.
template <int MODE, typename C, typename R>
__device__ __forceinline__ C rk_update(C nv, long long idx, R e, R e2, const StepBufs<R> &b) {
  const R dt = (MODE >= MODE_RK1 && MODE <= MODE_RK4) ? stage_dt(b) : (R)0;  // M1/M2: loaded in rk_stage
  if (MODE == MODE_RK1) {
    const C uu = b.u[idx];
    const R c1 = dt * e / (R)6;
    b.acc[idx] = C{e * uu.x + c1 * nv.x, e * uu.y + c1 * nv.y};
    const R h = dt / (R)2;
    return C{e2 * (uu.x + h * nv.x), e2 * (uu.y + h * nv.y)};
  } else if (MODE == MODE_RK2) {
    const C uu = b.u[idx], a = b.acc[idx];
    const R c2 = dt * e2 / (R)3;
    b.acc[idx] = C{a.x + c2 * nv.x, a.y + c2 * nv.y};
    const R h = dt / (R)2;
    return C{e2 * uu.x + h * nv.x, e2 * uu.y + h * nv.y};
  } else if (MODE == MODE_RK3) {
    const C uu = b.u[idx], a = b.acc[idx];
    const R c2 = dt * e2 / (R)3;
    b.acc[idx] = C{a.x + c2 * nv.x, a.y + c2 * nv.y};
    const R c3 = dt * e2;
    return C{e * uu.x + c3 * nv.x, e * uu.y + c3 * nv.y};
  } else if (MODE == MODE_RK4) {
    const C a = b.acc[idx];
    const R c4 = dt / (R)6;
    const C un = C{a.x + c4 * nv.x, a.y + c4 * nv.y};
    b.u[idx] = un;
    return un;
  } else if (MODE == MODE_M1 || MODE == MODE_M2) {
    return rk_stage<MODE>(nv, b.u[idx], czero<C>(), e, e2, b, idx);
  } else {  // MODE_RHS, MODE_PROJ: write the term itself
    b.dst[idx] = nv;
    return czero<C>();
  }
}

// Slots of a column thread that can hold a retained wavenumber: n = t + (N/8) m
// is retained only for m in {0, 1, 2, 5, 6, 7} (kc < 3N/8 and N - kc > 5N/8),
// packed as j = 0..5.
__host__ __device__ constexpr int rk_slot(int m) { return m < 3 ? m : m - 2; }

// fwd1 (3D): z forward of the three product fields, dealias, 1/N^3, projection,
// forcing, RK stage; INV: curl + z inverse of the next stage input into zb.
// Persistent: each block walks the column tiles (ky row, W kx columns) with
// stride gridDim.x.  At the start of a tile the RK operands (u and/or acc) of
// its retained modes are copied with cp.async into thread-private shared slots
// [operand][comp][6][threads]; they land while the three forward transforms run.
template <typename R, int N, int W, int MODE, bool INV>
__global__ void __launch_bounds__((N / 8) * W) k3_fwd1(Geo g, StepBufs<R> b) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr int NT = T * W;
  // single exchange tile: the RK operand slots already take most of the
  // shared memory, and a larger carve-out would shrink the L1 that serves the
  // table and twiddle loads
  constexpr size_t EXTRA_SMEM = kSmemMax;  // forces a single buffer below
  constexpr bool NEED_U = MODE == MODE_RK1 || MODE == MODE_RK2 || MODE == MODE_RK3 || MODE == MODE_M1 || MODE == MODE_M2;
  constexpr bool NEED_ACC = MODE == MODE_RK2 || MODE == MODE_RK3 || MODE == MODE_RK4;
  C *sm = dyn_smem<C>();
  // operand slots [3][6][NT] each; a stage with one operand allocates one set
  C *rku = sm + N * P;
  C *rka = (NEED_U && NEED_ACC) ? rku + 18 * NT : rku;
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int nkt = g.hs / W;
  const int ntiles = g.c * nkt;
  const long long plane = (long long)g.c * g.hs;
  const long long st = g.st_comp;
  constexpr bool DB = col_db(N, W, sizeof(C), EXTRA_SMEM);
  const SmCol<C, DB> view{sm + w, P, N * P};
  const R scale = (R)1 / ((R)N * (R)N * (R)N);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int iy = tile / nkt;
    const int kx = (tile % nkt) * W + w;
    const bool valid = kx < g.h;
    const int ky = ktr_of(iy, g.kc, g.c);
    const R kxr = (R)kx, kyr = (R)ky;
    const long long col = (long long)iy * g.hs + kx;
    const R exy = valid ? axis_factor(b.ef, kx) * axis_factor(b.ef, ky) : (R)0;
    const R exy2 = valid ? axis_factor(b.ef2, kx) * axis_factor(b.ef2, ky) : (R)0;
    C s0[8], s1[8], s2[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const long long off = (long long)(t + T * m) * plane + col;
      s0[m] = valid ? ld_stream(b.zb + off) : czero<C>();
      s1[m] = valid ? ld_stream(b.zb + g.zb_f + off) : czero<C>();
      s2[m] = valid ? ld_stream(b.zb + 2 * g.zb_f + off) : czero<C>();
    }
    if (NEED_U || NEED_ACC) {
      // 16-byte L2-only copies: an 8-byte element type copies the slots of a
      // column pair (kx even, kx + 1: adjacent threads and adjacent slots)
      // from the even thread; kx + 1 < hs always, its value unused if >= h
      constexpr bool PAIR = sizeof(C) == 8;
      static_assert(!PAIR || W % 2 == 0, "column pairs");
      if (!PAIR || (w & 1) == 0) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          if (m == 3 || m == 4) continue;
          const int n = t + T * m;
          const bool ok = valid && retained(n, N, g.kc);
          const long long idx = ok ? (long long)compact_of(n, N, g.kc, g.c) * plane + col : 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int slot = (c * 6 + rk_slot(m)) * NT + threadIdx.x;
            if (NEED_U) cp_async_cg16(rku + slot, b.u + c * st + idx, ok);
            if (NEED_ACC) cp_async_cg16(rka + slot, b.acc + c * st + idx, ok);
          }
        }
      }
      cp_async_commit();
    }
    fft_line<N, -1>(s0, t, b.tw + N, view);
    fft_line<N, -1>(s1, t, b.tw + N, view);
    fft_line<N, -1>(s2, t, b.tw + N, view);
    if (NEED_U || NEED_ACC) {
      cp_async_wait_all();
      __syncwarp();  // the partner's copies into this thread's slots are visible
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int n = t + T * m;
      if (m == 3 || m == 4 || !valid || !retained(n, N, g.kc)) {
        s0[m] = s1[m] = s2[m] = czero<C>();
        continue;
      }
      const int kz = kfull_of(n, N, g.kc);
      const R kzr = (R)kz;
      const int k2 = kx * kx + ky * ky + kz * kz;
      C ax = cscale(s0[m], scale), ay = cscale(s1[m], scale), az = cscale(s2[m], scale);
      if (k2 == 0) {
        ax = ay = az = czero<C>();
      } else {
        const R inv = (R)1 / (R)k2;
        const C kd = C{(kxr * ax.x + kyr * ay.x + kzr * az.x) * inv, (kxr * ax.y + kyr * ay.y + kzr * az.y) * inv};
        ax = C{ax.x - kxr * kd.x, ax.y - kxr * kd.y};
        ay = C{ay.x - kyr * kd.x, ay.y - kyr * kd.y};
        az = C{az.x - kzr * kd.x, az.y - kzr * kd.y};
      }
      const long long idx = (long long)compact_of(n, N, g.kc, g.c) * plane + col;
      if (MODE != MODE_PROJ && b.F != nullptr) {
        ax = cadd(ax, b.F[idx]);
        ay = cadd(ay, b.F[st + idx]);
        az = cadd(az, b.F[2 * st + idx]);
      }
      C nv[3] = {ax, ay, az};
      C out[3];
      R e, e2;
      if (b.ek2 != nullptr) {
        e = __ldg(b.ek2 + k2);
        e2 = __ldg(b.ek22 + k2);
      } else {
        e = exy * axis_factor(b.ef, kz);
        e2 = exy2 * axis_factor(b.ef2, kz);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int slot = (c * 6 + rk_slot(m)) * NT + threadIdx.x;
        const long long gi = c * st + idx;
        out[c] = rk_stage<MODE>(nv[c], NEED_U ? rku[slot] : czero<C>(), NEED_ACC ? rka[slot] : czero<C>(), e, e2, b, gi);
      }
      s0[m] = out[0];
      s1[m] = out[1];
      s2[m] = out[2];
    }
    if (INV) {
      // omega_z = i (kx u_y - ky u_x) has no kz: its z inverse is formed from
      // the inverses of u_x and u_y (five transforms for six fields)
      C zx[8];
      for (int f = 0; f < 5; ++f) {
        C v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const R kzr = (R)kfull_of(t + T * m, N, g.kc);
          if (f == 0) v[m] = s0[m];
          else if (f == 1) v[m] = s1[m];
          else if (f == 2) v[m] = s2[m];
          else if (f == 3) v[m] = cmuli(C{kyr * s2[m].x - kzr * s1[m].x, kyr * s2[m].y - kzr * s1[m].y});
          else v[m] = cmuli(C{kzr * s0[m].x - kxr * s2[m].x, kzr * s0[m].y - kxr * s2[m].y});
        }
        fft_line<N, +1>(v, t, b.tw + N, view);
        if (valid) {
#pragma unroll
          for (int m = 0; m < 8; ++m) b.zb[f * g.zb_f + (long long)(t + T * m) * plane + col] = v[m];
        }
        if (f == 0) {
#pragma unroll
          for (int m = 0; m < 8; ++m) zx[m] = v[m];
        } else if (f == 1 && valid) {
#pragma unroll
          for (int m = 0; m < 8; ++m)
            b.zb[5 * g.zb_f + (long long)(t + T * m) * plane + col] =
                cmuli(C{kxr * v[m].x - kyr * zx[m].x, kxr * v[m].y - kyr * zx[m].y});
        }
      }
    }
  }
}

// fwd1 with a shared spectral tile (FP32 at 256 and 512 points): the same
// arithmetic as k3_fwd1, rearranged so that a thread holds one field at a
// time and two 512-thread blocks share an SM (64 registers).  Per column
// tile (ky row, W kx columns), persistent over tiles:
//   1. the three z forward transforms, each field's retained rows into the
//      tile Q [3][c][W];
//   2. per retained mode (thread (w, t): rows t, t + T, ...): normalise,
//      project, add forcing, RK stage with its operands loaded from global
//      memory, next stage input back into Q;
//   3. (INV) the curl and the z inverse of the next stage input from Q: five
//      transforms for six fields, omega_z = i (kx u_y - ky u_x) formed from
//      the inverse of u_y and the inverse of u_x this thread has just stored.
// The other block of the SM overlaps phase 2's memory latency.
template <typename R, int N, int W>
__host__ __device__ constexpr size_t fwd1t_smem() {
  return col_tile_bytes(N, W, 2 * sizeof(R)) + (size_t)3 * trunc_rows(N) * W * 2 * sizeof(R);
}
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// PFR >= 0: the tile's RK operand rows are prefetched into L2 while phase 1
// transforms field PFR; PFN >= 0: the next tile's three input columns while
// phase 3 transforms field PFN (a prefetch ahead of its loads, not a copy).
template <typename R, int N, int W, int MODE, bool INV, bool PF = false, int UR = 1, int MINB = 2, int PFR = -1,
          int PFN = -1>
__global__ void __launch_bounds__((N / 8) * W, MINB) k3_fwd1t(Geo g, StepBufs<R> b) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr int CR = trunc_rows(N);
  constexpr bool NEED_U = MODE == MODE_RK1 || MODE == MODE_RK2 || MODE == MODE_RK3 || MODE == MODE_M1 || MODE == MODE_M2;
  constexpr bool NEED_ACC = MODE == MODE_RK2 || MODE == MODE_RK3 || MODE == MODE_RK4;
  C *sm = dyn_smem<C>();
  C *Q = sm + N * P;  // [3][CR][W]
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int nkt = g.hs / W;
  const int ntiles = g.c * nkt;
  const long long plane = (long long)g.c * g.hs;
  const long long st = g.st_comp;
  const SmCol<C, false> view{sm + w, P, 0};
  const R scale = (R)1 / ((R)N * (R)N * (R)N);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int iy = tile / nkt;
    const int kx = (tile % nkt) * W + w;
    const bool valid = kx < g.h;
    const int ky = ktr_of(iy, g.kc, g.c);
    const long long col = (long long)iy * g.hs + kx;
    // 1. forward transforms into Q (rows of the retained kz only); PF: the
    // next field's column is loaded while the current one is transformed
    C xn[8];
    if (PF) {
#pragma unroll
      for (int m = 0; m < 8; ++m) xn[m] = valid ? ld_stream(b.zb + (long long)(t + T * m) * plane + col) : czero<C>();
    }
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
      C v[8];
      if (f == PFR) {  // the W-column row segments of u, acc and F this tile's phase 2 reads
        const long long col0 = (long long)iy * g.hs + (tile % nkt) * W;
        const C *fo = MODE != MODE_PROJ ? b.F : nullptr;  // operands in order, null ones last
        const C *op0 = NEED_U ? b.u : (NEED_ACC ? b.acc : fo);
        const C *op1 = NEED_U && NEED_ACC ? b.acc : (NEED_U || NEED_ACC ? fo : nullptr);
        const C *op2 = NEED_U && NEED_ACC ? fo : nullptr;
        const int no = (op0 != nullptr) + (op1 != nullptr) + (op2 != nullptr);
        for (int i = threadIdx.x; i < 3 * no * CR; i += blockDim.x) {
          const int o = i / CR, r = i % CR;
          const C *op = o < 3 ? op0 : (o < 6 ? op1 : op2);
          prefetch_l2(op + (o % 3) * st + (long long)r * plane + col0);
        }
      }
      if (PF) {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = xn[m];
        if (f < 2) {
#pragma unroll
          for (int m = 0; m < 8; ++m)
            xn[m] = valid ? ld_stream(b.zb + (f + 1) * g.zb_f + (long long)(t + T * m) * plane + col) : czero<C>();
        }
      } else {
#pragma unroll
        for (int m = 0; m < 8; ++m)
          v[m] = valid ? ld_stream(b.zb + f * g.zb_f + (long long)(t + T * m) * plane + col) : czero<C>();
      }
      fft_line<N, -1>(v, t, b.tw + N, view);
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int n = t + T * m;
        if (m != 3 && m != 4 && retained(n, N, g.kc)) Q[(f * CR + compact_of(n, N, g.kc, g.c)) * W + w] = v[m];
      }
    }
    __syncthreads();
    // 2. projection, forcing and the RK stage per retained mode (UR rows of
    // a thread at a time, their operand loads issued together)
    if (valid) {
      const R kxr = (R)kx, kyr = (R)ky;
      const R exy = axis_factor(b.ef, kx) * axis_factor(b.ef, ky);
      const R exy2 = axis_factor(b.ef2, kx) * axis_factor(b.ef2, ky);
#pragma unroll 1
      for (int r0 = t; r0 < CR; r0 += UR * T) {
        C uu[UR][3], aa[UR][3];
#pragma unroll
        for (int q = 0; q < UR; ++q) {
          const int r = r0 + q * T;
          const long long idx = (long long)(r < CR ? r : 0) * plane + col;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uu[q][c] = NEED_U && r < CR ? ld_stream(b.u + c * st + idx) : czero<C>();
            aa[q][c] = NEED_ACC && r < CR ? ld_stream(b.acc + c * st + idx) : czero<C>();
          }
        }
#pragma unroll
        for (int q = 0; q < UR; ++q) {
          const int r = r0 + q * T;
          if (r >= CR) break;
          const int kz = ktr_of(r, g.kc, g.c);
          const R kzr = (R)kz;
          const int k2 = kx * kx + ky * ky + kz * kz;
          C ax = cscale(Q[r * W + w], scale), ay = cscale(Q[(CR + r) * W + w], scale),
            az = cscale(Q[(2 * CR + r) * W + w], scale);
          if (k2 == 0) {
            ax = ay = az = czero<C>();
          } else {
            const R inv = (R)1 / (R)k2;
            const C kd = C{(kxr * ax.x + kyr * ay.x + kzr * az.x) * inv, (kxr * ax.y + kyr * ay.y + kzr * az.y) * inv};
            ax = C{ax.x - kxr * kd.x, ax.y - kxr * kd.y};
            ay = C{ay.x - kyr * kd.x, ay.y - kyr * kd.y};
            az = C{az.x - kzr * kd.x, az.y - kzr * kd.y};
          }
          const long long idx = (long long)r * plane + col;
          if (MODE != MODE_PROJ && b.F != nullptr) {
            ax = cadd(ax, b.F[idx]);
            ay = cadd(ay, b.F[st + idx]);
            az = cadd(az, b.F[2 * st + idx]);
          }
          R e, e2;
          if (b.ek2 != nullptr) {
            e = __ldg(b.ek2 + k2);
            e2 = __ldg(b.ek22 + k2);
          } else {
            e = exy * axis_factor(b.ef, kz);
            e2 = exy2 * axis_factor(b.ef2, kz);
          }
          const C nv[3] = {ax, ay, az};
#pragma unroll
          for (int c = 0; c < 3; ++c)
            Q[(c * CR + r) * W + w] = rk_stage<MODE>(nv[c], uu[q][c], aa[q][c], e, e2, b, c * st + idx);
        }
      }
    }
    if (INV) {
      __syncthreads();
      // 3. curl and z inverse of the next stage input
      const R kxr = (R)kx, kyr = (R)ky;
#pragma unroll 1
      for (int f = 0; f < 5; ++f) {
        C v[8];
        if (f == PFN && tile + (int)gridDim.x < ntiles) {
          const int nt = tile + gridDim.x;
          const long long col0 = (long long)(nt / nkt) * g.hs + (nt % nkt) * W;
          for (int i = threadIdx.x; i < 3 * N; i += blockDim.x)
            prefetch_l2(b.zb + (i / N) * g.zb_f + (long long)(i % N) * plane + col0);
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int n = t + T * m;
          C x = czero<C>();
          if (m != 3 && m != 4 && retained(n, N, g.kc)) {
            const int r = compact_of(n, N, g.kc, g.c);
            const R kzr = (R)kfull_of(n, N, g.kc);
            if (f < 3) {
              x = Q[(f * CR + r) * W + w];
            } else if (f == 3) {  // omega_x = i (ky u_z - kz u_y)
              const C a2 = Q[(2 * CR + r) * W + w], a1 = Q[(CR + r) * W + w];
              x = cmuli(C{kyr * a2.x - kzr * a1.x, kyr * a2.y - kzr * a1.y});
            } else {  // omega_y = i (kz u_x - kx u_z)
              const C a0 = Q[r * W + w], a2 = Q[(2 * CR + r) * W + w];
              x = cmuli(C{kzr * a0.x - kxr * a2.x, kzr * a0.y - kxr * a2.y});
            }
          }
          v[m] = x;
        }
        fft_line<N, +1>(v, t, b.tw + N, view);
        if (valid) {
#pragma unroll
          for (int m = 0; m < 8; ++m) b.zb[f * g.zb_f + (long long)(t + T * m) * plane + col] = v[m];
          if (f == 1 && !b.wz) {  // omega_z = i (kx u_y - ky u_x), u_x as this thread stored it for f = 0
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const long long o = (long long)(t + T * m) * plane + col;
              const C ux = b.zb[o];
              b.zb[5 * g.zb_f + o] = cmuli(C{kxr * v[m].x - kyr * ux.x, kxr * v[m].y - kyr * ux.y});
            }
          }
        }
      }
    }
    __syncthreads();  // Q and the exchange tile are free for the next tile
  }
}

// ================================================================== 2D ====
// inv1 (2D): y inverse from a state-shaped array.  VEL: four fields
// u_x = i ky psi, u_y = -i kx psi, d_x w = i kx w, d_y w = i ky w with
// psi = w/|k|^2; otherwise one field (w itself).
template <typename R, int N, int W, bool VEL>
__device__ __forceinline__ void inv1_2d_unit(const Geo &g, const typename CplxOf<R>::T *__restrict__ src,
                                             typename CplxOf<R>::T *__restrict__ yb,
                                             const typename CplxOf<R>::T *__restrict__ tw, int unit,
                                             typename CplxOf<R>::T *sm) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr size_t EXTRA_SMEM = 0;
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = unit * W + w;
  const bool valid = kx < g.h;
  constexpr bool DB = col_db(N, W, sizeof(C), EXTRA_SMEM);
  const SmCol<C, DB> view{sm + w, P, N * P};
  C wv[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int n = t + T * m;
    wv[m] = (valid && retained(n, N, g.kc)) ? src[(long long)compact_of(n, N, g.kc, g.c) * g.hs + kx] : czero<C>();
  }
  constexpr int NF = VEL ? 4 : 1;
  for (int f = 0; f < NF; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (!VEL) {
        v[m] = wv[m];
        continue;
      }
      const int ky = kfull_of(t + T * m, N, g.kc);
      const int k2 = kx * kx + ky * ky;
      const R kxr = (R)kx, kyr = (R)ky;
      const R ip = k2 > 0 ? (R)1 / (R)k2 : (R)0;
      if (f == 0) v[m] = cmuli(cscale(wv[m], kyr * ip));
      else if (f == 1) v[m] = cmuli(cscale(wv[m], -kxr * ip));
      else if (f == 2) v[m] = cmuli(cscale(wv[m], kxr));
      else v[m] = cmuli(cscale(wv[m], kyr));
    }
    fft_line<N, +1>(v, t, tw + N, view);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 8; ++m) yb[f * g.yb_f + (long long)(t + T * m) * g.hs + kx] = v[m];
    }
  }
}

template <typename R, int N, int W, bool VEL>
__global__ void __launch_bounds__((N / 8) * W) k2_inv1(Geo g, const typename CplxOf<R>::T *__restrict__ src,
                                                        typename CplxOf<R>::T *__restrict__ yb,
                                                        const typename CplxOf<R>::T *__restrict__ tw) {
  using C = typename CplxOf<R>::T;
  inv1_2d_unit<R, N, W, VEL>(g, src, yb, tw, blockIdx.x, dyn_smem<C>());
}

// xpass (2D): lines y; fields u_x, u_y, d_x w, d_y w in; n = -(u . grad w)
// out (field 0).
template <typename R, int N, int L>
__global__ void __launch_bounds__((N / 16) * L) k2_xpass(Geo g, typename CplxOf<R>::T *__restrict__ yb,
                                                          const typename CplxOf<R>::T *__restrict__ tw,
                                                          unsigned long long *__restrict__ umax) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, SL = smline_len(H);
  C *S = dyn_smem<C>();
  const int t = threadIdx.x % TX, l = threadIdx.x / TX;
  const long long line0 = (long long)blockIdx.x * L;
  const SmLine<C> view{S + l * SL};
  C ux[8], uy[8], nn[8];
  for (int f = 0; f < 4; ++f) {
    __syncthreads();
    stage_lines<C, H, L>(S, yb + f * g.yb_f, line0, g.h, g.hs);
    __syncthreads();
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = c2r_pre<C, N>(S + l * SL, t + TX * m, tw);
    fft_line<H, +1>(v, t, tw + N + stage_tw_len(N), view);
    if (umax != nullptr && f < 2) umax_merge(v, umax + f * kUmaxSlots + blockIdx.x % kUmaxSlots);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (f == 0) ux[m] = v[m];
      else if (f == 1) uy[m] = v[m];
      else if (f == 2) nn[m] = pmul(C{-ux[m].x, -ux[m].y}, v[m]);
      else nn[m] = pfms(uy[m], v[m], nn[m]);
    }
  }
  fft_line<H, -1>(nn, t, tw + N + stage_tw_len(N), view);
  emit_r2c<C, N, L>(nn, t, l, S, yb, line0, g.h, g.hs, tw);
}

// xpass (2D), one warp per line group (see k3_xpass_w); `unit` selects the
// group of WPB * LPW lines.
// Sw is this warp's own shared region (at least LPW line buffers).
template <typename R, int N, int WPB>
__device__ __forceinline__ void xpass_2d_unit(const Geo &g, typename CplxOf<R>::T *__restrict__ yb,
                                              const typename CplxOf<R>::T *__restrict__ tw, int unit,
                                              typename CplxOf<R>::T *Sw, unsigned long long *umax = nullptr) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, LPW = 32 / TX;
  constexpr int SL = xw_line_len<N, (LPW > 1)>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane % TX, sub = lane / TX;
  const long long line = ((long long)unit * WPB + warp) * LPW + sub;
  const SmLine<C, N / 2> view{Sw + sub * SL};
  const C *src = yb + line * g.hs;
  const C wt = __ldg(tw + t);
  C xn[8];
  load_line<C, TX>(xn, src, t, g.h);
  C ux[8], uy[8], nn[8];
#pragma unroll 1
  for (int f = 0; f < 4; ++f) {
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = c2r_pre_reg<C, N, TX>(xn, m, t, wt);
    if (f < 3) load_line<C, TX>(xn, src + (f + 1) * g.yb_f, t, g.h);
    fft_line<H, +1, C, SmLine<C, N / 2>, SYNC_WARP>(v, t, tw + N + stage_tw_len(N), view);
    if (umax != nullptr && f < 2) umax_merge(v, umax + f * kUmaxSlots + unit % kUmaxSlots);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (f == 0) ux[m] = v[m];
      else if (f == 1) uy[m] = v[m];
      else if (f == 2) nn[m] = pmul(C{-ux[m].x, -ux[m].y}, v[m]);
      else nn[m] = pfms(uy[m], v[m], nn[m]);
    }
  }
  fft_line<H, -1, C, SmLine<C, N / 2>, SYNC_WARP>(nn, t, tw + N + stage_tw_len(N), view);
  C *dst = yb + line * g.hs;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const C x = r2c_post_reg<C, N, TX>(nn, m, t, wt);
    const int k = t + TX * m;
    if (k < g.h) dst[k] = x;
  }
}

template <typename R, int N, int WPB>
__global__ void __launch_bounds__(32 * WPB) k2_xpass_w(Geo g, typename CplxOf<R>::T *__restrict__ yb,
                                                        const typename CplxOf<R>::T *__restrict__ tw,
                                                        unsigned long long *__restrict__ umax) {
  using C = typename CplxOf<R>::T;
  constexpr int LPW = 32 / (N / 16);
  xpass_2d_unit<R, N, WPB>(g, yb, tw, blockIdx.x,
                           dyn_smem<C>() + (threadIdx.x >> 5) * LPW * xw_line_len<N, (LPW > 1)>(), umax);
}

// fwd1 (2D): y forward of field 0, dealias, 1/N^2, forcing, RK stage; INV:
// the four inverse fields of the next stage input.  `unit` is the kx tile.
template <typename R, int N, int W, int MODE, bool INV>
__device__ __forceinline__ void fwd1_2d_unit(const Geo &g, const StepBufs<R> &b, int unit,
                                             typename CplxOf<R>::T *sm) {
  using C = typename CplxOf<R>::T;
  constexpr int T = N / 8;
  constexpr int P = pitch_of(W, sizeof(C));
  constexpr size_t EXTRA_SMEM = 0;
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = unit * W + w;
  const bool valid = kx < g.h;
  constexpr bool DB = col_db(N, W, sizeof(C), EXTRA_SMEM);
  const SmCol<C, DB> view{sm + w, P, N * P};
  const R scale = (R)1 / ((R)N * (R)N);
  C s[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) s[m] = valid ? b.yb[(long long)(t + T * m) * g.hs + kx] : czero<C>();
  fft_line<N, -1>(s, t, b.tw + N, view);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int n = t + T * m;
    if (!valid || !retained(n, N, g.kc)) {
      s[m] = czero<C>();
      continue;
    }
    const int ky = kfull_of(n, N, g.kc);
    const int k2 = kx * kx + ky * ky;
    C nv = k2 == 0 ? czero<C>() : cscale(s[m], scale);
    const long long idx = (long long)compact_of(n, N, g.kc, g.c) * g.hs + kx;
    if (MODE != MODE_PROJ && b.F != nullptr) nv = cadd(nv, b.F[idx]);
    R e, e2;
    if (b.ek2 != nullptr) {
      e = __ldg(b.ek2 + k2);
      e2 = __ldg(b.ek22 + k2);
    } else {
      e = axis_factor(b.ef, kx) * axis_factor(b.ef, ky);
      e2 = axis_factor(b.ef2, kx) * axis_factor(b.ef2, ky);
    }
    s[m] = rk_update<MODE>(nv, idx, e, e2, b);
  }
  if (INV) {
    for (int f = 0; f < 4; ++f) {
      C v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int ky = kfull_of(t + T * m, N, g.kc);
        const int k2 = kx * kx + ky * ky;
        const R kxr = (R)kx, kyr = (R)ky;
        const R ip = k2 > 0 ? (R)1 / (R)k2 : (R)0;
        if (f == 0) v[m] = cmuli(cscale(s[m], kyr * ip));
        else if (f == 1) v[m] = cmuli(cscale(s[m], -kxr * ip));
        else if (f == 2) v[m] = cmuli(cscale(s[m], kxr));
        else v[m] = cmuli(cscale(s[m], kyr));
      }
      fft_line<N, +1>(v, t, b.tw + N, view);
      if (valid) {
#pragma unroll
        for (int m = 0; m < 8; ++m) b.yb[f * g.yb_f + (long long)(t + T * m) * g.hs + kx] = v[m];
      }
    }
  }
}


template <typename R, int N, int W, int MODE, bool INV>
__global__ void __launch_bounds__((N / 8) * W) k2_fwd1(Geo g, StepBufs<R> b) {
  using C = typename CplxOf<R>::T;
  fwd1_2d_unit<R, N, W, MODE, INV>(g, b, blockIdx.x, dyn_smem<C>());
}

// ================================================ real lines (set / get) ===
// xfwd_real: FP64 real lines of length N -> X[0..h-1] (row stride hs).
template <typename R, int N, int L>
__global__ void __launch_bounds__((N / 16) * L) k_xfwd_real(Geo g, const double *__restrict__ phys,
                                                             typename CplxOf<R>::T *__restrict__ dst,
                                                             const typename CplxOf<R>::T *__restrict__ tw) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, SL = smline_len(H);
  C *S = dyn_smem<C>();
  const int t = threadIdx.x % TX, l = threadIdx.x / TX;
  const long long line0 = (long long)blockIdx.x * L;
  const double2 *row = reinterpret_cast<const double2 *>(phys + (line0 + l) * N);
  C v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const double2 p = row[t + TX * m];
    v[m] = C{(R)p.x, (R)p.y};
  }
  fft_line<H, -1>(v, t, tw + N + stage_tw_len(N), SmLine<C>{S + l * SL});
  emit_r2c<C, N, L>(v, t, l, S, dst, line0, g.h, g.hs, tw);
}

// xinv_real: X[0..h-1] (row stride hs) -> FP64 real lines of length N.
template <typename R, int N, int L>
__global__ void __launch_bounds__((N / 16) * L) k_xinv_real(Geo g, const typename CplxOf<R>::T *__restrict__ src,
                                                             double *__restrict__ phys,
                                                             const typename CplxOf<R>::T *__restrict__ tw) {
  using C = typename CplxOf<R>::T;
  constexpr int H = N / 2, TX = H / 8, SL = smline_len(H);
  C *S = dyn_smem<C>();
  const int t = threadIdx.x % TX, l = threadIdx.x / TX;
  const long long line0 = (long long)blockIdx.x * L;
  stage_lines<C, H, L>(S, src, line0, g.h, g.hs);
  __syncthreads();
  C v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = c2r_pre<C, N>(S + l * SL, t + TX * m, tw);
  fft_line<H, +1>(v, t, tw + N + stage_tw_len(N), SmLine<C>{S + l * SL});
  double2 *row = reinterpret_cast<double2 *>(phys + (line0 + l) * N);
#pragma unroll
  for (int m = 0; m < 8; ++m) row[t + TX * m] = make_double2((double)v[m].x, (double)v[m].y);
}

// ============================================================= launching ===
template <typename K>
inline void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
inline StepBufs<R> step_bufs(const Args &a) {
  using C = typename CplxOf<R>::T;
  StepBufs<R> b;
  b.tw = (const C *)a.tw;
  b.ef = (const R *)a.ef;
  b.ef2 = (const R *)a.ef2;
  b.u = (C *)a.u;
  b.acc = (C *)a.acc;
  b.F = (const C *)a.F;
  b.zb = (C *)a.zb;
  b.yb = (C *)a.yb;
  b.dst = (C *)a.dst;
  b.dt = (R)a.dt;
  b.dtp = a.dtp;
  b.ek2 = (const R *)a.ek2;
  b.ek22 = (const R *)a.ek22;
  b.wz = a.wz;
  return b;
}

// fwd1 with the shared spectral tile in a given shape: W columns, next-field
// prefetch PF, UR rows of RK operands in flight, MINB resident blocks per SM
template <typename R, int N, int W, bool PF, int UR, int MINB, int PFR = -1, int PFN = -1>
struct Fwd1T {
  static constexpr size_t SM = fwd1t_smem<R, N, W>();
  static void prepare() {
    set_smem(k3_fwd1t<R, N, W, MODE_RK1, true, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_RK2, true, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_RK3, true, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_RK4, true, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_RHS, false, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_PROJ, false, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_M1, true, PF, UR, MINB, PFR, PFN>, SM);
    set_smem(k3_fwd1t<R, N, W, MODE_M2, true, PF, UR, MINB, PFR, PFN>, SM);
  }
  static void launch(int mode, int nsm, const Geo &g, const StepBufs<R> &b, cudaStream_t s) {
    const int tiles = g.c * (g.hs / W), grid = cmin(tiles, MINB * (nsm > 0 ? nsm : 1));
    constexpr int NT = (N / 8) * W;
    switch (mode) {
      case MODE_RK1: k3_fwd1t<R, N, W, MODE_RK1, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_RK2: k3_fwd1t<R, N, W, MODE_RK2, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_RK3: k3_fwd1t<R, N, W, MODE_RK3, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_RK4: k3_fwd1t<R, N, W, MODE_RK4, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_RHS: k3_fwd1t<R, N, W, MODE_RHS, false, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_M1: k3_fwd1t<R, N, W, MODE_M1, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      case MODE_M2: k3_fwd1t<R, N, W, MODE_M2, true, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
      default: k3_fwd1t<R, N, W, MODE_PROJ, false, PF, UR, MINB, PFR, PFN><<<grid, NT, SM, s>>>(g, b); break;
    }
  }
};
// The shape used: 16 columns (128-byte rows) with the next field prefetched
// and two rows of RK operands in flight; 512 points: 1024 threads, one block
// per SM (fwd1 1.146 -> 1.034 ms per launch against the register-resident
// form); 256 points: 512 threads, two blocks per SM (0.154 -> 0.148 ms;
// 32 columns: 0.164 ms); 1024 points: 8 columns, 1024 threads, one block per
// SM (exchange tile 74 KB + spectral tile 131 KB).  L2 prefetches (256 and
// 512 points): the RK operands while the last input field is transformed, the
// next tile's inputs while the fourth of the five inverse transforms runs
// (512 points: 0.980 -> 0.937 ms; the RK operands one field earlier 0.952, the
// next tile one field later 0.966, either one alone 0.960 / 0.963; at 1024
// points, with half-line rows, 14.51 -> 15.04 ms, so none there).
template <typename R, int N>
using Fwd1Pick = Fwd1T<R, N, (N == 1024 ? 8 : 16), true, 2, (N == 256 ? 2 : 1), (N == 1024 ? -1 : 2),
                       (N == 1024 ? -1 : 3)>;

// Prefetch argument of the TMA y passes (see k3_inv2_tma): the block one
// wave later (SMs x resident blocks per SM), at item `at` of this block.
inline int wave_pf(int nsm, int per_sm, int at) { return 8 * (nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1) + at; }

template <typename R, int N>
struct Launch3 {
  using C = typename CplxOf<R>::T;
  static constexpr int T = N / 8;
  static constexpr int WL = w_light<R, N>();
  static constexpr int WH = w_heavy<R, N>();
  static constexpr int L = x_lines<R, N>();
  static constexpr int WYI = w_yinv<R, N>(), WYF = w_yfwd<R, N>();
  static constexpr size_t SM_L = col_smem(N, WL, sizeof(C), 0);
  static constexpr size_t SM_YI = col_smem(N, WYI, sizeof(C), 0), SM_YF = col_smem(N, WYF, sizeof(C), 0);
  // y passes with TMA tile loads where the landing tile fits beside the
  // exchange tile (forward: 128-byte tile rows)
  static constexpr size_t SM_YFT = col_smem(N, WYF, sizeof(C), (size_t)N * WYF * sizeof(C) + 16);
  static constexpr bool YF_TMA = WYF * sizeof(C) == 128 && SM_YFT <= kSmemMax;
  static constexpr size_t SM_YIT = col_smem(
      N, WYI, sizeof(C), (size_t)tma_boxes(trunc_rows(N)) * tma_box_rows(trunc_rows(N)) * WYI * sizeof(C) + 16);
  static constexpr bool YI_TMA = (WYI * sizeof(C)) % 16 == 0 && SM_YIT <= kSmemMax;
  // inv2 forming omega_z from u_x and u_y (two landing tiles): FP32 at 256 and
  // 512 points, where the exchange tile stays double-buffered beside them
  static constexpr size_t SM_YIW = col_smem(
      N, WYI, sizeof(C), 2 * (size_t)tma_boxes(trunc_rows(N)) * tma_box_rows(trunc_rows(N)) * WYI * sizeof(C) + 32);
  static constexpr bool YI_WZ = YI_TMA && sizeof(R) == 4 && (N == 256 || N == 512);
  // resident blocks per SM of the TMA y passes (their L2 prefetch looks one wave ahead)
  static inline int occ_yi = 1, occ_yiw = 1, occ_yf = 1;
  static_assert(!YI_WZ || SM_YIW <= kSmemMax, "inv2 with two landing tiles");
  // persistent fwd1: exchange tile + RK operand slots (3 comps x 6 per thread
  // for each operand: two for RK2/RK3, one for the other stages; the smaller
  // allocation leaves more of the SM's L1, which fwd1 is sensitive to)
  static constexpr size_t SM_F1 = col_tile_bytes(N, WH, sizeof(C)) + (size_t)36 * T * WH * sizeof(C);
  static constexpr size_t SM_F1S = col_tile_bytes(N, WH, sizeof(C)) + (size_t)18 * T * WH * sizeof(C);
  static_assert(SM_F1 <= kSmemMax, "fwd1 shared memory");
  // fwd1 with the shared spectral tile: FP32, 256 to 1024 points
  static constexpr bool F1T = sizeof(R) == 4 && (N == 256 || N == 512 || N == 1024);
  static constexpr size_t SM_X = (size_t)L * smline_len(N / 2) * sizeof(C);
  static constexpr size_t SM_XP = SM_X + (size_t)24 * (N / 16) * L * sizeof(C);  // + parked velocity fields
  // warp-per-line x pass when a line fits in one warp
  static constexpr bool XW = N / 16 <= 32;
  static constexpr int XW_WPB = 4;
  static constexpr int XW_LPW = XW ? 32 / (N / 16) : 1;
  static constexpr size_t SM_XW =
      (size_t)XW_WPB * (XW_LPW * xw_line_len<N, (XW_LPW > 1)>() + 3 * 8 * 32) * sizeof(C);
  // paired-field x pass (FP32, 128 <= N <= 1024)
  static constexpr bool XP = sizeof(R) == 4 && N >= 128 && N <= 1024;
  static constexpr int XP_G = xp_groups<N>();
  static constexpr size_t SM_XPP = (size_t)XP_G * xp_group_elems(N) * sizeof(C);

  static int run(int op, const Args &a, cudaStream_t s) {
    const Geo &g = a.g;
    const C *tw = (const C *)a.tw;
    switch (op) {
      case OP_PREPARE:
        if constexpr (XP)
          set_smem(k3_xpass_p<N, XP_G>, SM_XPP);
        else if constexpr (XW)
          set_smem(k3_xpass_w<R, N, XW_WPB>, SM_XW);
        set_smem(k3_inv1<R, N, WL, true>, SM_L);
        set_smem(k3_inv1<R, N, WL, false>, SM_L);
        set_smem(k3_inv2<R, N, WYI>, SM_YI);
        if constexpr (YI_TMA) {
          set_smem(k3_inv2_tma<R, N, WYI>, SM_YIT);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_yi, k3_inv2_tma<R, N, WYI>, T * WYI, SM_YIT);
        }
        if constexpr (YI_WZ) {
          set_smem(k3_inv2_tma<R, N, WYI, true>, SM_YIW);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_yiw, k3_inv2_tma<R, N, WYI, true>, T * WYI, SM_YIW);
        }
        set_smem(k3_fwd2<R, N, WYF>, SM_YF);
        if constexpr (YF_TMA) {
          set_smem(k3_fwd2_tma<R, N, WYF>, SM_YFT);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_yf, k3_fwd2_tma<R, N, WYF>, T * WYF, SM_YFT);
        }
        if constexpr (!XW) set_smem(k3_xpass<R, N, L>, SM_XP);
        set_smem(k_xfwd_real<R, N, L>, SM_X);
        set_smem(k_xinv_real<R, N, L>, SM_X);
        if constexpr (F1T) {
          Fwd1Pick<R, N>::prepare();
        } else {
          set_smem(k3_fwd1<R, N, WH, MODE_RK1, true>, SM_F1S);
          set_smem(k3_fwd1<R, N, WH, MODE_RK2, true>, SM_F1);
          set_smem(k3_fwd1<R, N, WH, MODE_RK3, true>, SM_F1);
          set_smem(k3_fwd1<R, N, WH, MODE_RK4, true>, SM_F1S);
          set_smem(k3_fwd1<R, N, WH, MODE_RHS, false>, SM_F1S);
          set_smem(k3_fwd1<R, N, WH, MODE_PROJ, false>, SM_F1S);
          set_smem(k3_fwd1<R, N, WH, MODE_M1, true>, SM_F1S);
          set_smem(k3_fwd1<R, N, WH, MODE_M2, true>, SM_F1S);
        }
        break;
      case OP_INV1: {
        const dim3 grid(g.c * (g.hs / WL));
        if (a.curl)
          k3_inv1<R, N, WL, true><<<grid, T * WL, SM_L, s>>>(g, (const C *)a.src, (C *)a.zb, tw, a.wz);
        else
          k3_inv1<R, N, WL, false><<<grid, T * WL, SM_L, s>>>(g, (const C *)a.src, (C *)a.zb, tw, 0);
        break;
      }
      case OP_INV2: {
        const int nz = a.nz > 0 ? a.nz : N;
        if (a.wz && a.nf == 6) {  // omega_z is formed here: only the TMA form with two landing tiles does it
          if constexpr (YI_WZ) {
            if (a.tmap_zb != nullptr && a.nf == 6) {
              k3_inv2_tma<R, N, WYI, true><<<dim3(g.hs / WYI, nz), T * WYI, SM_YIW, s>>>(
                  g, a.nf, a.z0, *reinterpret_cast<const CUtensorMap *>(a.tmap_zb), (C *)a.yb, tw, a.err,
                  wave_pf(a.nsm, occ_yiw, 4));
              break;
            }
          }
          return -1;
        }
        if constexpr (YI_TMA) {
          if (a.tmap_zb != nullptr) {
            k3_inv2_tma<R, N, WYI><<<dim3(g.hs / WYI, nz), T * WYI, SM_YIT, s>>>(
                g, a.nf, a.z0, *reinterpret_cast<const CUtensorMap *>(a.tmap_zb), (C *)a.yb, tw, a.err,
                wave_pf(a.nsm, occ_yi, a.nf > 4 ? 4 : a.nf - 1));
            break;
          }
        }
        k3_inv2<R, N, WYI><<<dim3(g.hs / WYI, nz), T * WYI, SM_YI, s>>>(g, a.nf, a.z0, (const C *)a.zb, (C *)a.yb, tw);
        break;
      }
      case OP_XPASS:
        if constexpr (XP) {
          const long long lines = (long long)(a.nz > 0 ? a.nz : N) * N;
          k3_xpass_p<N, XP_G><<<(unsigned)(lines / (2 * XP_G)), (N / 8) * XP_G, SM_XPP, s>>>(
              g, (long long)a.z0 * N, (float2 *)a.yb, (const float2 *)tw, a.umax);
        } else if constexpr (XW) {
          const long long lines = (long long)(a.nz > 0 ? a.nz : N) * N;
          k3_xpass_w<R, N, XW_WPB><<<(unsigned)(lines / (XW_WPB * XW_LPW)), 32 * XW_WPB, SM_XW, s>>>(
              g, (long long)a.z0 * N, (C *)a.yb, tw, a.umax);
        } else {
          const long long lines = (long long)(a.nz > 0 ? a.nz : N) * N;
          k3_xpass<R, N, L><<<(unsigned)(lines / L), (N / 16) * L, SM_XP, s>>>(g, (long long)a.z0 * N, (C *)a.yb, tw,
                                                                                a.umax);
        }
        break;
      case OP_FWD2: {
        const int nz = a.nz > 0 ? a.nz : N;
        if constexpr (YF_TMA) {
          if (a.tmap_yb != nullptr) {
            k3_fwd2_tma<R, N, WYF><<<dim3(g.hs / WYF, nz), T * WYF, SM_YFT, s>>>(
                g, a.nf, a.z0, *reinterpret_cast<const CUtensorMap *>(a.tmap_yb), (C *)a.zb, tw, a.err,
                wave_pf(a.nsm, occ_yf, a.nf > 2 ? 2 : a.nf - 1));
            break;
          }
        }
        k3_fwd2<R, N, WYF><<<dim3(g.hs / WYF, nz), T * WYF, SM_YF, s>>>(g, a.nf, a.z0, (const C *)a.yb, (C *)a.zb, tw);
        break;
      }
      case OP_FWD1: {
        const StepBufs<R> b = step_bufs<R>(a);
        if constexpr (F1T) {
          Fwd1Pick<R, N>::launch(a.mode, a.nsm, g, b, s);
        } else {
          // persistent: one wave of resident blocks (the kernel walks the tiles)
          const int tiles = g.c * (g.hs / WH);
          static int per_sm = 0;
          if (per_sm == 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_fwd1<R, N, WH, MODE_RK2, true>, T * WH, SM_F1);
            if (per_sm < 1) per_sm = 1;
          }
          const int grid = cmin(tiles, per_sm * (a.nsm > 0 ? a.nsm : 1));
          switch (a.mode) {
            case MODE_RK1: k3_fwd1<R, N, WH, MODE_RK1, true><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
            case MODE_RK2: k3_fwd1<R, N, WH, MODE_RK2, true><<<grid, T * WH, SM_F1, s>>>(g, b); break;
            case MODE_RK3: k3_fwd1<R, N, WH, MODE_RK3, true><<<grid, T * WH, SM_F1, s>>>(g, b); break;
            case MODE_RK4: k3_fwd1<R, N, WH, MODE_RK4, true><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
            case MODE_RHS: k3_fwd1<R, N, WH, MODE_RHS, false><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
            case MODE_M1: k3_fwd1<R, N, WH, MODE_M1, true><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
            case MODE_M2: k3_fwd1<R, N, WH, MODE_M2, true><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
            default: k3_fwd1<R, N, WH, MODE_PROJ, false><<<grid, T * WH, SM_F1S, s>>>(g, b); break;
          }
        }
        break;
      }
      case OP_XFWD_REAL:
        k_xfwd_real<R, N, L><<<(unsigned)((long long)N * N / L), (N / 16) * L, SM_X, s>>>(
            g, a.phys_in, (C *)a.yb + a.field * g.yb_f, tw);
        break;
      case OP_XINV_REAL:
        k_xinv_real<R, N, L><<<(unsigned)((long long)N * N / L), (N / 16) * L, SM_X, s>>>(
            g, (const C *)a.yb + a.field * g.yb_f, a.phys_out, tw);
        break;
      default:
        return -1;
    }
    return (int)cudaGetLastError();
  }
};

template <typename R, int N>
struct Launch2 {
  using C = typename CplxOf<R>::T;
  static constexpr int T = N / 8;
  static constexpr int WL = w_light<R, N>();
  static constexpr int WH = w_heavy<R, N>();
  static constexpr int L = x_lines<R, N>();
  static constexpr size_t SM_L = col_smem(N, WL, sizeof(C), 0);
  static constexpr size_t SM_H = col_smem(N, WH, sizeof(C), 0);
  static constexpr size_t SM_X = (size_t)L * smline_len(N / 2) * sizeof(C);
  static constexpr size_t SM_XP = SM_X + (size_t)24 * (N / 16) * L * sizeof(C);  // + parked velocity fields
  static constexpr int XW_WPB = 4;
  static constexpr int XW_LPW = N / 16 <= 32 ? 32 / (N / 16) : 1;
  // warp-per-line x pass when a line fits in one warp and there are enough lines
  static constexpr bool XW2 = N / 16 <= 32 && N >= 64 && N % (XW_WPB * XW_LPW) == 0;
  static constexpr size_t SM_XW = (size_t)XW_WPB * XW_LPW * xw_line_len<N, (XW_LPW > 1)>() * sizeof(C);

  static int run(int op, const Args &a, cudaStream_t s) {
    const Geo &g = a.g;
    const C *tw = (const C *)a.tw;
    switch (op) {
      case OP_PREPARE:
        if constexpr (XW2) set_smem(k2_xpass_w<R, N, XW_WPB>, SM_XW);
        set_smem(k2_inv1<R, N, WL, true>, SM_L);
        set_smem(k2_inv1<R, N, WL, false>, SM_L);
        set_smem(k2_xpass<R, N, L>, SM_X);
        set_smem(k_xfwd_real<R, N, L>, SM_X);
        set_smem(k_xinv_real<R, N, L>, SM_X);
        set_smem(k2_fwd1<R, N, WH, MODE_RK1, true>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_RK2, true>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_RK3, true>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_RK4, true>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_RHS, false>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_PROJ, false>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_M1, true>, SM_H);
        set_smem(k2_fwd1<R, N, WH, MODE_M2, true>, SM_H);
        break;
      case OP_INV1:
        if (a.curl)
          k2_inv1<R, N, WL, true><<<g.hs / WL, T * WL, SM_L, s>>>(g, (const C *)a.src, (C *)a.yb, tw);
        else
          k2_inv1<R, N, WL, false><<<g.hs / WL, T * WL, SM_L, s>>>(g, (const C *)a.src, (C *)a.yb, tw);
        break;
      case OP_XPASS:
        if constexpr (XW2) {
          k2_xpass_w<R, N, XW_WPB><<<N / (XW_WPB * XW_LPW), 32 * XW_WPB, SM_XW, s>>>(g, (C *)a.yb, tw, a.umax);
        } else {
          k2_xpass<R, N, L><<<N / L, (N / 16) * L, SM_X, s>>>(g, (C *)a.yb, tw, a.umax);
        }
        break;
      case OP_FWD1: {
        const StepBufs<R> b = step_bufs<R>(a);
        const unsigned grid = g.hs / WH;
        switch (a.mode) {
          case MODE_RK1: k2_fwd1<R, N, WH, MODE_RK1, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_RK2: k2_fwd1<R, N, WH, MODE_RK2, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_RK3: k2_fwd1<R, N, WH, MODE_RK3, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_RK4: k2_fwd1<R, N, WH, MODE_RK4, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_RHS: k2_fwd1<R, N, WH, MODE_RHS, false><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_M1: k2_fwd1<R, N, WH, MODE_M1, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          case MODE_M2: k2_fwd1<R, N, WH, MODE_M2, true><<<grid, T * WH, SM_H, s>>>(g, b); break;
          default: k2_fwd1<R, N, WH, MODE_PROJ, false><<<grid, T * WH, SM_H, s>>>(g, b); break;
        }
        break;
      }
      case OP_XFWD_REAL:
        k_xfwd_real<R, N, L><<<N / L, (N / 16) * L, SM_X, s>>>(g, a.phys_in, (C *)a.yb + a.field * g.yb_f, tw);
        break;
      case OP_XINV_REAL:
        k_xinv_real<R, N, L><<<N / L, (N / 16) * L, SM_X, s>>>(g, (const C *)a.yb + a.field * g.yb_f,
                                                               a.phys_out, tw);
        break;
      default:
        return -1;
    }
    return (int)cudaGetLastError();
  }
};

}  // namespace nsk
