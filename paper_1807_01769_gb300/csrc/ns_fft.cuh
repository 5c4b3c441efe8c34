// ns_fft.cuh -- device-side building blocks of the pass kernels: complex
// arithmetic and a batched power-of-two FFT whose data live in registers
// (8 points per thread) and move between radix stages through shared memory.
//
// The FFT is the self-sorting (Stockham) decimation-in-time form: with
// T = L/8 threads per line, thread t holds x[t + T m], m = 0..7, before the
// first stage and X[t + T m] after the last one, so a pass kernel can load its
// inputs straight from global memory and store its outputs straight back with
// the same, coalesced, index pattern.  A stage of radix R and span Ns takes
// butterfly j from x[j + r L/R], twiddles input r by exp(+-2 pi i r (j mod Ns)
// / (Ns R)), does a length-R DFT in registers and writes output r to
// y[(j / Ns) Ns R + j mod Ns + r Ns].  L = 8^a * R0 with R0 in {1, 2, 4}; the
// small radix, if any, is the first stage (no twiddles there).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nsk {

template <typename R>
struct CplxOf;
template <>
struct CplxOf<float> {
  using T = float2;
};
template <>
struct CplxOf<double> {
  using T = double2;
};

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  return C{a.x + b.x, a.y + b.y};
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  return C{a.x - b.x, a.y - b.y};
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C>
__device__ __forceinline__ C cconj(C a) {
  return C{a.x, -a.y};
}
template <typename C, typename R>
__device__ __forceinline__ C cscale(C a, R s) {
  return C{a.x * s, a.y * s};
}
// i * a
template <typename C>
__device__ __forceinline__ C cmuli(C a) {
  return C{-a.y, a.x};
}
// (DIR i) * a, DIR = +1 or -1
template <int DIR, typename C>
__device__ __forceinline__ C cmul_diri(C a) {
  return DIR > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <typename C>
__device__ __forceinline__ C czero() {
  return C{0, 0};
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// ------------------------------------------------------------ small DFTs --
// X_s = sum_r a_r exp(DIR 2 pi i r s / R), natural order in and out.
template <int DIR, typename C>
__device__ __forceinline__ void dft2(C &a0, C &a1) {
  const C t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int DIR, typename C>
__device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3) {
  const C t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const C t2 = cadd(a1, a3), t3 = cmul_diri<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int DIR, typename C>
__device__ __forceinline__ void dft8(C (&a)[8]) {
  using R = decltype(a[0].x);
  const R h = (R)0.70710678118654752440084436210484903928;  // 1/sqrt(2)
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  // o_k *= w^k, w = exp(DIR 2 pi i / 8) = (1 + DIR i)/sqrt(2)
  o1 = C{h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x)};
  o2 = cmul_diri<DIR>(o2);
  o3 = C{h * (-o3.x - DIR * o3.y), h * (-o3.y + DIR * o3.x)};
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1);
  a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3);
  a[7] = csub(e3, o3);
}

template <int R, int DIR, typename C>
__device__ __forceinline__ void dftR(C (&a)[R]);
template <>
__device__ __forceinline__ void dftR<2, -1, float2>(float2 (&a)[2]) { dft2<-1>(a[0], a[1]); }
template <>
__device__ __forceinline__ void dftR<2, 1, float2>(float2 (&a)[2]) { dft2<1>(a[0], a[1]); }
template <>
__device__ __forceinline__ void dftR<2, -1, double2>(double2 (&a)[2]) { dft2<-1>(a[0], a[1]); }
template <>
__device__ __forceinline__ void dftR<2, 1, double2>(double2 (&a)[2]) { dft2<1>(a[0], a[1]); }
template <>
__device__ __forceinline__ void dftR<4, -1, float2>(float2 (&a)[4]) { dft4<-1>(a[0], a[1], a[2], a[3]); }
template <>
__device__ __forceinline__ void dftR<4, 1, float2>(float2 (&a)[4]) { dft4<1>(a[0], a[1], a[2], a[3]); }
template <>
__device__ __forceinline__ void dftR<4, -1, double2>(double2 (&a)[4]) { dft4<-1>(a[0], a[1], a[2], a[3]); }
template <>
__device__ __forceinline__ void dftR<4, 1, double2>(double2 (&a)[4]) { dft4<1>(a[0], a[1], a[2], a[3]); }
template <>
__device__ __forceinline__ void dftR<8, -1, float2>(float2 (&a)[8]) { dft8<-1>(a); }
template <>
__device__ __forceinline__ void dftR<8, 1, float2>(float2 (&a)[8]) { dft8<1>(a); }
template <>
__device__ __forceinline__ void dftR<8, -1, double2>(double2 (&a)[8]) { dft8<-1>(a); }
template <>
__device__ __forceinline__ void dftR<8, 1, double2>(double2 (&a)[8]) { dft8<1>(a); }

// Table entry j of a table holding exp(-2 pi i (...)), conjugated for DIR = +1.
template <int DIR, typename C>
__device__ __forceinline__ C twiddle(const C *__restrict__ tw, int j) {
  const C w = __ldg(tw + j);
  return DIR < 0 ? w : cconj(w);
}

// Radix and span of stage s of a length-L transform (host and device).
__host__ __device__ constexpr int plan_r0(int L) { return 1 << (ilog2(L) % 3); }
__host__ __device__ constexpr int plan_nst(int L) { return ilog2(L) / 3 + (plan_r0(L) > 1 ? 1 : 0); }
__host__ __device__ constexpr int plan_radix(int L, int s) { return (s == 0 && plan_r0(L) > 1) ? plan_r0(L) : 8; }
__host__ __device__ constexpr int plan_span(int L, int s) {
  return s == 0 ? 1 : (plan_r0(L) > 1 ? plan_r0(L) * (1 << (3 * (s - 1))) : (1 << (3 * s)));
}
// Stage twiddle table of a length-L transform: for every stage s >= 1 a block
// of (R_s - 1) NS_s entries, entry (r - 1) NS_s + j = exp(-2 pi i r j / (NS_s R_s)),
// so the twiddles of consecutive butterflies j are consecutive in memory (the
// transform reads the r = 1 row and forms the other powers by products).
__host__ __device__ constexpr int stage_tw_offset(int L, int s) {
  return s <= 1 ? 0 : stage_tw_offset(L, s - 1) + (plan_radix(L, s - 1) - 1) * plan_span(L, s - 1);
}
__host__ __device__ constexpr int stage_tw_len(int L) { return stage_tw_offset(L, plan_nst(L)); }

// Shared-memory views used for the exchanges between stages.  ld<X>/st<X>
// address the exchange that follows stage X.  With DB (double buffer) the
// exchanges alternate between two buffers bofs elements apart, so a thread
// may write the next exchange while others still read the previous one: a
// transform then needs one barrier per exchange instead of two.
//   column tile [n][pitch], this thread's column at base
template <typename C, bool DBUF = false>
struct SmCol {
  static constexpr bool DB = DBUF;
  C *base;
  int pitch;
  int bofs;
  template <int X>
  __device__ __forceinline__ C ld(int n) const {
    return base[(DB && (X & 1) ? bofs : 0) + n * pitch];
  }
  template <int X>
  __device__ __forceinline__ void st(int n, C v) const {
    base[(DB && (X & 1) ? bofs : 0) + n * pitch] = v;
  }
};
//   contiguous line of a length-L transform with one pad slot every 8 entries,
//   or every 16 after a radix-2/4 first stage (its stride-2/4 writes are then
//   free of bank conflicts; the stride-8 writes of radix-8 stages and the
//   grouped writes of later stages need the 1-in-8 padding)
template <typename C, int L = 0, bool DBUF = false>
struct SmLine {
  static constexpr bool DB = DBUF;
  C *base;
  int bofs;
  template <int X>
  static __device__ __forceinline__ int pad(int n) {
    return (X == 0 && L > 0 && plan_r0(L) != 1) ? n + (n >> 4) : n + (n >> 3);
  }
  template <int X>
  __device__ __forceinline__ C ld(int n) const {
    return base[(DB && (X & 1) ? bofs : 0) + pad<X>(n)];
  }
  template <int X>
  __device__ __forceinline__ void st(int n, C v) const {
    base[(DB && (X & 1) ? bofs : 0) + pad<X>(n)] = v;
  }
};
__host__ __device__ constexpr int smline_len(int L) { return L + L / 8; }
//   contiguous line of a length-512 transform held by 64 threads, unpadded
//   and XOR-swizzled within rows of 16 entries: entry n lives at
//   16 a + ((n mod 16) xor phi(a)), a = n / 16, phi(a) = (a & 7) | ((a & 4) << 1).
//   Every half-warp access of the plan (contiguous loads, the stride-8 stores
//   of stage 0, the grouped stores of stage 1) then touches 16 distinct
//   8-byte bank pairs, where the 1-in-8 padding costs the contiguous loads an
//   extra wavefront.
template <typename C, bool DBUF = false>
struct SmLineX {
  static constexpr bool DB = DBUF;
  C *base;
  int bofs;
  static __device__ __forceinline__ int swz(int n) {
    const int a = n >> 4;
    return (n & ~15) | ((n & 15) ^ ((a & 7) | ((a & 4) << 1)));
  }
  template <int X>
  __device__ __forceinline__ C ld(int n) const {
    return base[(DB && (X & 1) ? bofs : 0) + swz(n)];
  }
  template <int X>
  __device__ __forceinline__ void st(int n, C v) const {
    base[(DB && (X & 1) ? bofs : 0) + swz(n)] = v;
  }
};

// One radix-R stage of span NS on a line of length L (see file header).
template <int L, int R, int NS, int TWOFF, int DIR, bool LAST, int XS, typename C, typename SM>
__device__ __forceinline__ void fft_stage(C (&v)[8], int t, const C *__restrict__ stw, const SM &sm) {
  constexpr int T = L / 8;
  constexpr int Q = 8 / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = t + T * q;
    C a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = v[q + r * Q];
    if (NS > 1) {
      // w^r from one table load, by a product tree of depth <= 3
      C wp[8];
      wp[1] = twiddle<DIR>(stw + TWOFF, b % NS);
      if (R > 2) wp[2] = cmul(wp[1], wp[1]);
      if (R > 3) wp[3] = cmul(wp[2], wp[1]);
      if (R > 4) {
        wp[4] = cmul(wp[2], wp[2]);
        wp[5] = cmul(wp[4], wp[1]);
        wp[6] = cmul(wp[4], wp[2]);
        wp[7] = cmul(wp[4], wp[3]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) a[r] = cmul(a[r], wp[r]);
    }
    dftR<R, DIR>(a);
    if (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + r * Q] = a[r];
    } else {
      const int base = (b / NS) * NS * R + (b % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) sm.template st<XS>(base + r * NS, a[r]);
    }
  }
}

template <int L, int S>
struct StagePlan {
  static constexpr int LOG = ilog2(L);
  static constexpr int R0 = plan_r0(L);
  static constexpr int NST = plan_nst(L);
  static constexpr int RADIX = plan_radix(L, S);
  static constexpr int NS = plan_span(L, S);  // span before stage S
  static constexpr int TWOFF = stage_tw_offset(L, S);
};

// Synchronisation scope of the exchanges: a whole block, one warp when every
// line exchanged lives inside that warp, or (SY >= 64, a multiple of 32) the
// group of SY consecutive threads that owns the line, through the named
// barrier 1 + threadIdx.x / SY (barrier 0 is the block's; at most 15 groups).
enum SyncScope { SYNC_BLOCK = 0, SYNC_WARP = 1 };
template <int SY>
__device__ __forceinline__ void fft_sync() {
  if constexpr (SY == SYNC_WARP) {
    __syncwarp();
  } else if constexpr (SY >= 64) {
    static_assert(SY % 32 == 0, "named-barrier groups are whole warps");
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + (int)threadIdx.x / SY), "n"(SY) : "memory");
  } else {
    __syncthreads();
  }
}

template <int L, int S, int DIR, int SY, typename C, typename SM>
struct FftRun {
  __device__ __forceinline__ static void run(C (&v)[8], int t, const C *__restrict__ stw, const SM &sm) {
    using P = StagePlan<L, S>;
    constexpr int T = L / 8;
    if (S > 0) {
      fft_sync<SY>();  // the previous stage's shared writes are visible
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = sm.template ld<S - 1>(t + T * m);
      // single buffer: everyone read before the next writes
      if (!SM::DB && S < P::NST - 1) fft_sync<SY>();
    }
    fft_stage<L, P::RADIX, P::NS, P::TWOFF, DIR, S == P::NST - 1, S>(v, t, stw, sm);
    FftRun<L, S + 1, DIR, SY, C, SM>::next(v, t, stw, sm);
  }
  __device__ __forceinline__ static void next(C (&v)[8], int t, const C *__restrict__ stw, const SM &sm) {
    if constexpr (S < StagePlan<L, 0>::NST) FftRun<L, S, DIR, SY, C, SM>::run(v, t, stw, sm);
  }
};

// Length-L FFT of one line held as v[m] = x[t + T m] (T = L/8) by threads
// t = 0..T-1.  Every thread of the sync scope (the block, or the warp for
// SYNC_WARP) must call it; sm is this thread's view of a scratch line of at
// least L entries (two, bofs apart, for a double-buffered view).  On return
// v[m] = X[t + T m], X_k = sum_j x_j exp(DIR 2 pi i j k / L).  stw is the
// stage twiddle table of length L (stage_tw_len(L) entries, see
// stage_tw_offset).  The leading barrier protects the scratch from the
// previous transform's last reads; a double-buffered view whose last exchange
// uses the second buffer does not need it.
template <int L, int DIR, typename C, typename SM, int SY = SYNC_BLOCK>
__device__ __forceinline__ void fft_line(C (&v)[8], int t, const C *__restrict__ stw, const SM &sm) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "power of two >= 8");
  constexpr int NST = StagePlan<L, 0>::NST;
  if (NST > 1 && !(SM::DB && ((NST - 2) & 1))) fft_sync<SY>();
  FftRun<L, 0, DIR, SY, C, SM>::run(v, t, stw, sm);
}

}  // namespace nsk
