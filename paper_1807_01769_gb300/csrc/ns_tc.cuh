// ns_tc.cuh -- the 3D x pass on the fifth-generation tensor cores (tcgen05),
// used by precision NS_FP32_TC: same state, tables and other passes as
// NS_FP32; only the x-line transforms and the product run here.
//
// Fields are paired into complex lines, z = x_a + i x_b: the six inverse
// fields as (u_x, u_y), (u_z, w_x), (w_y, w_z), with u_z scaled per line by
// a power of two to the size of w_x; the forward fields as (n_x, n_y) of one
// line and n_z of two neighbouring lines.  Every transform
// is then one complex DFT of length N = R1 R2, written as two GEMMs.  With
// n = R2 a + b, k = c + R1 d and w = exp(2 pi i / N):
//   stage A   Y[b][c]     = sum_a x[R2 a + b] w^(R2 a c)          (DFT-R1 over a)
//   twiddle   Y'[b][c]    = w^(b c) Y[b][c]
//   stage B   X[c + R1 d] = sum_b Y'[b][c] w^(R1 b d)             (DFT-R2 over b)
// In real-block form a length-R DFT is a 2R x 2R real matrix [[C, S], [-S, C]]
// (rows: real then imaginary input parts); stage A multiplies the rows
// (line, b) of 2 R1 reals by it, stage B the rows (line, c) of 2 R2 reals.
// Operands are split into BF16 pairs, x = hi + lo (both rounded to nearest),
// the DFT matrices from their FP64 values; three MMAs (hi*hi, hi*lo, lo*hi)
// accumulate in FP32 in tensor memory, leaving about 2^-16 relative error per
// product (the dropped lo*lo term and the rounding of lo).  The forward
// transform reuses the inverse matrices on conjugated input:
// DFT_-(z) = conj(DFT_+(conj z)).
//
// A block (256 threads, two per tensor-memory lane, each taking half of its
// row's values) owns L = 128 / R1 lines per tile.  Stage-A operands are K-major (thread = row, each writes its own
// 16-byte row segments), stage-B operands MN-major (the thread holding row
// (line, b) of stage A writes column b of the rows (line, c)), so no register
// transposes are needed.  The spectral rows of each inverse pair arrive by
// TMA in a landing tile, one pair ahead of the one being transformed.  The
// three inverse results stay in tensor memory while the product is formed;
// one thread issues the MMAs and commits them to an mbarrier that the block
// waits on with a bounded poll.
#pragma once
#include <cuda_bf16.h>

#include "ns_kernels.cuh"

namespace nsk {
namespace tc {

// ------------------------------------------------------------ primitives --
// Shared-memory matrix descriptor, no swizzle: start address, leading
// dimension byte offset (between core matrices along K), stride dimension byte
// offset (between core matrices along M or N), descriptor version 1 (bit 46).
// A core matrix is 8 rows of 16 bytes stored contiguously.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), A MN-major when a_mn (bit 15), B K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int Nn, bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((unsigned)(Nn >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                    unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on bar once every MMA this thread issued before has completed
__device__ __forceinline__ void commit(unsigned long long *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// one warp: allocate ncols tensor-memory columns (a power of two >= 32), base address into *slot
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// this warp's 32 lanes, X consecutive 32-bit columns from taddr (warp-collective)
__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8]) {
  unsigned r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(unsigned taddr, float (&v)[4]) {
  unsigned r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
template <int X>
__device__ __forceinline__ void tmem_ld(unsigned taddr, float (&v)[X]) {
  static_assert(X % 4 == 0, "multiples of 4 columns");
#pragma unroll
  for (int i = 0; i < X / 8; ++i) {
    float t[8];
    tmem_ld8(taddr + 8 * i, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[8 * i + j] = t[j];
  }
  if constexpr (X % 8 != 0) {
    float t[4];
    tmem_ld4(taddr + X - 4, t);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[X - 4 + j] = t[j];
  }
}
// bounded wait for the completion of the mbarrier phase with parity ph
__device__ __forceinline__ bool wait_phase(unsigned long long *bar, unsigned ph) {
  for (long long i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, ph)) return true;
  return false;
}
// x0 = h0 + l0, x1 = h1 + l1 with BF16 h, l rounded to nearest; packed pairs
__device__ __forceinline__ void split2(float x0, float x1, unsigned &hi, unsigned &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  hi = *reinterpret_cast<const unsigned *>(&h);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - h0, x1 - h1);
  lo = *reinterpret_cast<const unsigned *>(&l);
}
// 8 consecutive K (or M) elements: one 16-byte segment of hi and one of lo
__device__ __forceinline__ void put8(unsigned char *hi, unsigned char *lo, const float *x) {
  uint4 h, l;
  split2(x[0], x[1], h.x, l.x);
  split2(x[2], x[3], h.y, l.y);
  split2(x[4], x[5], h.z, l.z);
  split2(x[6], x[7], h.w, l.w);
  *reinterpret_cast<uint4 *>(hi) = h;
  *reinterpret_cast<uint4 *>(lo) = l;
}
__device__ __forceinline__ void put4(unsigned char *hi, unsigned char *lo, float x0, float x1, float x2, float x3) {
  uint2 h, l;
  split2(x0, x1, h.x, l.x);
  split2(x2, x3, h.y, l.y);
  *reinterpret_cast<uint2 *>(hi) = h;
  *reinterpret_cast<uint2 *>(lo) = l;
}

// ------------------------------------------------------------------ plan --
template <int N>
struct Plan;
template <>
struct Plan<64> {
  static constexpr int R1 = 8, R2 = 8;
};
template <>
struct Plan<128> {
  static constexpr int R1 = 8, R2 = 16;
};
template <>
struct Plan<256> {
  static constexpr int R1 = 16, R2 = 16;
};
template <>
struct Plan<512> {
  static constexpr int R1 = 16, R2 = 32;
};

// Shared-memory map (bytes) and tensor-memory columns of the kernel for N.
//  OPA : MT stage-A tiles, each a hi and a lo K-major [128][KA] BF16 matrix;
//        core (r/8, k/8) at (r/8) KA*16 + (k/8) 128, row r % 8 at 16 (r % 8)
//  OPB : stage-B operand, hi and lo MN-major [K = KB][M = 128]; core
//        (m/8, k/8) at (k/8) 2048 + (m/8) 128, row k % 8 at 16 (k % 8); it
//        also holds the stage-A tile of the forward n_z pairs (laid out as an
//        OPA tile), which is consumed before the next stage-B operand is built;
//        OPA, free by then, takes the n_z pairs' stage-B operand (same size,
//        same layout) so that both forward stage-B GEMMs run together
//  FA, FB : real-block DFT-R1 / DFT-R2 matrices (+ sign), hi and lo,
//        K-major [n][k] like OPA
//  LAND : TMA landing tile of one inverse pair: [2 fields][L lines][HS]
//        complex64 (HS = the padded row length of the spectral buffers)
//  TW   : the twiddles w^(b c) = exp(+2 pi i b c / N) as [c][b] complex64
//        (the lanes of a warp hold consecutive b)
// Tensor memory: GA = stage-A results (MT tiles x KA columns), T1..T3 = the
// three inverse pair results (KB columns each; T1, T2 then take the forward
// stage-B results and T3 the forward n_z stage-A result).
template <int N>
struct Geom {
  static constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
  static constexpr int L = 128 / R1, MT = R2 / R1, KA = 2 * R1, KB = 2 * R2;
  static constexpr int KC = (N - 1) / 3;
  static constexpr int HS = (KC + 1 + 15) / 16 * 16;  // complex64 rows padded to 128 bytes
  static constexpr unsigned TILE_A = 128u * KA * 2;
  static constexpr unsigned OPA = 0, OPA_BYTES = MT * 2 * TILE_A;
  static constexpr unsigned OPB = OPA + OPA_BYTES, OPB_HALF = 128u * KB * 2;
  static constexpr unsigned FA = OPB + 2 * OPB_HALF, FA_HALF = (unsigned)KA * KA * 2;
  static constexpr unsigned FB = FA + 2 * FA_HALF, FB_HALF = (unsigned)KB * KB * 2;
  static constexpr unsigned MATS_BYTES = 2 * FA_HALF + 2 * FB_HALF;
  static constexpr unsigned LAND = FB + 2 * FB_HALF, LAND_FIELD = (unsigned)L * HS * 8;
  static constexpr unsigned TW = LAND + 2 * LAND_FIELD, TW_BYTES = (unsigned)R1 * R2 * 8;
  static constexpr unsigned USED = TW + (TW_BYTES + 127u) / 128u * 128u;
  static constexpr unsigned TCOLS = 4 * KB;  // a power of two: 64, 128 or 256
  static constexpr unsigned GA = 0, T1 = KB, T2 = 2 * KB, T3 = 3 * KB;
  static constexpr int CTAS = 512 / TCOLS;  // blocks per SM the tensor memory holds
  // dynamic shared memory requested: enough that no more than CTAS blocks are
  // resident on an SM (228 KB per SM, 1 KB reserved per block)
  static constexpr unsigned FLOOR = 233472u / (CTAS + 1) - 1024u + 128u;
  static constexpr unsigned SMEM = ((USED > FLOOR ? USED : FLOOR) + 127u) / 128u * 128u;
  static constexpr unsigned IDA = idesc_bf16(128, KA, false), IDB = idesc_bf16(128, KB, true);
  static_assert(KB <= 64 && MT * KA == KB, "tensor-memory map");
  static_assert(2 * TILE_A <= 2 * OPB_HALF && OPA_BYTES == 2 * OPB_HALF && LAND % 128 == 0 && HS <= 256 && L <= 256,
                "shared-memory map");
  static_assert(SMEM <= 232448, "shared memory");
};

// -------------------------------------------------------------- kernel --
// Two threads per tensor-memory lane: thread tid serves row (tid mod 128) and
// takes half h = tid / 128 of the row's values in every phase.
constexpr int kThreads = 256;

// NV (4 or 8) consecutive BF16 elements: hi at p, lo at p + lo_off
template <int NV>
__device__ __forceinline__ void put_run(unsigned char *p, unsigned lo_off, const float *x) {
  static_assert(NV == 4 || NV == 8, "runs of 8 or 16 bytes");
  if constexpr (NV == 8)
    put8(p, p + lo_off, x);
  else
    put4(p, p + lo_off, x[0], x[1], x[2], x[3]);
}
// element k of K-major row r of an operand tile at p (row stride in core matrices: kbytes16 = K * 16)
__device__ __forceinline__ unsigned char *kmajor(unsigned char *p, int r, int k, int kbytes16) {
  return p + (r >> 3) * kbytes16 + (r & 7) * 16 + (k >> 3) * 128 + (k & 7) * 2;
}

// Stage-B operand from one stage-A row (group grp = line or line pair, index
// b) whose outputs sit in this warp's lanes from tensor-memory address taddr
// (re c at column c, im at R1 + c): the half h of them, c in [h R1/2,
// (h+1) R1/2), twiddled by w^(b c) and written as column (p R2 + b) of the
// MN-major rows (grp R1 + c) of the stage-B operand at byte offset opb.
// Warp-collective (the load); `store` = the row is real.
template <int N>
__device__ __forceinline__ void stage_b_half(unsigned char *sm, unsigned opb, unsigned taddr, int grp, int b, int h,
                                             bool store) {
  using G = Geom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, CH = R1 / 2;
  float vr[CH], vi[CH];
  tmem_ld<CH>(taddr + h * CH, vr);
  tmem_ld<CH>(taddr + R1 + h * CH, vi);
  tmem_wait_ld();
  if (!store) return;
  const float2 *tws = reinterpret_cast<const float2 *>(sm + G::TW);
  float yr[CH], yi[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const float2 w = tws[(h * CH + i) * R2 + b];  // exp(+2 pi i b c / N)
    yr[i] = fmaf(vr[i], w.x, -(vi[i] * w.y));
    yi[i] = fmaf(vi[i], w.x, vr[i] * w.y);
  }
  const int m0 = grp * R1 + h * CH;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int kp = p * R2 + b;
    unsigned char *dst = sm + opb + (kp >> 3) * 2048 + (kp & 7) * 16 + (m0 >> 3) * 128 + (m0 & 7) * 2;
    put_run<CH>(dst, G::OPB_HALF, p ? yi : yr);
  }
}

// Stage-A MMAs of the operand tile at byte offset tile_off into tensor-memory
// column col; stage-B MMAs of the operand at byte offset opb into col.
// Issued by one thread.
template <int N>
__device__ __forceinline__ void issue_a(unsigned sbase, unsigned tmem, unsigned tile_off, unsigned col) {
  using G = Geom<N>;
#pragma unroll
  for (int pr = 0; pr < 3; ++pr)
#pragma unroll
    for (int q = 0; q < G::KA / 16; ++q) {
      const unsigned a = sbase + tile_off + (pr == 2 ? G::TILE_A : 0) + q * 256;
      const unsigned b = sbase + G::FA + (pr == 1 ? G::FA_HALF : 0) + q * 256;
      mma(tmem + col, sdesc(a, 128, G::KA * 16), sdesc(b, 128, G::KA * 16), G::IDA, (pr | q) != 0);
    }
}
template <int N>
__device__ __forceinline__ void issue_b(unsigned sbase, unsigned tmem, unsigned opb, unsigned col) {
  using G = Geom<N>;
#pragma unroll
  for (int pr = 0; pr < 3; ++pr)
#pragma unroll
    for (int q = 0; q < G::KB / 16; ++q) {
      const unsigned a = sbase + opb + (pr == 2 ? G::OPB_HALF : 0) + q * 4096;
      const unsigned b = sbase + G::FB + (pr == 1 ? G::FB_HALF : 0) + q * 256;
      mma(tmem + col, sdesc(a, 2048, 128), sdesc(b, 128, G::KB * 16), G::IDB, (pr | q) != 0);
    }
}

// Forward stage-B result of row (grp, c) in this warp's lanes from taddr:
// G[k] = conj of the forward DFT of the pair z = y_a + i y_b, k = c + R1 d.
// Writes Y_b (second = true) or Y_a for k = c + R1 d <= KC to out[k]; the
// partner G[N - k] comes from lane (grp, (R1 - c) mod R1).  Warp-collective.
template <int N>
__device__ __forceinline__ void split_store(unsigned taddr, int c, int lane, bool second, bool store,
                                            float2 *__restrict__ out) {
  using G = Geom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, DM = G::KC / R1 + 1;
  float v[G::KB];
  tmem_ld<G::KB>(taddr, v);
  tmem_wait_ld();
  const int src = (lane & ~(R1 - 1)) | ((R1 - c) & (R1 - 1));
#pragma unroll
  for (int d = 0; d < DM; ++d) {
    // the partner of (c, d) is (R1 - c, R2 - 1 - d), or (0, (R2 - d) mod R2) for c = 0
    const int i0 = (R2 - d) % R2, i1 = R2 - 1 - d;
    const float sr = c == 0 ? v[i0] : v[i1], si = c == 0 ? v[R2 + i0] : v[R2 + i1];
    const float hr = __shfl_sync(0xffffffffu, sr, src), hi = __shfl_sync(0xffffffffu, si, src);
    const float gr = v[d], gi = v[R2 + d];
    // Z = conj G: Y_a = (Z[k] + conj Z[N-k]) / 2, Y_b = (Z[k] - conj Z[N-k]) / (2 i)
    const float2 y = second ? make_float2(-0.5f * (gi + hi), 0.5f * (hr - gr))
                            : make_float2(0.5f * (gr + hr), 0.5f * (hi - gi));
    if (store && c + R1 * d <= G::KC) out[c + R1 * d] = y;
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 2)
    k3_xpass_tc(Geo g, long long line_base, long long tiles, float2 *__restrict__ yb, const float2 *__restrict__ tw,
                const uint4 *__restrict__ mats, const __grid_constant__ CUtensorMap tm,
                unsigned long long *__restrict__ umax, int *__restrict__ err) {
  using G = Geom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, L = G::L, MT = G::MT, KA = G::KA, KC = G::KC;
  constexpr int CH = R1 / 2;                        // a (or c) values per half row
  constexpr int CHK = R2 / 8 >= 2 ? 8 : 4;          // points per product chunk
  constexpr int NCH = R2 / CHK;                     // chunks per row (even: split by half)
  static_assert(NCH % 2 == 0, "product chunks split between the halves");
  unsigned char *sm = dyn_smem<unsigned char>();
  __shared__ __align__(8) unsigned long long bars[3];  // stage A done, stage B done, tile landed
  __shared__ unsigned tslot;
  __shared__ float lscale[128];  // 1 / (scale of u_z) per line of the tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & 127, h = tid >> 7;
  const unsigned sbase = smem_addr(sm);
  const long long fs = g.yb_f, hs = g.hs;

  for (unsigned i = tid; i < G::MATS_BYTES / 16; i += kThreads)
    reinterpret_cast<uint4 *>(sm + G::FA)[i] = __ldg(mats + i);
  for (unsigned i = tid; i < G::TW_BYTES / 8; i += kThreads) {
    const float2 w = __ldg(tw + (i / R2) * (i % R2));  // exp(-2 pi i b c / N), b c < N: store the conjugate
    reinterpret_cast<float2 *>(sm + G::TW)[i] = make_float2(w.x, -w.y);
  }
  if (warp == 0) tmem_alloc(&tslot, G::TCOLS);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem = tslot;
  const unsigned tlane = tmem + ((unsigned)((warp & 3) * 32) << 16);  // this warp's lanes
  unsigned pha = 0, phb = 0, pht = 0;
  bool bad = false, tma_pending = false, failed = false;
  // a commit to bars[0] / bars[1] whose completion this thread has not seen,
  // and the parity of the phase that completes it (drained before the
  // tensor memory is freed on the failure path)
  bool pend_a = false, pend_b = false;
  unsigned par_a = 0, par_b = 0;
  const float2 *land = reinterpret_cast<const float2 *>(sm + G::LAND);
  const long long nn = (long long)N * N;  // lines per field
  // one thread: the spectral rows of fields f, f + 1 of the tile's lines into LAND
  auto fetch = [&](int f, long long first_line) {
    mbar_expect_tx(&bars[2], 2 * G::LAND_FIELD);
    for (int i = 0; i < 2; ++i)
      tma_load_2d(sm + G::LAND + i * G::LAND_FIELD, &tm, 0, (int)((f + i) * nn + first_line), &bars[2]);
  };
  if (tid == 0 && (long long)blockIdx.x < tiles) fetch(0, line_base + (long long)blockIdx.x * L);
  tma_pending = (long long)blockIdx.x < tiles;
  // stage A done -> its results; stage B done -> its results or a free operand
  auto wait_a = [&]() {
    const bool ok = wait_phase(&bars[0], pha);
    bad |= !ok;
    pend_a = pend_a && !ok;
    pha ^= 1u;
    fence_after();
  };
  auto wait_b = [&]() {
    const bool ok = wait_phase(&bars[1], phb);
    bad |= !ok;
    pend_b = pend_b && !ok;
    phb ^= 1u;
    fence_after();
  };
  // every thread notes each commit (the issuing thread is thread 0)
  auto note_a = [&]() {
    pend_a = true;
    par_a = pha;
  };
  auto note_b = [&]() {
    pend_b = true;
    par_b = phb;
  };
  auto wait_t = [&]() {
    bad |= !wait_phase(&bars[2], pht);
    pht ^= 1u;
    tma_pending = false;
  };
  // operands written and tensor-memory reads finished by every thread; false: give up
  auto publish = [&]() {
    fence_async_smem();
    fence_before();
    return !__syncthreads_or(bad);
  };
#define NS_TC_PUBLISH_OR_LEAVE \
  if (!publish()) {            \
    failed = true;             \
    goto out;                  \
  }

  const int line = row / R1, c = row % R1;  // this thread's stage-B row
  float umx = 0.f, umy = 0.f, umz = 0.f;

  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long line0 = line_base + tile * L;
    // ---------------------------------------------- inverse: three pairs --
    for (int pp = 0; pp < 3; ++pp) {
      wait_t();  // fields 2 pp, 2 pp + 1 of this tile's lines are in LAND
      // the pair (u_z, w_x) mixes fields of different size (|w| ~ |k| |u|),
      // and a transform's rounding scales with the larger of its two fields:
      // u_z of a line enters scaled by s = 2^e, the power of two that brings
      // the line's largest |u_z| near its largest |w_x| (exact both ways),
      // and the product divides it out.  The R2 lanes that build a line's
      // rows reduce its maxima together (both thread halves alike), so no
      // block barrier is needed.
      float sa[MT];
#pragma unroll
      for (int j = 0; j < MT; ++j) {
        sa[j] = 1.f;
        if (pp == 1) {
          const int ra = row + 128 * j, ln = ra / R2, gl = lane % R2;
          const float2 *pa = land + ln * G::HS, *pb = pa + L * G::HS;
          float ma = 0.f, mb = 0.f;
          for (int k = gl; k <= KC; k += R2) {
            const float2 xa = pa[k], xb = pb[k];
            ma = fmaxf(ma, fmaxf(fabsf(xa.x), fabsf(xa.y)));
            mb = fmaxf(mb, fmaxf(fabsf(xb.x), fabsf(xb.y)));
          }
#pragma unroll
          for (int off = R2 / 2; off > 0; off >>= 1) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, off, R2));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, off, R2));
          }
          float inv = 1.f;
          if (ma > 0.f && mb > 0.f) {
            int ea, eb;
            frexpf(ma, &ea);
            frexpf(mb, &eb);
            const int e = max(-64, min(64, eb - ea));
            sa[j] = ldexpf(1.f, e);
            inv = ldexpf(1.f, -e);
          }
          if (h == 0 && gl == 0) lscale[ln] = inv;  // read by the product after the next barriers
        }
      }
#pragma unroll
      for (int j = 0; j < MT; ++j) {
        const int ra = row + 128 * j, ln = ra / R2, b = ra % R2;
        const float2 *pa = land + ln * G::HS, *pb = pa + L * G::HS;
        float zr[CH], zi[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) {
          const int k = R2 * (h * CH + i) + b;
          const bool lo = k <= KC, hi = k >= N - KC;
          float2 xa = make_float2(0.f, 0.f), xb = xa;
          if (lo || hi) {
            const int idx = lo ? k : N - k;
            xa = pa[idx];
            xb = pb[idx];
          }
          if (k == 0) xa.y = xb.y = 0.f;  // the self-conjugate mode is real
          if (pp == 1) {
            xa.x *= sa[j];
            xa.y *= sa[j];
          }
          // k <= kc: z = xa + i xb;  k >= N - kc: z = conj(xa) + i conj(xb)
          zr[i] = lo ? xa.x - xb.y : xa.x + xb.y;
          zi[i] = lo ? xa.y + xb.x : xb.x - xa.y;
        }
        unsigned char *tile_p = sm + G::OPA + j * 2 * G::TILE_A;
        put_run<CH>(kmajor(tile_p, row, h * CH, KA * 16), G::TILE_A, zr);
        put_run<CH>(kmajor(tile_p, row, R1 + h * CH, KA * 16), G::TILE_A, zi);
      }
      NS_TC_PUBLISH_OR_LEAVE
      // LAND is free: the next pair of this tile, or the first pair of the next tile
      {
        const bool more = pp < 2 || tile + gridDim.x < tiles;
        if (tid == 0) {
          fence_after();
          for (int t = 0; t < MT; ++t) issue_a<N>(sbase, tmem, G::OPA + t * 2 * G::TILE_A, G::GA + t * KA);
          commit(&bars[0]);
          if (more) {
            fence_proxy_async_smem();
            if (pp < 2)
              fetch(2 * pp + 2, line0);
            else
              fetch(0, line0 + (long long)gridDim.x * L);
          }
        }
        tma_pending = more;
        note_a();
      }
      wait_a();
      if (pp > 0) wait_b();  // the previous pair's stage B has read the operand
#pragma unroll
      for (int j = 0; j < MT; ++j) {
        const int ra = row + 128 * j;
        stage_b_half<N>(sm, G::OPB, tlane + G::GA + j * KA, ra / R2, ra % R2, h, true);
      }
      NS_TC_PUBLISH_OR_LEAVE
      if (tid == 0) {
        fence_after();
        issue_b<N>(sbase, tmem, G::OPB, G::T1 + pp * G::KB);
        commit(&bars[1]);
      }
      note_b();
    }
    wait_b();
    // ------------------------------------- product, forward stage-A rows --
    // this thread: points n = c + R1 d of line `line`, d in its chunks; u =
    // (T1.re, T1.im, T2.re), w = (T2.im, T3.re, T3.im); forward operands z =
    // conj(n_x + i n_y) into the OPA tiles and z = conj(n_z[even line] + i
    // n_z[odd line]) into the OPB region (free: the last inverse stage B has
    // completed), laid out as a stage-A tile
    {
      const int par = line & 1, q = line >> 1;
#pragma unroll
      for (int cc = 0; cc < NCH / 2; ++cc) {
        const int d0 = (2 * cc + h) * CHK;
        float ux[CHK], uy[CHK], uz[CHK], wx[CHK], wy[CHK], wz[CHK];
        tmem_ld<CHK>(tlane + G::T1 + d0, ux);
        tmem_ld<CHK>(tlane + G::T1 + R2 + d0, uy);
        tmem_ld<CHK>(tlane + G::T2 + d0, uz);
        tmem_ld<CHK>(tlane + G::T2 + R2 + d0, wx);
        tmem_ld<CHK>(tlane + G::T3 + d0, wy);
        tmem_ld<CHK>(tlane + G::T3 + R2 + d0, wz);
        tmem_wait_ld();
        const float inv_suz = lscale[line];
#pragma unroll
        for (int i = 0; i < CHK; ++i) uz[i] *= inv_suz;
        float nx[CHK], ny[CHK], nz[CHK], nzp[CHK];
#pragma unroll
        for (int i = 0; i < CHK; ++i) {
          nx[i] = fmaf(uy[i], wz[i], -(uz[i] * wy[i]));
          ny[i] = -fmaf(uz[i], wx[i], -(ux[i] * wz[i]));  // stored negated: z = conj(n_x + i n_y)
          nz[i] = fmaf(ux[i], wy[i], -(uy[i] * wx[i]));
          umx = fmaxf(umx, fabsf(ux[i]));
          umy = fmaxf(umy, fabsf(uy[i]));
          umz = fmaxf(umz, fabsf(uz[i]));
        }
#pragma unroll
        for (int i = 0; i < CHK; ++i) nzp[i] = __shfl_xor_sync(0xffffffffu, nz[i], R1);
        // (n_x, -n_y) rows (line, c + R1 jj), K = a = d / MT
        constexpr int RUN = CHK / MT;
#pragma unroll
        for (int jj = 0; jj < MT; ++jj) {
          const int ra = line * R2 + c + R1 * jj;
          unsigned char *tile_p = sm + G::OPA + (ra >> 7) * 2 * G::TILE_A;
          float xr[RUN], xi[RUN];
#pragma unroll
          for (int e = 0; e < RUN; ++e) {
            xr[e] = nx[jj + MT * e];
            xi[e] = ny[jj + MT * e];
          }
          const int a0 = d0 / MT;
          put_run<RUN>(kmajor(tile_p, ra & 127, a0, KA * 16), G::TILE_A, xr);
          put_run<RUN>(kmajor(tile_p, ra & 127, R1 + a0, KA * 16), G::TILE_A, xi);
        }
        // n_z pair rows (q, b): MT = 2: b = c + R1 par, the points of parity
        // par; MT = 1: b = c, the K range split between the two lines
        {
          float xr[RUN], xi[RUN];
          bool mine;
          int r, a0;
          if constexpr (MT == 2) {
#pragma unroll
            for (int e = 0; e < RUN; ++e) {
              const float own = par ? nz[2 * e + 1] : nz[2 * e], oth = par ? nzp[2 * e + 1] : nzp[2 * e];
              xr[e] = par ? oth : own;
              xi[e] = -(par ? own : oth);
            }
            mine = true;
            r = q * R2 + c + R1 * par;
            a0 = d0 / 2;
          } else {
#pragma unroll
            for (int e = 0; e < RUN; ++e) {
              xr[e] = par ? nzp[e] : nz[e];
              xi[e] = -(par ? nz[e] : nzp[e]);
            }
            mine = (d0 >= R1 / 2 ? 1 : 0) == par;
            r = q * R2 + c;
            a0 = d0;
          }
          if (mine) {
            put_run<RUN>(kmajor(sm + G::OPB, r, a0, KA * 16), G::TILE_A, xr);
            put_run<RUN>(kmajor(sm + G::OPB, r, R1 + a0, KA * 16), G::TILE_A, xi);
          }
        }
      }
    }
    NS_TC_PUBLISH_OR_LEAVE
    if (tid == 0) {
      fence_after();
      for (int t = 0; t < MT; ++t) issue_a<N>(sbase, tmem, G::OPA + t * 2 * G::TILE_A, G::GA + t * KA);
      issue_a<N>(sbase, tmem, G::OPB, G::T3);
      commit(&bars[0]);
    }
    note_a();
    wait_a();
    // ------------------------------------------------ forward stage B ------
    // (n_x, n_y) pairs into OPB, n_z pairs into OPA (both stage-A operands
    // have been read: stage A has completed)
#pragma unroll
    for (int j = 0; j < MT; ++j) {
      const int ra = row + 128 * j;
      stage_b_half<N>(sm, G::OPB, tlane + G::GA + j * KA, ra / R2, ra % R2, h, true);
    }
    stage_b_half<N>(sm, G::OPA, tlane + G::T3, row / R2, row % R2, h, row < 64 * MT);
    NS_TC_PUBLISH_OR_LEAVE
    if (tid == 0) {
      fence_after();
      issue_b<N>(sbase, tmem, G::OPB, G::T1);
      issue_b<N>(sbase, tmem, G::OPA, G::T2);
      commit(&bars[1]);
    }
    note_b();
    // ----------------------------------------------------------- outputs ---
    wait_b();
    // F1 rows (line, c): half 0 stores n_x, half 1 n_y
    split_store<N>(tlane + G::T1, c, lane, h == 1, true, yb + h * fs + (line0 + line) * hs);
    // F2 rows (q, c), q < L / 2 (lanes 0..63): half 0 stores n_z of line 2q, half 1 of line 2q + 1
    if ((warp & 3) < 2) split_store<N>(tlane + G::T2, c, lane, h == 1, true, yb + 2 * fs + (line0 + 2 * line + h) * hs);
    if (__syncthreads_or(bad)) {  // (also keeps the blocks' warps in step: 1.34 ms with it, 1.40 without)
      failed = true;
      goto out;
    }
  }
#undef NS_TC_PUBLISH_OR_LEAVE
out:
  if (umax != nullptr) {
    double m[3] = {umx, umy, umz};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      for (int off = 16; off > 0; off >>= 1) m[i] = fmax(m[i], __shfl_xor_sync(0xffffffffu, m[i], off));
      if (lane == 0)
        atomicMax(umax + i * kUmaxSlots + blockIdx.x % kUmaxSlots, (unsigned long long)__double_as_longlong(m[i]));
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 2);
    if (tma_pending) wait_phase(&bars[2], pht);  // let a copy in flight land before the block leaves
    // MMAs this thread has not seen complete may still write tensor memory:
    // give each one a last bounded wait before the memory is freed
    if (pend_a) wait_phase(&bars[0], par_a);
    if (pend_b) wait_phase(&bars[1], par_b);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, G::TCOLS);
}

}  // namespace tc
}  // namespace nsk
