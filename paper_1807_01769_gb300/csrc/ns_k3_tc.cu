// ns_k3_tc.cu -- instantiates the tensor-core 3D x pass (ns_tc.cuh) and builds
// its DFT matrices.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ns_tc.cuh"
#include "ns_tc.h"

namespace nsk {
namespace {

uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (finite values)
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Real-block matrix of the length-R DFT with exponent +2 pi i a c / R, as the
// K-major B operand [n'][k'] (n' = q R + c output, k' = p R + a input; q, p =
// 0 real, 1 imaginary): entries cos, -sin (p = 1, q = 0), sin (p = 0, q = 1),
// cos.  hi and lo BF16 halves at out and out + (2R)^2 * 2 bytes.
void put_dft(unsigned char *out, int R) {
  const int K = 2 * R;
  const size_t half = (size_t)K * K * 2;
  for (int q = 0; q < 2; ++q)
    for (int c = 0; c < R; ++c)
      for (int p = 0; p < 2; ++p)
        for (int a = 0; a < R; ++a) {
          const double th = 2.0 * M_PI * (double)((a * c) % R) / R;
          const double v = (p == q) ? std::cos(th) : (p == 1 ? -std::sin(th) : std::sin(th));
          const int n = q * R + c, k = p * R + a;
          const size_t off = (size_t)(n / 8) * (K * 16) + (size_t)(k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
          const uint16_t hi = bf16_rn((float)v);
          const uint16_t lo = bf16_rn((float)(v - bf16_value(hi)));
          std::memcpy(out + off, &hi, 2);
          std::memcpy(out + half + off, &lo, 2);
        }
}

template <int N>
std::vector<unsigned char> matrices() {
  using G = tc::Geom<N>;
  std::vector<unsigned char> m(G::MATS_BYTES, 0);
  put_dft(m.data(), G::R1);
  put_dft(m.data() + 2 * G::FA_HALF, G::R2);
  return m;
}

// blocks per SM of the kernel for N, found once at OP_PREPARE (outside any
// stream capture, where the occupancy query may not run)
template <int N>
int &blocks_per_sm() {
  static int v = 0;
  return v;
}

template <int N>
int launch(int op, const Args &a, const void *mats, const void *tmap, cudaStream_t s) {
  using G = tc::Geom<N>;
  if (op == OP_PREPARE) {
    set_smem(tc::k3_xpass_tc<N>, G::SMEM);
    // the largest shared-memory carveout, so that the SM holds the blocks the
    // tensor memory allows
    cudaFuncSetAttribute(tc::k3_xpass_tc<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    // resident blocks from the kernel's registers and shared memory and the
    // tensor memory it allocates (counted here: the occupancy query does not
    // see the tensor memory and answered one block per SM for this kernel)
    int per_sm = 1;
    cudaFuncAttributes fa{};
    int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0;
    if (cudaFuncGetAttributes(&fa, tc::k3_xpass_tc<N>) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
      const int regs_block = (fa.numRegs + 7) / 8 * 8 * tc::kThreads;
      const int by_regs = regs_block > 0 ? regs_sm / regs_block : 1;
      const int by_smem = smem_sm / (int)(G::SMEM + fa.sharedSizeBytes + reserved);
      per_sm = by_regs < by_smem ? by_regs : by_smem;
    }
    blocks_per_sm<N>() = per_sm < 1 ? 1 : (per_sm > G::CTAS ? G::CTAS : per_sm);
    cudaGetLastError();
    return dispatch3_f32(op, a, s);
  }
  if (op != OP_XPASS) return dispatch3_f32(op, a, s);
  if (tmap == nullptr || a.g.hs != G::HS) return (int)cudaErrorInvalidValue;
  const int per_sm = blocks_per_sm<N>() > 0 ? blocks_per_sm<N>() : 1;
  const long long lines = (long long)(a.nz > 0 ? a.nz : N) * N, tiles = lines / G::L;
  const long long slots = (long long)per_sm * (a.nsm > 0 ? a.nsm : 1);
  const long long grid = tiles < slots ? tiles : slots;
  tc::k3_xpass_tc<N><<<(unsigned)grid, tc::kThreads, G::SMEM, s>>>(a.g, (long long)a.z0 * N, tiles, (float2 *)a.yb,
                                                                   (const float2 *)a.tw, (const uint4 *)mats,
                                                                   *reinterpret_cast<const CUtensorMap *>(tmap),
                                                                   a.umax, a.err);
  return (int)cudaGetLastError();
}

}  // namespace

bool tc_supported(int N) { return N == 64 || N == 128 || N == 256 || N == 512; }

std::vector<unsigned char> tc_matrices(int N) {
  switch (N) {
    case 64: return matrices<64>();
    case 128: return matrices<128>();
    case 256: return matrices<256>();
    case 512: return matrices<512>();
    default: return {};
  }
}

int tc_lines_per_tile(int N) {
  switch (N) {
    case 64: return tc::Geom<64>::L;
    case 128: return tc::Geom<128>::L;
    case 256: return tc::Geom<256>::L;
    case 512: return tc::Geom<512>::L;
    default: return 0;
  }
}

int dispatch3_tc(int op, const Args &a, const void *mats, const void *tmap, cudaStream_t s) {
  switch (a.g.N) {
    case 64: return launch<64>(op, a, mats, tmap, s);
    case 128: return launch<128>(op, a, mats, tmap, s);
    case 256: return launch<256>(op, a, mats, tmap, s);
    case 512: return launch<512>(op, a, mats, tmap, s);
    default: return -1;
  }
}

}  // namespace nsk
