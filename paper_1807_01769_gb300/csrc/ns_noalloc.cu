// ns_noalloc.cu -- ns_diagnostics_noalloc: the FP64 diagnostics reduction
// (energy, enstrophy, shell spectrum) for callers that cannot allocate device
// memory themselves.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator's hook, under a memory pool that must
// not grow, or in a process whose device memory is owned and budgeted by
// another framework.  Such a caller already holds the spectrum and an output
// buffer; the only device memory the reduction needs beyond them is the
// per-block partial sums, and here that scratch is a fixed array compiled into
// the library.
//
// The array is file-scope device memory: every GPU that loads the library
// holds NS_NOALLOC_SCRATCH_DOUBLES doubles (2 MiB) for the life of the
// process.  In host code its name is only a host-side stand-in, never a device
// address, so its address is looked up with cudaGetSymbolAddress once per
// device, with that device current, on the first call made on that device.
// Every call shares the array.  Each block overwrites its own partial row
// before the final pass reads it, so nothing has to be cleared between calls,
// but two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ns.h"
#include "ns_internal.h"

namespace {

static __device__ __align__(256) double g_noalloc_scratch[NS_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" int ns_diagnostics_noalloc(const ns_grid *grid, const void *spec_dev, double *out_dev,
                                      void *cuda_stream) {
  if (!grid || !spec_dev || !out_dev) return NS_EINVAL;
  if ((grid->dim != 2 && grid->dim != 3) || !is_pow2(grid->n) ||
      (grid->precision != NS_FP64 && grid->precision != NS_FP32))
    return NS_EINVAL;
  if (grid->n < 16 || grid->n > (grid->dim == 3 ? 1024 : 2048))
    return NS_EUNSUPPORTED;
  nsk::Geo g{};
  g.dim = grid->dim;
  g.N = grid->n;
  g.kc = (g.N - 1) / 3;
  g.c = 2 * g.kc + 1;
  g.h = g.kc + 1;
  g.hs = g.h;  // canonical layout: rows of h complex numbers, no padding
  g.st_comp = (g.dim == 3 ? (long long)g.c * g.c : (long long)g.c) * g.h;
  const int nbins = (int)std::floor(std::sqrt((double)g.dim * g.kc * g.kc) + 0.5) + 1;
  const long long need = nsk::diag_scratch_doubles(g, nbins);
  if (need > NS_NOALLOC_SCRATCH_DOUBLES) return NS_EUNSUPPORTED;  // grid too large for the static scratch
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return NS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return NS_EUNSUPPORTED;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return NS_ECUDA;
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  const int rc = nsk::diagnostics(grid->precision, g, spec_dev, nbins, scratch, out_dev, (cudaStream_t)cuda_stream);
  if (rc != 0) return NS_ECUDA;
  return NS_OK;
}
