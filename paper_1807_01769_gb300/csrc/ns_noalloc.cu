// ns_noalloc.cu -- ns_diagnostics_noalloc: the FP64 diagnostics reduction
// (energy, enstrophy, shell spectrum) for callers that cannot allocate device
// memory themselves.
//
// Who needs it: ordinary host code that must not call cudaMalloc -- a custom
// allocator's hook, code running under a memory pool that must not grow, or a
// process whose device memory is owned and budgeted by another framework.
// Such a caller already holds the spectrum and an output buffer; the only
// device memory the reduction needs beyond them is the per-block partial sums,
// and here that scratch is a fixed array compiled into the library.  The call
// itself makes CUDA runtime calls and launches kernels, so it cannot be made
// from a stream callback or a host function enqueued with cudaLaunchHostFunc.
//
// The array is file-scope device memory: every GPU that loads the library
// holds NS_NOALLOC_SCRATCH_DOUBLES doubles (2 MiB) for the life of the
// process.  With CUDA's lazy module loading the module that holds it is
// loaded, and those 2 MiB committed, on its first use on a device: the first
// call on each device is a warm-up to make outside any region where
// allocation is forbidden and before any stream capture.  In host code the
// array's name is only a host-side stand-in, never a device address, so every
// call looks up the device address with cudaGetSymbolAddress, with the
// calling device current (cheap next to the two launches, and never stale
// after a device reset reloads the module).
// Every call shares the array.  Each block overwrites its own partial row
// before the final pass reads it, so nothing has to be cleared between calls,
// but two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on the array.
#include <cuda_runtime.h>

#include <cmath>

#include "ns.h"
#include "ns_internal.h"

namespace {

static __device__ __align__(256) double g_noalloc_scratch[NS_NOALLOC_SCRATCH_DOUBLES];

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
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return NS_ECUDA;
  double *scratch = static_cast<double *>(p);
  const int rc = nsk::diagnostics(grid->precision, g, spec_dev, nbins, scratch, out_dev, (cudaStream_t)cuda_stream);
  if (rc != 0) return NS_ECUDA;
  return NS_OK;
}
