// ns_tma.cu -- host side of the TMA loads: tensor maps for the pass buffers,
// encoded through the driver's cuTensorMapEncodeTiled (reached through the
// runtime's entry-point query, so the library needs no link to libcuda).
#include <cuda.h>
#include <cuda_runtime.h>

#include "ns_internal.h"

namespace nsk {

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  }
  return fn;
}
}  // namespace

int make_tensor_map(void *out, const void *base, int rank, const unsigned long long *dims,
                    const unsigned long long *strides_bytes, const unsigned *box) {
  EncodeTiled fn = encoder();
  if (!fn) return (int)cudaErrorNotSupported;
  if (rank < 2 || rank > 3) return (int)cudaErrorInvalidValue;
  // 8-byte elements (FLOAT64 as a container: the copy moves bits, it converts nothing)
  cuuint64_t d[3], st[2];
  cuuint32_t b[3], estr[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i + 1 < rank; ++i) st[i] = strides_bytes[i];
  const CUresult r = fn(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank,
                        const_cast<void *>(base), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace nsk
