// ns_k2_f64.cu -- instantiates the 2D pass kernels in double for every supported N.
#include "ns_kernels.cuh"

namespace nsk {

int dispatch2_f64(int op, const Args &a, cudaStream_t s) {
  switch (a.g.N) {
    case 16: return Launch2<double, 16>::run(op, a, s);
    case 32: return Launch2<double, 32>::run(op, a, s);
    case 64: return Launch2<double, 64>::run(op, a, s);
    case 128: return Launch2<double, 128>::run(op, a, s);
    case 256: return Launch2<double, 256>::run(op, a, s);
    case 512: return Launch2<double, 512>::run(op, a, s);
    case 1024: return Launch2<double, 1024>::run(op, a, s);
    case 2048: return Launch2<double, 2048>::run(op, a, s);
    default: return -1;
  }
}

}  // namespace nsk
