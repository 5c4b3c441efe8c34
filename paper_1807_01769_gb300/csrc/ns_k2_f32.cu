// ns_k2_f32.cu -- instantiates the 2D pass kernels in float for every supported N.
#include "ns_kernels.cuh"

namespace nsk {

int dispatch2_f32(int op, const Args &a, cudaStream_t s) {
  switch (a.g.N) {
    case 16: return Launch2<float, 16>::run(op, a, s);
    case 32: return Launch2<float, 32>::run(op, a, s);
    case 64: return Launch2<float, 64>::run(op, a, s);
    case 128: return Launch2<float, 128>::run(op, a, s);
    case 256: return Launch2<float, 256>::run(op, a, s);
    case 512: return Launch2<float, 512>::run(op, a, s);
    case 1024: return Launch2<float, 1024>::run(op, a, s);
    case 2048: return Launch2<float, 2048>::run(op, a, s);
    default: return -1;
  }
}

}  // namespace nsk
