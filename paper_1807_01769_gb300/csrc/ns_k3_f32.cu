// ns_k3_f32.cu -- instantiates the 3D pass kernels in float for every supported N.
#include "ns_kernels.cuh"

namespace nsk {

int dispatch3_f32(int op, const Args &a, cudaStream_t s) {
  switch (a.g.N) {
    case 16: return Launch3<float, 16>::run(op, a, s);
    case 32: return Launch3<float, 32>::run(op, a, s);
    case 64: return Launch3<float, 64>::run(op, a, s);
    case 128: return Launch3<float, 128>::run(op, a, s);
    case 256: return Launch3<float, 256>::run(op, a, s);
    case 512: return Launch3<float, 512>::run(op, a, s);
    case 1024: return Launch3<float, 1024>::run(op, a, s);
    default: return -1;
  }
}

}  // namespace nsk
