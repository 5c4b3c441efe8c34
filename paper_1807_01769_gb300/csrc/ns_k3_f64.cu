// ns_k3_f64.cu -- instantiates the 3D pass kernels in double for every supported N.
#include "ns_kernels.cuh"

namespace nsk {

int dispatch3_f64(int op, const Args &a, cudaStream_t s) {
  switch (a.g.N) {
    case 16: return Launch3<double, 16>::run(op, a, s);
    case 32: return Launch3<double, 32>::run(op, a, s);
    case 64: return Launch3<double, 64>::run(op, a, s);
    case 128: return Launch3<double, 128>::run(op, a, s);
    case 256: return Launch3<double, 256>::run(op, a, s);
    case 512: return Launch3<double, 512>::run(op, a, s);
    case 1024: return Launch3<double, 1024>::run(op, a, s);
    default: return -1;
  }
}

}  // namespace nsk
