// Skew-packed streaming contraction, instantiations for GROM_F64 storage.
#include "k1p_dispatch.cuh"

namespace grom {

cudaError_t k1p_dispatch_f64(int qm, int nb, const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  return K1PDispatch<GROM_F64, 64>::run(qm, nb, pl, a, b0, s);
}

}  // namespace grom
