// Persistent skew-packed stepper, instantiations for GROM_F32X2 storage.
#include "k1pp_dispatch.cuh"

namespace grom {

cudaError_t k1pp_dispatch_f32x2(int qm, int nb, const K1Plan& pl, const K1Args& a, const StepArgs& st,
                             const K1PPArgs& pp, cudaStream_t s) {
  return K1PPDispatch<GROM_F32X2, 32>::run(qm, nb, pl, a, st, pp, s);
}

}  // namespace grom
