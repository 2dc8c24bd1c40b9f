// Persistent skew-packed stepper, instantiations for GROM_BF16 storage.
#include "k1pp_dispatch.cuh"

namespace grom {

cudaError_t k1pp_dispatch_bf16(int qm, int nb, const K1Plan& pl, const K1Args& a, const StepArgs& st,
                             const K1PPArgs& pp, cudaStream_t s) {
  return K1PPDispatch<GROM_BF16, 64>::run(qm, nb, pl, a, st, pp, s);
}

}  // namespace grom
