// K1 streaming contraction, instantiations for GROM_F32X2 storage.
#include "k1_stream.cuh"

namespace grom {

template <int QM, int NB>
static constexpr bool k1_valid() {
  return K1Traits<GROM_F32X2>::ACC_WORDS * K1Traits<GROM_F32X2>::EPV * QM * NB <= 32;
}

template <int QM, int NB>
static cudaError_t pick(const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  if constexpr (k1_valid<QM, NB>()) return k1_launch_one<GROM_F32X2, QM, NB>(pl, a, b0, s);
  return cudaErrorInvalidValue;
}

template <int QM>
static cudaError_t pick_nb(int nb, const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  switch (nb) {
    case 1: return pick<QM, 1>(pl, a, b0, s);
    case 2: return pick<QM, 2>(pl, a, b0, s);
    case 4: return pick<QM, 4>(pl, a, b0, s);
    case 8: return pick<QM, 8>(pl, a, b0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t k1_dispatch_f32x2(int qm, int nb, const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  switch (qm) {
    case 1: return pick_nb<1>(nb, pl, a, b0, s);
    case 2: return pick_nb<2>(nb, pl, a, b0, s);
    case 4: return pick_nb<4>(nb, pl, a, b0, s);
    case 8: return pick_nb<8>(nb, pl, a, b0, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace grom
