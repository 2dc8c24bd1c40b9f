// Template-width dispatch of the packed streaming kernel for one storage type:
// QM (positions per thread per row) and NB (trajectories per pass) are
// compile-time; widths whose accumulators exceed the register cap are not
// instantiated.
#pragma once

#include "k1_packed.cuh"

namespace grom {

template <int ST, int CAP>
struct K1PDispatch {
  template <int QM, int NB>
  static constexpr bool valid() {
    return K1Traits<ST>::ACC_WORDS * K1Traits<ST>::EPV * QM * NB <= CAP;
  }
  template <int QM, int NB>
  static cudaError_t pick(const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
    if constexpr (valid<QM, NB>()) return k1p_launch_one<ST, QM, NB>(pl, a, b0, s);
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
  static cudaError_t run(int qm, int nb, const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
    switch (qm) {
      case 1: return pick_nb<1>(nb, pl, a, b0, s);
      case 2: return pick_nb<2>(nb, pl, a, b0, s);
      case 4: return pick_nb<4>(nb, pl, a, b0, s);
      case 8: return pick_nb<8>(nb, pl, a, b0, s);
    }
    return cudaErrorInvalidValue;
  }
};

}  // namespace grom
