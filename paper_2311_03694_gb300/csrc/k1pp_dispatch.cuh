// Template-width dispatch of the persistent skew-packed stepper for one
// storage type (widths as for the streaming kernel, at most 4 trajectories so
// that the ring, the states and the step's shared tables fit one CTA).
#pragma once

#include "k1p_persist.cuh"

namespace grom {

template <int ST, int CAP>
struct K1PPDispatch {
  template <int QM, int NB>
  static cudaError_t pick(const K1Plan& pl, const K1Args& a, const StepArgs& st, const K1PPArgs& pp, cudaStream_t s) {
    if constexpr (K1Traits<ST>::ACC_WORDS * K1Traits<ST>::EPV * QM * NB <= CAP && NB <= 4)
      return k1pp_launch_one<ST, QM, NB>(pl, a, st, pp, s);
    return cudaErrorInvalidValue;
  }
  template <int QM>
  static cudaError_t pick_nb(int nb, const K1Plan& pl, const K1Args& a, const StepArgs& st, const K1PPArgs& pp,
                             cudaStream_t s) {
    switch (nb) {
      case 1: return pick<QM, 1>(pl, a, st, pp, s);
      case 2: return pick<QM, 2>(pl, a, st, pp, s);
      case 4: return pick<QM, 4>(pl, a, st, pp, s);
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t run(int qm, int nb, const K1Plan& pl, const K1Args& a, const StepArgs& st, const K1PPArgs& pp,
                         cudaStream_t s) {
    switch (qm) {
      case 1: return pick_nb<1>(nb, pl, a, st, pp, s);
      case 2: return pick_nb<2>(nb, pl, a, st, pp, s);
    }
    return cudaErrorInvalidValue;
  }
};

}  // namespace grom
