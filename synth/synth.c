/*
 * Seeded synthetic workload generator (shared by the CPU oracle tests and the
 * GPU library's tests and benchmark).  It holds none of the method's
 * arithmetic: it only draws counter-based random numbers and assembles the
 * workload tensors that the paper's experiments would have loaded from disk.
 *
 * Random numbers: a counter-based SplitMix64 stream.  Draw number `ctr` of
 * stream `stream` under `seed` is
 *     mix64( mix64(seed ^ (stream * K_STREAM)) + ctr * K_GOLDEN )
 * where mix64 is the SplitMix64 finaliser (Steele, Lea, Flood 2014).  A
 * standard normal with linear index `idx` uses draws 2*idx and 2*idx+1 as two
 * 53-bit uniforms u1 in (0,1], u2 in [0,1) and takes the cosine branch of the
 * Box-Muller transform, z = sqrt(-2 ln u1) cos(2 pi u2), in FP64 with libm.
 *
 * Every element is a pure function of (seed, stream, index), so a row slab of
 * a tensor that is too big for host memory can be regenerated on demand.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define K_GOLDEN 0x9E3779B97F4A7C15ULL
#define K_STREAM 0xD1B54A32D192ED03ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return mix64(mix64(seed ^ (stream * K_STREAM)) + ctr * K_GOLDEN);
}

uint64_t synth_draw_u64(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return draw(seed, stream, ctr);
}

/* uniform in [0,1) from draw number ctr */
double synth_uniform(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return (double)(draw(seed, stream, ctr) >> 11) * 0x1.0p-53;
}

double synth_normal(uint64_t seed, uint64_t stream, uint64_t idx) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = (double)((draw(seed, stream, 2 * idx) >> 11) + 1) * 0x1.0p-53;
  double u2 = (double)(draw(seed, stream, 2 * idx + 1) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

void synth_fill_normal(uint64_t seed, uint64_t stream, uint64_t start, int64_t count,
                       double scale, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < count; ++t) out[t] = scale * synth_normal(seed, stream, start + (uint64_t)t);
}

/*
 * Adds scale * (G_ijk - G_kji) to rows i0..i1-1 of an n x n x n row-major
 * tensor slab (out has (i1-i0)*n*n entries, entry ((i-i0)*n+j)*n+k), with
 * G_ijk = normal(seed, stream, (i*n+j)*n+k).  The difference of two FP64
 * numbers is negated exactly when its operands swap, so the added part is
 * exactly skew in the first and third index.
 */
void synth_add_skew_normal_slab(int64_t n, uint64_t seed, uint64_t stream, double scale,
                                int64_t i0, int64_t i1, double* out) {
  int64_t rows = (i1 - i0) * n;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r) {
    int64_t i = i0 + r / n, j = r % n;
    double* o = out + r * n;
    for (int64_t k = 0; k < n; ++k) {
      double g = synth_normal(seed, stream, (uint64_t)((i * n + j) * n + k));
      double gt = synth_normal(seed, stream, (uint64_t)((k * n + j) * n + i));
      o[k] += scale * (g - gt);
    }
  }
}
