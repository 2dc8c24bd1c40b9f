// K1: single/few-trajectory dense advection contraction, HBM streaming.
//
//   c_i = sum_j u_j sum_k C_ijk u_k            (Sec. 2.2, eq. Cu; 2N^3 flops, N^3 words)
//
// The stored tensor is a sequence of N*m rows (i, j) of np elements (k padded
// with zeros); m = N for the G-ROM.  For the SVD-ROM (Sec. 4.4.2) the same
// kernel streams the slices V[i][r][k] (m = rank) with the middle index
// weighted by beta = sigma o (U^T u) instead of u.  A persistent grid splits the rows into chunks of whole rows
// that never straddle a test index i, and each CTA streams a contiguous range
// of chunks through a ring of shared-memory stages filled by bulk TMA copies
// (cp.async.bulk, completion on an mbarrier).  One producer warp issues the
// copies; eight consumer warps read the stages.
//
// The consumers accumulate per advected index: each thread owns fixed
// positions k of the row and keeps acc_k = sum_j C_ijk u_j over the rows j of
// the current test index (u_j is a shared-memory broadcast), so no reduction
// happens per row.  When the test index changes, each thread folds its
// accumulators into sum_k u_k acc_k and every warp writes one partial per
// trajectory; a finalize kernel sums the partials of each i in a fixed order
// (deterministic, no atomics).
#pragma once

#include "ds_arith.cuh"
#include "grom_internal.h"
#include "ptx.cuh"

namespace grom {

template <int ST>
struct K1Traits;
template <>
struct K1Traits<GROM_F64> {
  static constexpr int EPV = 2;          // elements per 16-byte vector
  static constexpr int U_BYTES = 8;      // shared-memory bytes of u per element
  static constexpr int ACC_WORDS = 2;    // 32-bit registers per accumulator
};
template <>
struct K1Traits<GROM_F32X2> {
  static constexpr int EPV = 4;  // per plane (hi plane, then lo plane, per row)
  static constexpr int U_BYTES = 8;
  static constexpr int ACC_WORDS = 2;
};
template <>
struct K1Traits<GROM_F32> {
  static constexpr int EPV = 4;
  static constexpr int U_BYTES = 4;
  static constexpr int ACC_WORDS = 1;
};
template <>
struct K1Traits<GROM_BF16> {
  static constexpr int EPV = 8;
  static constexpr int U_BYTES = 4;
  static constexpr int ACC_WORDS = 1;
};

// Row layout of the stored tensor: a row of np elements occupies
// np * elem_bytes bytes.  F32X2 rows are [hi(np floats) | lo(np floats)].
// Vector positions per row (16-byte vectors, per plane for F32X2):
template <int ST>
__host__ __device__ inline int64_t k1_positions(int64_t np) {
  return np / K1Traits<ST>::EPV;
}

// Accumulator types.
template <int ST>
struct Acc;
template <>
struct Acc<GROM_F64> {
  double v;
  __device__ void zero() { v = 0.0; }
};
template <>
struct Acc<GROM_F32X2> {
  float S, s;
  __device__ void zero() { S = 0.f; s = 0.f; }
};
template <>
struct Acc<GROM_F32> {
  float v;
  __device__ void zero() { v = 0.f; }
};
template <>
struct Acc<GROM_BF16> {
  float v;
  __device__ void zero() { v = 0.f; }
};

// Error-free accumulation of C*u for F32X2 storage: ds_mac (ds_arith.cuh) of
// the stored (hi, lo) pair and the state's (uh, ul) pair into the
// accumulator (S, s), which ds_renorm renormalises before every streamed
// chunk (every 4 rows per accumulator at N = 1024).  Per-evaluation error at
// N = 256 in a CPU emulation of the arithmetic: 3.7e-14, against 1.1e-13 for
// Knuth's full TwoSum per term without renormalisation.
template <int ST, int QM, int EPV, int NB, typename A>
__device__ __forceinline__ void ds_renorm_all(A (&acc)[QM][EPV][NB]) {
  if constexpr (ST == GROM_F32X2) {
#pragma unroll
    for (int q = 0; q < QM; ++q)
#pragma unroll
      for (int e = 0; e < EPV; ++e)
#pragma unroll
        for (int b = 0; b < NB; ++b) ds_renorm(acc[q][e][b].S, acc[q][e][b].s);
  }
}

// Loads one vector per trajectory of the pass into shared memory in the
// arithmetic type of the storage (F32X2: a hi plane, then a lo plane):
// entry (b, k) = src(b, k) for k < len, where src returns 0 past the
// meaningful length and for inactive trajectories.
template <int ST, int NB, typename F>
__device__ __forceinline__ void k1_load_vec(uint8_t* dst, int64_t len, F src) {
  for (int64_t idx = threadIdx.x; idx < (int64_t)NB * len; idx += blockDim.x) {
    const int b = (int)(idx / len);
    const double v = src(b, idx - (int64_t)b * len);
    if constexpr (ST == GROM_F64) {
      reinterpret_cast<double*>(dst)[idx] = v;
    } else if constexpr (ST == GROM_F32X2) {
      const float h = __double2float_rn(v);
      reinterpret_cast<float*>(dst)[idx] = h;
      reinterpret_cast<float*>(dst)[(int64_t)NB * len + idx] = __double2float_rn(v - (double)h);
    } else {
      reinterpret_cast<float*>(dst)[idx] = __double2float_rn(v);
    }
  }
}

// u of the pass into ureg (np per trajectory) and, with separate middle
// weights, those into the array after it (mp per trajectory).  Returns the
// middle-weight array and its per-trajectory length through mreg and mp.
template <int ST, int NB>
__device__ __forceinline__ void k1_load_state(const K1Plan& pl, const K1Args& a, int b0, uint8_t* ureg,
                                              const uint8_t*& mreg, int64_t& mp) {
  const int64_t n = pl.n, np = pl.np;
  auto live = [&](int b) { return b < a.nb && (a.active == nullptr || a.active[b0 + b]); };
  k1_load_vec<ST, NB>(ureg, np, [&](int b, int64_t k) -> double {
    if (!live(b) || k >= n) return 0.0;
    const int bg = b0 + b;
    const double* ub = a.taken ? a.hist + bg * a.hist_stride + (a.taken[bg] % 3) * n : a.u + bg * a.u_stride;
    return ub[k];
  });
  mreg = ureg;
  mp = np;
  if (pl.has_mid) {
    uint8_t* m = ureg + (int64_t)NB * np * K1Traits<ST>::U_BYTES;
    k1_load_vec<ST, NB>(m, pl.mp, [&](int b, int64_t r) -> double {
      if (!live(b) || r >= pl.m) return 0.0;
      return a.mid[(int64_t)(b0 + b) * a.mid_stride + r];
    });
    mreg = m;
    mp = pl.mp;
  }
}

template <int ST, int QM, int NB>
__global__ void __launch_bounds__(K1_THREADS, 1) k1_stream_kernel(const K1Plan pl, const K1Args a, const int b0) {
  using TR = K1Traits<ST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + K1_STAGES * K1_STAGE_BYTES);
  uint64_t* empty = full + K1_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + K1_STAGES);
  uint8_t* ureg = reinterpret_cast<uint8_t*>(empty + K1_STAGES) + 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = pl.n, np = pl.np, row_bytes = pl.row_bytes;
  const int64_t G = gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * pl.T / G, c1 = ((int64_t)blockIdx.x + 1) * pl.T / G;

  if (tid == 0) {
    for (int s = 0; s < K1_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], K1_CONSUMERS / 32);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }

  // u of the NB trajectories of this pass (zero-padded to np) and the middle
  // weights (u itself for the G-ROM), in the arithmetic type of the storage
  const uint8_t* mreg;
  int64_t mp;
  k1_load_state<ST, NB>(pl, a, b0, ureg, mreg, mp);
  __syncthreads();

  if (warp == K1_CONSUMERS / 32) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t it = 0;
      int64_t i = c0 / pl.cpi, jc = c0 - i * pl.cpi;  // chunk (i, jc), advanced incrementally
      int s = 0;
      uint32_t ph = 0;
      for (int64_t c = c0; c < c1; ++c, ++it) {
        if (it >= K1_STAGES && !ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
          *abort_flag = 1;
          atomicOr(a.err, DEV_ERR_TIMEOUT);
          break;
        }
        const int64_t j0 = jc * pl.rpc;
        const int64_t rows = pl.m - j0 < pl.rpc ? pl.m - j0 : pl.rpc;
        const uint32_t bytes = (uint32_t)(rows * row_bytes);
        ptx::mbar_arrive_expect_tx(&full[s], bytes);
        ptx::bulk_g2s(stages + (size_t)s * K1_STAGE_BYTES, a.tensor + (i * pl.m + j0) * row_bytes, bytes, &full[s]);
        if (++jc == pl.cpi) { jc = 0; ++i; }
        if (++s == K1_STAGES) { s = 0; ph ^= 1u; }
      }
      // Let every copy this CTA issued land before the CTA can exit.
      const int64_t issued = it;
      for (int64_t q = issued > K1_STAGES ? issued - K1_STAGES : 0; q < issued; ++q) {
        if (!ptx::mbar_wait(&full[q % K1_STAGES], (uint32_t)((q / K1_STAGES) & 1), nullptr))
          atomicOr(a.err, DEV_ERR_TIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int64_t P = k1_positions<ST>(np);
    int64_t rpr, ro, pos0;
    bool act;
    if (P >= K1_CONSUMERS) {
      rpr = 1; ro = 0; pos0 = tid; act = true;
    } else {
      rpr = K1_CONSUMERS / P; ro = tid / P; pos0 = tid % P; act = ro < rpr;
    }
    Acc<ST> acc[QM][TR::EPV][NB];
#pragma unroll
    for (int q = 0; q < QM; ++q)
#pragma unroll
      for (int e = 0; e < TR::EPV; ++e)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[q][e][b].zero();

    const int64_t first_i = c0 / pl.cpi;
    int64_t cur_i = -1;

    auto flush = [&](int64_t i_seg) {
      double contrib[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) contrib[b] = 0.0;
      if (act) {
#pragma unroll
        for (int q = 0; q < QM; ++q) {
          const int64_t pos = pos0 + (int64_t)q * K1_CONSUMERS;
          if (pos < P) {
#pragma unroll
            for (int e = 0; e < TR::EPV; ++e) {
              const int64_t k = pos * TR::EPV + e;
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                if constexpr (ST == GROM_F64) {
                  contrib[b] = fma(reinterpret_cast<const double*>(ureg)[b * np + k], acc[q][e][b].v, contrib[b]);
                } else if constexpr (ST == GROM_F32X2) {
                  const double uk = (double)reinterpret_cast<const float*>(ureg)[b * np + k] +
                                    (double)reinterpret_cast<const float*>(ureg)[(int64_t)NB * np + b * np + k];
                  contrib[b] = fma(uk, (double)acc[q][e][b].S + (double)acc[q][e][b].s, contrib[b]);
                } else {
                  contrib[b] = fma((double)reinterpret_cast<const float*>(ureg)[b * np + k], (double)acc[q][e][b].v,
                                   contrib[b]);
                }
                acc[q][e][b].zero();
              }
            }
          }
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        double v = contrib[b];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        contrib[b] = v;
      }
      if (lane == 0) {
        const int64_t seg = i_seg - first_i;
        double* dst = a.part + (((int64_t)blockIdx.x * pl.maxseg + seg) * (K1_CONSUMERS / 32) + warp) * NB;
#pragma unroll
        for (int b = 0; b < NB; ++b) dst[b] = contrib[b];
      }
    };

    // Each thread owns at most RMAX rows x QM positions of a chunk (the plan
    // caps the rows per chunk accordingly).  It copies them to registers and
    // releases the stage at once, so the ring refills while it computes.
    // Offsets inside a stage are 32-bit; chunks advance without divisions.
    constexpr int PLANES = (ST == GROM_F32X2) ? 2 : 1;
    constexpr int RMAX = k1_rmax(QM, PLANES);
    const int rowb = (int)row_bytes;
    const int t_off = (int)(ro * row_bytes + pos0 * 16);  // this thread's first vector in a stage
    const int t_step = (int)(rpr * row_bytes);             // next row of this thread
    const int plane_off = (int)(np * 4);                    // F32X2: lo plane
    const bool full_pos = act && (pos0 + (int64_t)(QM - 1) * K1_CONSUMERS < P);
    // rows of a full chunk held by this thread (other chunks: the last of a test index)
    int nrow_full = act ? ((int)pl.rpc - (int)ro + (int)rpr - 1) / (int)rpr : 0;
    if (nrow_full > RMAX) nrow_full = RMAX;
    if (nrow_full < 0) nrow_full = 0;
    (void)rowb;
    int64_t ci = c0 / pl.cpi, cj = c0 - ci * pl.cpi;
    int s = 0;
    uint32_t ph = 0;
    for (int64_t c = c0; c < c1; ++c) {
      const int64_t i = ci;
      const int j0 = (int)(cj * pl.rpc);
      const int rows = (int)(pl.m - j0 < pl.rpc ? pl.m - j0 : pl.rpc);
      if (++cj == pl.cpi) { cj = 0; ++ci; }
      if (i != cur_i) {
        if (cur_i >= 0) flush(cur_i);
        cur_i = i;
      }
      // warp-uniform: a lane whose wait timed out takes its whole warp along
      // (the flush shuffles need every lane)
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[s], ph, abort_flag))) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(a.err, DEV_ERR_TIMEOUT);
        }
        break;
      }
      const uint8_t* st = stages + s * K1_STAGE_BYTES + t_off;
      // rows of this chunk held by this thread
      int nrow;
      if constexpr (ST == GROM_F32X2) {
        // full chunks: the precomputed count
        nrow = nrow_full;
        if (rows != (int)pl.rpc) {
          nrow = act ? (rows - (int)ro + (int)rpr - 1) / (int)rpr : 0;
          if (nrow > RMAX) nrow = RMAX;
          if (nrow < 0) nrow = 0;
        }
      } else {
        nrow = act ? (rows - (int)ro + (int)rpr - 1) / (int)rpr : 0;
        if (nrow > RMAX) nrow = RMAX;
        if (nrow < 0) nrow = 0;
      }
      uint4 vec[RMAX][QM][PLANES];
      if (full_pos && nrow == RMAX) {
#pragma unroll
        for (int t = 0; t < RMAX; ++t)
#pragma unroll
          for (int q = 0; q < QM; ++q)
#pragma unroll
            for (int p2 = 0; p2 < PLANES; ++p2)
              vec[t][q][p2] = *reinterpret_cast<const uint4*>(st + t * t_step + q * (K1_CONSUMERS * 16) + p2 * plane_off);
      } else {
#pragma unroll
        for (int t = 0; t < RMAX; ++t)
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const bool ok = t < nrow && (pos0 + (int64_t)q * K1_CONSUMERS < P);
#pragma unroll
            for (int p2 = 0; p2 < PLANES; ++p2)
              vec[t][q][p2] = ok ? *reinterpret_cast<const uint4*>(st + t * t_step + q * (K1_CONSUMERS * 16) + p2 * plane_off)
                                 : make_uint4(0, 0, 0, 0);
          }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[s]);
      if (++s == K1_STAGES) { s = 0; ph ^= 1u; }
      // zero vectors of rows beyond nrow contribute nothing; u_j of such rows
      // is read at a clamped, valid index
      const int jt = j0 + (int)ro;
      ds_renorm_all<ST>(acc);
#pragma unroll
      for (int t = 0; t < RMAX; ++t) {
        if (t >= nrow) break;
        const int j = jt + t * (int)rpr;
        if constexpr (ST == GROM_F64) {
          double uj[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const double*>(mreg)[b * (int)mp + j];
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const double x0 = __hiloint2double((int)vec[t][q][0].y, (int)vec[t][q][0].x);
            const double x1 = __hiloint2double((int)vec[t][q][0].w, (int)vec[t][q][0].z);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              acc[q][0][b].v = fma(x0, uj[b], acc[q][0][b].v);
              acc[q][1][b].v = fma(x1, uj[b], acc[q][1][b].v);
            }
          }
        } else if constexpr (ST == GROM_F32X2) {
          float uh[NB], ul[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            uh[b] = reinterpret_cast<const float*>(mreg)[b * (int)mp + j];
            ul[b] = reinterpret_cast<const float*>(mreg)[(NB + b) * (int)mp + j];
          }
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const uint4 h = vec[t][q][0];
            const uint4 l = vec[t][q][PLANES - 1];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              ds_mac(__uint_as_float(h.x), __uint_as_float(l.x), uh[b], ul[b], acc[q][0][b].S, acc[q][0][b].s);
              ds_mac(__uint_as_float(h.y), __uint_as_float(l.y), uh[b], ul[b], acc[q][1][b].S, acc[q][1][b].s);
              ds_mac(__uint_as_float(h.z), __uint_as_float(l.z), uh[b], ul[b], acc[q][2][b].S, acc[q][2][b].s);
              ds_mac(__uint_as_float(h.w), __uint_as_float(l.w), uh[b], ul[b], acc[q][3][b].S, acc[q][3][b].s);
            }
          }
        } else if constexpr (ST == GROM_F32) {
          float uj[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const float*>(mreg)[b * (int)mp + j];
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const uint4 x = vec[t][q][0];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              acc[q][0][b].v = fmaf(__uint_as_float(x.x), uj[b], acc[q][0][b].v);
              acc[q][1][b].v = fmaf(__uint_as_float(x.y), uj[b], acc[q][1][b].v);
              acc[q][2][b].v = fmaf(__uint_as_float(x.z), uj[b], acc[q][2][b].v);
              acc[q][3][b].v = fmaf(__uint_as_float(x.w), uj[b], acc[q][3][b].v);
            }
          }
        } else {  // BF16
          float uj[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const float*>(mreg)[b * (int)mp + j];
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const uint32_t ws[4] = {vec[t][q][0].x, vec[t][q][0].y, vec[t][q][0].z, vec[t][q][0].w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float x0 = __uint_as_float(ws[h] << 16);
              const float x1 = __uint_as_float(ws[h] & 0xffff0000u);
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                acc[q][2 * h][b].v = fmaf(x0, uj[b], acc[q][2 * h][b].v);
                acc[q][2 * h + 1][b].v = fmaf(x1, uj[b], acc[q][2 * h + 1][b].v);
              }
            }
          }
        }
      }
    }
    if (cur_i >= 0 && !__any_sync(0xffffffffu, *abort_flag != 0)) flush(cur_i);
  }
  __syncthreads();
}

// Sums the per-warp partials of every test index in CTA order.
template <int NB>
__global__ void k1_finalize_kernel(const K1Plan pl, const K1Args a, const int b0) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = pl.n;
  if (idx >= n * a.nb) return;
  const int b = (int)(idx / n);
  const int64_t i = idx - (int64_t)b * n;
  const int bg = b0 + b;
  if (a.active && !a.active[bg]) return;
  const int64_t G = pl.grid, T = pl.T;
  // CTA that owns chunk c: the largest g with floor(g*T/G) <= c.
  auto owner = [&](int64_t c) { return ((c + 1) * G - 1) / T; };
  const int64_t g_lo = owner(i * pl.cpi), g_hi = owner((i + 1) * pl.cpi - 1);
  double s = 0.0;
  for (int64_t g = g_lo; g <= g_hi; ++g) {
    const int64_t first_i = (g * T / G) / pl.cpi;
    const double* src = a.part + ((g * pl.maxseg + (i - first_i)) * (K1_CONSUMERS / 32)) * NB + b;
#pragma unroll
    for (int w = 0; w < K1_CONSUMERS / 32; ++w) s += src[w * NB];
  }
  double* dst = a.taken ? a.hist + bg * a.hist_stride + (3 + a.taken[bg] % 3) * n : a.c + bg * a.c_stride;
  dst[i] = s;
}

template <int ST, int QM, int NB>
cudaError_t k1_launch_one(const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  auto kern = k1_stream_kernel<ST, QM, NB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if (a.ev0) prof_record(a.ev0, s);
  kern<<<pl.grid, K1_THREADS, pl.smem, s>>>(pl, a, b0);
  e = cudaGetLastError();
  if (e == cudaSuccess && a.ev1) e = prof_record(a.ev1, s);
  if (e != cudaSuccess) return e;
  if (a.skip_finalize) return cudaSuccess;
  const int64_t total = pl.n * a.nb;
  k1_finalize_kernel<NB><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pl, a, b0);
  return cudaGetLastError();
}

}  // namespace grom
