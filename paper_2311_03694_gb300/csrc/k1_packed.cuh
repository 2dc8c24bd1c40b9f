// K1 on the skew-packed layout (GROM_LAYOUT_SKEW_PACKED), HBM streaming.
//
// For a tensor skew in its test and advected index (Sec. 3.2: C_ijk = -C_kji)
// every slice M^j_ik = C_ijk is a skew matrix, so
//   c_i = sum_k D_ik u_k   with   D = sum_j u_j M^j   (skew as well).
// Row (i, j) of the packed tensor holds M^j_{i,k} for k = i + 1 + p (mod n),
// p = 0 .. h-1 (h = n/2), which covers every unordered pair {i, k} once.
// Streaming the rows of test index i yields D_{i,k} per stored position p by
// the same per-position accumulation as the dense kernel.  The flush adds
// D_{i,k} u_k to c_i and records D_{i,k} u_i, the term that c_k receives with
// a minus sign (D_ki = -D_ik).  After its last chunk each CTA folds its
// records into one window over k (window index w = k - first test index - 1,
// mod n), and the finalize subtracts the windows of all CTAs from the row
// sums.  Every sum runs in a fixed order, so results are deterministic.
//
// Thread mapping: a stored row is a sequence of 16-byte vectors (positions).
// A quarter warp covers 8 consecutive positions of one row (conflict-free
// shared loads), and the rg row groups that share a position sit in one
// warp, 8 lanes apart, so their partial D values combine with at most two
// shuffles at the flush.  Bytes and multiply-adds are half the dense ones.
#pragma once

#include "k1_stream.cuh"

namespace grom {

// Precision of the recorded values D_{i,k} u_i.
template <int ST>
struct K1PRec {
  using T = float;
};
template <>
struct K1PRec<GROM_F64> {
  using T = double;
};
template <>
struct K1PRec<GROM_F32X2> {
  using T = double;
};

// u (as stored in shared memory for this storage type) at index idx of the
// pass; `plane` is the offset of the F32X2 lo plane in floats.
template <int ST>
__device__ __forceinline__ double k1p_u(const uint8_t* ureg, int64_t idx, int64_t plane) {
  if constexpr (ST == GROM_F64) {
    return reinterpret_cast<const double*>(ureg)[idx];
  } else if constexpr (ST == GROM_F32X2) {
    return (double)reinterpret_cast<const float*>(ureg)[idx] + (double)reinterpret_cast<const float*>(ureg)[plane + idx];
  } else {
    return (double)reinterpret_cast<const float*>(ureg)[idx];
  }
}

template <int ST, int QM, int NB>
__global__ void __launch_bounds__(K1_THREADS, 1) k1_packed_kernel(const K1Plan pl, const K1Args a, const int b0) {
  using TR = K1Traits<ST>;
  using RT = typename K1PRec<ST>::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + K1_STAGES * K1_STAGE_BYTES);
  uint64_t* empty = full + K1_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + K1_STAGES);
  uint8_t* ureg = reinterpret_cast<uint8_t*>(empty + K1_STAGES) + 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = pl.n, np = pl.np, lp = pl.lp, row_bytes = pl.row_bytes;
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
  // weights (u itself for the G-ROM), in the arithmetic type of the storage;
  // F32X2 keeps a hi and a lo plane.
  const uint8_t* mreg;
  int64_t mp;
  k1_load_state<ST, NB>(pl, a, b0, ureg, mreg, mp);
  __syncthreads();

  if (warp == K1_CONSUMERS / 32) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t it = 0;
      int64_t i = c0 / pl.cpi, jc = c0 - i * pl.cpi;
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
      const int64_t issued = it;
      for (int64_t q = issued > K1_STAGES ? issued - K1_STAGES : 0; q < issued; ++q) {
        if (!ptx::mbar_wait(&full[q % K1_STAGES], (uint32_t)((q / K1_STAGES) & 1), nullptr))
          atomicOr(a.err, DEV_ERR_TIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int P = (int)(lp / TR::EPV);  // positions per stored row
    const int R = pl.rg;                // row groups sharing a position
    const int lgR = R == 4 ? 2 : (R == 2 ? 1 : 0);
    const int W = K1_CONSUMERS / R;     // positions per q-slab
    const int ro = (tid >> 3) & (R - 1);
    const int pos0 = ((tid >> (3 + lgR)) << 3) + (tid & 7);
    const bool act = pos0 < P;
    const int64_t uplane = (int64_t)NB * np;

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
      double contrib[NB], ui[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        contrib[b] = 0.0;
        ui[b] = k1p_u<ST>(ureg, (int64_t)b * np + i_seg, uplane);
      }
      RT* rec = reinterpret_cast<RT*>(a.dg) + (((int64_t)blockIdx.x * pl.maxseg + (i_seg - first_i)) * NB) * lp;
#pragma unroll
      for (int q = 0; q < QM; ++q) {
        const int pos = pos0 + q * W;
#pragma unroll
        for (int e = 0; e < TR::EPV; ++e) {
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            // D_{i,k} of this position: the partials of the R row groups
            double v;
            if constexpr (ST == GROM_BF16 || ST == GROM_F32) {
              float f = acc[q][e][b].v;
              if (R >= 2) f += __shfl_xor_sync(0xffffffffu, f, 8);
              if (R >= 4) f += __shfl_xor_sync(0xffffffffu, f, 16);
              v = (double)f;
            } else {
              double d;
              if constexpr (ST == GROM_F64) {
                d = acc[q][e][b].v;
              } else {
                d = (double)acc[q][e][b].S + (double)acc[q][e][b].s;
              }
              if (R >= 2) d += __shfl_xor_sync(0xffffffffu, d, 8);
              if (R >= 4) d += __shfl_xor_sync(0xffffffffu, d, 16);
              v = d;
            }
            acc[q][e][b].zero();
            if (ro == 0 && pos < P) {
              const int64_t p = (int64_t)pos * TR::EPV + e;
              double rv = 0.0;
              if (p < pl.h) {
                int64_t k = i_seg + 1 + p;
                if (k >= n) k -= n;
                contrib[b] = fma(k1p_u<ST>(ureg, (int64_t)b * np + k, uplane), v, contrib[b]);
                rv = v * ui[b];
              }
              rec[(int64_t)b * lp + p] = (RT)rv;
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

    // Each thread holds at most RMAX rows x QM positions of a chunk in
    // registers and releases the stage at once (as in the dense kernel).
    constexpr int RMAX = k1_rmax(QM, (ST == GROM_F32X2) ? 2 : 1);
    constexpr int PLANES = (ST == GROM_F32X2) ? 2 : 1;
    const int t_off = (int)(ro * row_bytes + pos0 * 16);
    const int t_step = (int)(R * row_bytes);
    const int q_step = W * 16;
    const int plane_off = (int)(lp * 4);  // F32X2: lo plane of a stored row
    const bool full_pos = act && (pos0 + (QM - 1) * W < P);
    // rows of a full chunk held by this thread (other chunks: the last of a test index)
    int nrow_full = act ? ((int)pl.rpc - ro + R - 1) >> lgR : 0;
    if (nrow_full > RMAX) nrow_full = RMAX;
    if (nrow_full < 0) nrow_full = 0;
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
      int nrow;
      if constexpr (ST == GROM_F32X2) {
        // full chunks: the precomputed count
        nrow = nrow_full;
        if (rows != (int)pl.rpc) {
          nrow = act ? (rows - ro + R - 1) >> lgR : 0;
          if (nrow > RMAX) nrow = RMAX;
          if (nrow < 0) nrow = 0;
        }
      } else {
        // (the precomputed count measured 6 % slower here for BF16 on GB300)
        nrow = act ? (rows - ro + R - 1) / R : 0;
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
              vec[t][q][p2] = *reinterpret_cast<const uint4*>(st + t * t_step + q * q_step + p2 * plane_off);
      } else {
#pragma unroll
        for (int t = 0; t < RMAX; ++t)
#pragma unroll
          for (int q = 0; q < QM; ++q) {
            const bool ok = t < nrow && (pos0 + q * W < P);
#pragma unroll
            for (int p2 = 0; p2 < PLANES; ++p2)
              vec[t][q][p2] = ok ? *reinterpret_cast<const uint4*>(st + t * t_step + q * q_step + p2 * plane_off)
                                 : make_uint4(0, 0, 0, 0);
          }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[s]);
      if (++s == K1_STAGES) { s = 0; ph ^= 1u; }
      const int jt = j0 + ro;
      ds_renorm_all<ST>(acc);
#pragma unroll
      for (int t = 0; t < RMAX; ++t) {
        if (t >= nrow) break;
        const int j = jt + t * R;
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
            const uint4 hv = vec[t][q][0];
            const uint4 lv = vec[t][q][PLANES - 1];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              ds_mac(__uint_as_float(hv.x), __uint_as_float(lv.x), uh[b], ul[b], acc[q][0][b].S, acc[q][0][b].s);
              ds_mac(__uint_as_float(hv.y), __uint_as_float(lv.y), uh[b], ul[b], acc[q][1][b].S, acc[q][1][b].s);
              ds_mac(__uint_as_float(hv.z), __uint_as_float(lv.z), uh[b], ul[b], acc[q][2][b].S, acc[q][2][b].s);
              ds_mac(__uint_as_float(hv.w), __uint_as_float(lv.w), uh[b], ul[b], acc[q][3][b].S, acc[q][3][b].s);
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
            for (int hh = 0; hh < 4; ++hh) {
              const float x0 = __uint_as_float(ws[hh] << 16);
              const float x1 = __uint_as_float(ws[hh] & 0xffff0000u);
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                acc[q][2 * hh][b].v = fmaf(x0, uj[b], acc[q][2 * hh][b].v);
                acc[q][2 * hh + 1][b].v = fmaf(x1, uj[b], acc[q][2 * hh + 1][b].v);
              }
            }
          }
        }
      }
    }
    if (cur_i >= 0 && !__any_sync(0xffffffffu, *abort_flag != 0)) flush(cur_i);
  }
  __syncthreads();
  if (*abort_flag) return;

  // Fold the records of this CTA into its window over k: the record of
  // segment sg at position p belongs to k = first_i + 1 + (sg + p) (mod n).
  const int64_t first_i = c0 / pl.cpi, last_i = (c1 - 1) / pl.cpi;
  const int64_t nseg = last_i - first_i + 1;
  const RT* rec = reinterpret_cast<const RT*>(a.dg) + (int64_t)blockIdx.x * pl.maxseg * NB * lp;
  double* win = a.tg + (int64_t)blockIdx.x * NB * pl.lw;
  for (int64_t idx = tid; idx < (int64_t)NB * pl.lw; idx += K1_THREADS) {
    const int b = (int)(idx / pl.lw);
    const int64_t w = idx - (int64_t)b * pl.lw;
    const int64_t s_lo = w - lp + 1 > 0 ? w - lp + 1 : 0;
    const int64_t s_hi = w < nseg - 1 ? w : nseg - 1;
    double t = 0.0;
    for (int64_t sg = s_lo; sg <= s_hi; ++sg) t += (double)rec[(sg * NB + b) * lp + (w - sg)];
    win[idx] = t;
  }
}

// c_i = (row sums of test index i) - (windows of every CTA at k = i), both in
// CTA order.  One block covers 32 test indices of one trajectory; warp w
// reads the windows of CTAs [w G/32, (w+1) G/32), with the CTAs' first test
// indices tabulated in shared memory.
constexpr int K1P_FIN_THREADS = 1024;
constexpr int K1P_FIN_MAX_GRID = 1024;

template <int NB>
__global__ void __launch_bounds__(K1P_FIN_THREADS) k1p_finalize_kernel(const K1Plan pl, const K1Args a, const int b0) {
  __shared__ double sh[32][33];
  __shared__ int fi_tab[K1P_FIN_MAX_GRID];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = pl.n;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const int bl = blockIdx.y;
  const int bg = b0 + bl;
  if (bl >= a.nb || (a.active && !a.active[bg])) return;  // uniform over the block
  const int G = pl.grid;
  const int64_t T = pl.T;
  for (int g = threadIdx.x; g < G; g += blockDim.x) fi_tab[g] = (int)(((int64_t)g * T / G) / pl.cpi);
  __syncthreads();
  double s = 0.0;
  if (i < n) {
    const int g0 = warp * G / 32, g1 = (warp + 1) * G / 32;
    for (int g = g0; g < g1; ++g) {
      int64_t w = i - fi_tab[g] - 1;
      if (w < 0) w += n;
      const double* win = a.tg + ((int64_t)g * NB + bl) * pl.lw;
      for (; w < pl.lw; w += n) s += win[w];
    }
  }
  sh[warp][lane] = s;
  double rs = 0.0;
  if (warp == 0 && i < n) {
    const int64_t g_lo = ((i * pl.cpi + 1) * G - 1) / T, g_hi = (((i + 1) * pl.cpi) * G - 1) / T;
    for (int64_t g = g_lo; g <= g_hi; ++g) {
      const double* src = a.part + ((g * pl.maxseg + (i - fi_tab[g])) * (K1_CONSUMERS / 32)) * NB + bl;
#pragma unroll
      for (int w = 0; w < K1_CONSUMERS / 32; ++w) rs += src[w * NB];
    }
  }
  __syncthreads();
  if (warp == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 32; ++w) t += sh[w][lane];
    double* dst = a.taken ? a.hist + bg * a.hist_stride + (3 + a.taken[bg] % 3) * n : a.c + bg * a.c_stride;
    dst[i] = rs - t;
  }
}

template <int ST, int QM, int NB>
cudaError_t k1p_launch_one(const K1Plan& pl, const K1Args& a, int b0, cudaStream_t s) {
  auto kern = k1_packed_kernel<ST, QM, NB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if (a.ev0) prof_record(a.ev0, s);
  kern<<<pl.grid, K1_THREADS, pl.smem, s>>>(pl, a, b0);
  e = cudaGetLastError();
  if (e == cudaSuccess && a.ev1) e = prof_record(a.ev1, s);
  if (e != cudaSuccess) return e;
  if (a.skip_finalize) return cudaSuccess;
  if (pl.grid > K1P_FIN_MAX_GRID) return cudaErrorInvalidValue;
  k1p_finalize_kernel<NB><<<dim3((unsigned)((pl.n + 31) / 32), (unsigned)a.nb), K1P_FIN_THREADS, 0, s>>>(pl, a, b0);
  return cudaGetLastError();
}

}  // namespace grom
