// Persistent stepper of the G-ROM with the skew-packed tensor: many
// BDFk/EXTk steps (Sec. 2.2, eq. nse_d1) in one cooperative launch.
//
// Every CTA keeps the stage ring of the packed streaming kernel
// (k1_packed.cuh) and the same static share of the chunks.  Per step:
//   1. the consumer warps load u^l into shared memory and stream their
//      chunks (per-position accumulators, flush per test index, records of
//      the transposed term) and fold the records into their window;
//   2. grid barrier;
//   3. each CTA finalises and steps its own slice of test indices: the row
//      sums of every CTA covering i minus the windows of all CTAs at k = i
//      (one warp per test index, lanes over CTAs, fixed shuffle tree), then
//      the diagonal step of element i (FP64) and the energy/invariant
//      partial of the CTA;
//   4. grid barrier, after which the next u is complete.
// The producer warp does not take part in the barriers: the tensor does not
// depend on u, so it keeps streaming the next step's chunks into the ring
// while the consumers finalise, and the first stages of each step are
// already resident when they return.  Barriers are consumer-only (a named
// barrier inside the CTA, a counter across CTAs) and every wait gives up
// after the library's time limit.
#pragma once

#include "k1_packed.cuh"
#include "step_elem.cuh"

namespace grom {

struct K1PPArgs {
  unsigned int* bar;  // grid barrier word (zero at creation; each barrier adds 2^31 in total)
  double* red;        // grid x NB x 2 energy / invariant partials
  int nsteps;
};

// Grid barrier of the consumer warps (256 threads) of every CTA.
__device__ __forceinline__ bool k1pp_barrier(unsigned int* bar, int* err, volatile int* abort_flag, int* ok_sh) {
  ptx::named_sync(1, K1_CONSUMERS);
  if (threadIdx.x == 0) {
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, inc);
    int ok = 1;
    const uint64_t t0 = ptx::globaltimer();
    for (uint32_t spin = 0;; ++spin) {
      const unsigned int now = *reinterpret_cast<volatile unsigned int*>(bar);
      if ((now ^ old) & 0x80000000u) break;
      if ((spin & 255u) == 255u && ptx::globaltimer() - t0 > ptx::WAIT_LIMIT_NS) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        *abort_flag = 1;
        ok = 0;
        break;
      }
    }
    __threadfence();
    *ok_sh = ok;
  }
  ptx::named_sync(1, K1_CONSUMERS);
  return *ok_sh != 0;
}

template <int ST, int QM, int NB>
__global__ void __launch_bounds__(K1_THREADS, 1)
    k1pp_kernel(const K1Plan pl, const K1Args a, const StepArgs st, const K1PPArgs pp) {
  using TR = K1Traits<ST>;
  using RT = typename K1PRec<ST>::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + K1_STAGES * K1_STAGE_BYTES);
  uint64_t* empty = full + K1_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + K1_STAGES);
  uint8_t* ureg = reinterpret_cast<uint8_t*>(empty + K1_STAGES) + 16;
  __shared__ int fi_tab[STEP_PK_MAX_GRID];
  __shared__ double wpart[K1_CONSUMERS / 32][NB][2];
  __shared__ int ok_sh;
  __shared__ int64_t l0s[NB];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = pl.n, np = pl.np, lp = pl.lp, row_bytes = pl.row_bytes;
  const int G = gridDim.x;
  const int g = blockIdx.x;
  const int64_t T = pl.T;
  const int64_t c0 = (int64_t)g * T / G, c1 = ((int64_t)g + 1) * T / G;
  const int nb = a.nb;

  if (tid == 0) {
    for (int s = 0; s < K1_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], K1_CONSUMERS / 32);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  for (int q = tid; q < G; q += K1_THREADS) fi_tab[q] = (int)(((int64_t)q * T / G) / pl.cpi);
  if (tid < NB) l0s[tid] = tid < nb ? st.taken[tid] : 0;
  __syncthreads();

  if (warp == K1_CONSUMERS / 32) {
    // ------------------------------------------------ producer, all steps
    if (lane == 0) {
      int64_t it = 0;
      int s = 0;
      uint32_t ph = 0;
      bool stop = false;
      for (int step = 0; step < pp.nsteps && !stop; ++step) {
        int64_t i = c0 / pl.cpi, jc = c0 - i * pl.cpi;
        for (int64_t c = c0; c < c1; ++c, ++it) {
          if (it >= K1_STAGES && !ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            *abort_flag = 1;
            atomicOr(a.err, DEV_ERR_TIMEOUT);
            stop = true;
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
      }
      const int64_t issued = it;
      for (int64_t q = issued > K1_STAGES ? issued - K1_STAGES : 0; q < issued; ++q) {
        if (!ptx::mbar_wait(&full[q % K1_STAGES], (uint32_t)((q / K1_STAGES) & 1), nullptr))
          atomicOr(a.err, DEV_ERR_TIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int P = (int)(lp / TR::EPV);
    const int R = pl.rg;
    const int lgR = R == 4 ? 2 : (R == 2 ? 1 : 0);
    const int W = K1_CONSUMERS / R;
    const int ro = (tid >> 3) & (R - 1);
    const int pos0 = ((tid >> (3 + lgR)) << 3) + (tid & 7);
    const bool act = pos0 < P;
    const int64_t uplane = (int64_t)NB * np;
    const int64_t first_i = c0 / pl.cpi, last_i = (c1 - 1) / pl.cpi;
    const int64_t nseg = last_i - first_i + 1;
    constexpr int RMAX = k1_rmax(QM, (ST == GROM_F32X2) ? 2 : 1);
    constexpr int PLANES = (ST == GROM_F32X2) ? 2 : 1;
    const int t_off = (int)(ro * row_bytes + pos0 * 16);
    const int t_step = (int)(R * row_bytes);
    const int q_step = W * 16;
    const int plane_off = (int)(lp * 4);
    const bool full_pos = act && (pos0 + (QM - 1) * W < P);
    // rows of a full chunk held by this thread (other chunks: the last of a test index)
    int nrow_full = act ? ((int)pl.rpc - ro + R - 1) >> lgR : 0;
    if (nrow_full > RMAX) nrow_full = RMAX;
    if (nrow_full < 0) nrow_full = 0;
    const int64_t i_lo = (int64_t)g * n / G, i_hi = ((int64_t)g + 1) * n / G;  // owned test indices
    int s = 0;
    uint32_t ph = 0;

    for (int step = 0; step < pp.nsteps; ++step) {
      // ---- u^l of this step into shared memory (written by every CTA in the
      // previous step: read through L2)
      for (int64_t idx = tid; idx < (int64_t)NB * np; idx += K1_CONSUMERS) {
        const int b = (int)(idx / np);
        const int64_t k = idx - (int64_t)b * np;
        double v = 0.0;
        if (b < nb && k < n) v = __ldcg(a.hist + b * a.hist_stride + ((l0s[b] + step) % 3) * n + k);
        if constexpr (ST == GROM_F64) {
          reinterpret_cast<double*>(ureg)[idx] = v;
        } else if constexpr (ST == GROM_F32X2) {
          const float hv = __double2float_rn(v);
          reinterpret_cast<float*>(ureg)[idx] = hv;
          reinterpret_cast<float*>(ureg)[uplane + idx] = __double2float_rn(v - (double)hv);
        } else {
          reinterpret_cast<float*>(ureg)[idx] = __double2float_rn(v);
        }
      }
      ptx::named_sync(1, K1_CONSUMERS);

      // ---- stream this CTA's chunks (as k1_packed_kernel)
      Acc<ST> acc[QM][TR::EPV][NB];
#pragma unroll
      for (int q = 0; q < QM; ++q)
#pragma unroll
        for (int e = 0; e < TR::EPV; ++e)
#pragma unroll
          for (int b = 0; b < NB; ++b) acc[q][e][b].zero();
      int64_t cur_i = -1;
      auto flush = [&](int64_t i_seg) {
        double contrib[NB], ui[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          contrib[b] = 0.0;
          ui[b] = k1p_u<ST>(ureg, (int64_t)b * np + i_seg, uplane);
        }
        RT* rec = reinterpret_cast<RT*>(a.dg) + (((int64_t)g * pl.maxseg + (i_seg - first_i)) * NB) * lp;
#pragma unroll
        for (int q = 0; q < QM; ++q) {
          const int pos = pos0 + q * W;
#pragma unroll
          for (int e = 0; e < TR::EPV; ++e) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
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
          double* dst = a.part + (((int64_t)g * pl.maxseg + (i_seg - first_i)) * (K1_CONSUMERS / 32) + warp) * NB;
#pragma unroll
          for (int b = 0; b < NB; ++b) dst[b] = contrib[b];
        }
      };

      int64_t ci = c0 / pl.cpi, cj = c0 - ci * pl.cpi;
      bool stop = false;
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
        // (the flush shuffles and the named barriers need every lane)
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[s], ph, abort_flag))) {
          if (lane == 0) {
            *abort_flag = 1;
            atomicOr(a.err, DEV_ERR_TIMEOUT);
          }
          stop = true;
          break;
        }
        const uint8_t* stg = stages + s * K1_STAGE_BYTES + t_off;
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
                vec[t][q][p2] = *reinterpret_cast<const uint4*>(stg + t * t_step + q * q_step + p2 * plane_off);
        } else {
#pragma unroll
          for (int t = 0; t < RMAX; ++t)
#pragma unroll
            for (int q = 0; q < QM; ++q) {
              const bool ok = t < nrow && (pos0 + q * W < P);
#pragma unroll
              for (int p2 = 0; p2 < PLANES; ++p2)
                vec[t][q][p2] = ok ? *reinterpret_cast<const uint4*>(stg + t * t_step + q * q_step + p2 * plane_off)
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
            for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const double*>(ureg)[b * (int)np + j];
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
              uh[b] = reinterpret_cast<const float*>(ureg)[b * (int)np + j];
              ul[b] = reinterpret_cast<const float*>(ureg)[(NB + b) * (int)np + j];
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
            for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const float*>(ureg)[b * (int)np + j];
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
            for (int b = 0; b < NB; ++b) uj[b] = reinterpret_cast<const float*>(ureg)[b * (int)np + j];
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
      if (!stop && cur_i >= 0) flush(cur_i);
      // every consumer warp arrives here; thread 0 reads the abort flag (the
      // producer may set it at any time) and every consumer acts on that value
      ptx::named_sync(1, K1_CONSUMERS);
      if (tid == 0) ok_sh = *abort_flag ? 0 : 1;
      ptx::named_sync(1, K1_CONSUMERS);
      if (!ok_sh) break;

      // ---- fold the records of this step into this CTA's window
      {
        const RT* rec = reinterpret_cast<const RT*>(a.dg) + (int64_t)g * pl.maxseg * NB * lp;
        double* win = a.tg + (int64_t)g * NB * pl.lw;
        for (int64_t idx = tid; idx < (int64_t)NB * pl.lw; idx += K1_CONSUMERS) {
          const int b = (int)(idx / pl.lw);
          const int64_t w = idx - (int64_t)b * pl.lw;
          const int64_t s_lo = w - lp + 1 > 0 ? w - lp + 1 : 0;
          const int64_t s_hi = w < nseg - 1 ? w : nseg - 1;
          double t = 0.0;
          for (int64_t sg = s_lo; sg <= s_hi; ++sg) t += (double)rec[(sg * NB + b) * lp + (w - sg)];
          win[idx] = t;
        }
      }
      if (!k1pp_barrier(pp.bar, a.err, abort_flag, &ok_sh)) break;

      // ---- finalise and step the owned test indices (a warp per index)
      double ew[NB], iw[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) ew[b] = iw[b] = 0.0;
      int bad = 0;
      for (int64_t i = i_lo + warp; i < i_hi; i += K1_CONSUMERS / 32) {
        const int64_t g_lo = ((i * pl.cpi + 1) * G - 1) / T, g_hi = (((i + 1) * pl.cpi) * G - 1) / T;
        const int nrp = (int)(g_hi - g_lo + 1) * (K1_CONSUMERS / 32);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (b >= nb) break;
          double v = 0.0;
          for (int q = lane; q < nrp; q += 32) {  // row sums of the CTAs covering i
            const int64_t go = g_lo + q / (K1_CONSUMERS / 32);
            const int wq = q % (K1_CONSUMERS / 32);
            v += __ldcg(a.part + ((go * pl.maxseg + (i - fi_tab[go])) * (K1_CONSUMERS / 32) + wq) * NB + b);
          }
          for (int q = lane; q < G; q += 32) {  // transposed-term windows of every CTA at k = i
            int64_t w = i - fi_tab[q] - 1;
            if (w < 0) w += n;
            const double* win = a.tg + ((int64_t)q * NB + b) * pl.lw;
            for (; w < pl.lw; w += n) v -= __ldcg(win + w);
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == 0) {
            const int64_t l = l0s[b] + step;
            const int k = (int)(l + 1 < st.order ? l + 1 : st.order);
            double* h = st.hist + b * st.hist_stride;
            h[(3 + l % 3) * n + i] = v;
            double ep, ip;
            int bb;
            step_elem(st, h, n, l, k, i, v, ep, ip, bb);
            ew[b] += ep;
            iw[b] += ip;
            if (bb) {
              bad = 1;
              atomicMin(st.first_bad, b);
            }
          }
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          wpart[warp][b][0] = ew[b];
          wpart[warp][b][1] = iw[b];
        }
        if (bad) atomicOr(st.err, DEV_ERR_NONFINITE);
      }
      ptx::named_sync(1, K1_CONSUMERS);
      if (tid < NB) {
        double e = 0.0, v = 0.0;
        for (int w = 0; w < K1_CONSUMERS / 32; ++w) {
          e += wpart[w][tid][0];
          v += wpart[w][tid][1];
        }
        pp.red[((int64_t)g * NB + tid) * 2] = e;
        pp.red[((int64_t)g * NB + tid) * 2 + 1] = v;
      }
      if (!k1pp_barrier(pp.bar, a.err, abort_flag, &ok_sh)) break;

      // ---- energy / invariant of the step: warp b of CTA 0 sums the CTA
      // partials of trajectory b (lane q adds CTAs q, q+32, ... in order)
      if (g == 0 && warp < nb && warp < NB && (st.energy || st.invariant)) {
        double e = 0.0, v = 0.0;
        for (int q = lane; q < G; q += 32) {
          e += __ldcg(pp.red + ((int64_t)q * NB + warp) * 2);
          v += __ldcg(pp.red + ((int64_t)q * NB + warp) * 2 + 1);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          e += __shfl_xor_sync(0xffffffffu, e, off);
          v += __shfl_xor_sync(0xffffffffu, v, off);
        }
        if (lane == 0) {
          if (st.energy) st.energy[(int64_t)step * st.batch + warp] = 0.5 * e;
          if (st.invariant) st.invariant[(int64_t)step * st.batch + warp] = v;
        }
      }
    }
    // the step count of every trajectory, once all CTAs are done with it
    if (g == 0 && tid < nb && !*abort_flag) st.taken[tid] = l0s[tid] + pp.nsteps;
  }
  __syncthreads();
}

template <int ST, int QM, int NB>
cudaError_t k1pp_launch_one(const K1Plan& pl, const K1Args& a, const StepArgs& st, const K1PPArgs& pp, cudaStream_t s) {
  auto kern = k1pp_kernel<ST, QM, NB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K1_THREADS, pl.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  K1Plan plc = pl;
  K1Args ac = a;
  StepArgs stc = st;
  K1PPArgs ppc = pp;
  void* args[] = {&plc, &ac, &stc, &ppc};
  if (a.ev0) prof_record(a.ev0, s);
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(pl.grid), dim3(K1_THREADS), args, pl.smem, s);
  if (e == cudaSuccess && a.ev1) e = prof_record(a.ev1, s);
  return e;
}

}  // namespace grom
