// K3D: the batched CP-form advection term (Sec. 3.1, eq. tc_ap; skew
// structure Sec. 3.3) of FP64 ROMs at FP64 tolerance on the FP32 pipe.
//
// GB300 issues about two FP64 FMAs per clock per SM against 128 FP32 ones,
// so the FP64 GEMMs of K3g run at ~1 TFLOP/s.  K3D keeps every operand as a
// double-single pair (ds_arith.cuh: hi = rn32(x), lo = rn32(x - hi), a
// 48-bit significand) and multiplies-adds with error-free transformations
// (ds_mac), renormalising every accumulator after each K tile so that the
// low word stays within an ulp of the high one (without it, the low word's
// own rounding error grows with K: 1.2e-12 instead of 1.5e-13 at N = R = 1024
// in a CPU emulation of this arithmetic).
// Per-evaluation error against exact FP64 arithmetic at N = R = 1024: ~1e-13.
//
//   prep:      the states of the batch as hi/lo planes (FP64 -> two floats).
//   project:   P = X V, Q = X W (and S = X U for the skew form), as
//              register-tiled double-single GEMMs over K splits; with one
//              split the epilogue forms H1 = P o Q, H2 = P o S itself.
//   hadamard:  (K splits) every (r, b) sums its splits' pairs in split
//              order and forms H1, H2 in double-single arithmetic.
//   expand:    c = H1 A^T (- H2 W^T) over K splits; with one split the FP64
//              result goes straight to the output or to the advection slot
//              of the history ring.
//   finish:    (K splits) every (b, i) sums its splits' pairs in order (when
//              stepping, the step kernel does this and writes the next
//              state's planes).
// Output tiles are 32 x 32, 2 x 2 per thread; several CTAs share an SM.
// Every operand tile is a run of whole rows of a plane laid out for it (the
// states and H as [k][b], the factors as [i][r] and, for the expansion,
// transposed [r][i] with the sign of W folded in), so it is copied into
// shared memory with 16-byte asynchronous copies, two stages deep: the next
// K tile lands while the current one is multiplied.  Planes are padded with
// zeros to whole tiles (batch and rank to 32, K to 16), so no copy needs a
// bound check.  The split sums run one thread per output over the whole GPU
// (a last-CTA reduction, one CTA summing a tile, set the time of small
// problems), in a fixed order (deterministic).
// The factor copies are made once, at create, from the FP64 panels.
#include <algorithm>

#include "ds_arith.cuh"
#include "grom_internal.h"
#include "cp_async.cuh"

namespace grom {

constexpr int D_BK = 16;          // K tile
constexpr int D_T = 32;           // output tile (both dimensions)
constexpr int D_MAX_SPLITS = 16;
constexpr int D_GROUP = 4;        // split partials in flight per thread in the split sums

static inline int64_t d_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct DDims {
  int64_t n, rp;  // modes; row pitch of the FP64 factor panels (the rank rounded up to 8)
  int64_t rq;     // rank rounded up to D_T: pitch of the factor copies, rows of H and the expansion's K
  int64_t kp;     // n rounded up to D_BK: rows of the factor copies and the state planes
  int64_t nq;     // n rounded up to D_T: pitch of the transposed factor copies
  int64_t bq;     // batch rounded up to D_T: pitch of the state planes, H and the projection partials
  int batch, nf;
};

struct DSplit {
  int ks;
  float* partial;  // ks x nf x 2 x rq x bq (project) or ks x 2 x batch x n (expand)
};

static DDims d_dims(int64_t n, int64_t rp, int batch, int nf) {
  return DDims{n, rp, d_up(rp, D_T), d_up(n, D_BK), d_up(n, D_T), d_up(batch, D_T), batch, nf};
}

// Factor copies: [fa | fb | fc] x [hi | lo], kp x rq each (zero past n and
// past the rank), then [fa^T | -fc^T] x [hi | lo], rq x nq each.
__host__ __device__ inline int64_t d_fplane(const DDims& d) { return d.kp * d.rq; }
__host__ __device__ inline int64_t d_tplane(const DDims& d) { return d.rq * d.nq; }

__global__ void k3d_build(const uint8_t* op, size_t panel_bytes, const DDims d, float* out) {
  const int64_t fpl = d_fplane(d), tpl = d_tplane(d);
  const int64_t total = 6 * fpl + 4 * tpl;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, r;
    int q, hl;
    double sgn = 1.0;
    if (t < 6 * fpl) {
      const int64_t plane = t / fpl, e = t - plane * fpl;
      q = (int)(plane / 2);
      hl = (int)(plane % 2);
      i = e / d.rq;
      r = e - i * d.rq;
    } else {
      const int64_t u = t - 6 * fpl, plane = u / tpl, e = u - plane * tpl;
      const int m = (int)(plane / 2);
      hl = (int)(plane % 2);
      q = m == 0 ? 0 : 2;
      sgn = m == 0 ? 1.0 : -1.0;
      r = e / d.nq;
      i = e - r * d.nq;
    }
    float h = 0.f, l = 0.f;
    if (i < d.n && r < d.rp) {
      const double* f = reinterpret_cast<const double*>(op + (size_t)q * panel_bytes);
      ds_split(sgn * f[i * d.rp + r], h, l);
    }
    out[t] = hl ? l : h;
  }
}

// The states of the batch as hi/lo planes [k][b], kp x bq each (zero past n,
// for padding columns and for inactive trajectories).
__global__ void k3d_prep(const DDims d, const K3Args a, float* xh) {
  const int64_t plane = d.kp * d.bq;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / d.bq;
    const int b = (int)(t - k * d.bq);
    float h = 0.f, l = 0.f;
    if (b < d.batch && k < d.n && (a.active == nullptr || a.active[b])) {
      const double* u = a.taken ? a.hist + b * a.hist_stride + (a.taken[b] % 3) * d.n : a.u + b * a.u_stride;
      ds_split(u[k], h, l);
    }
    xh[t] = h;
    xh[plane + t] = l;
  }
}

// Shared memory of one CTA: two stages of operand tiles, each [term][hi/lo]
// [16 k][32], reused after the main loop to transpose the epilogue's
// outputs.  NA terms of the row operand (states or H), NB of the column
// operand (factors).
template <int NA, int NB>
struct DSmem {
  float a[2][NA][2][D_BK][D_T];
  float b[2][NB][2][D_BK][D_T];
};

// One CTA's K range of a 32 x 32 output tile: for every term t,
// acc[t][x][y] += sum_k A[a_of(t)][k][2 ty + x] B[t][k][2 tx + y], with the
// tiles arriving by cp.async two stages deep.  load(stage, kt) issues this
// thread's copies of K tile kt; every thread commits one group per tile
// (possibly empty) so that the wait counts match.
template <int NA, int NB, int NT, typename Load, typename AOf>
__device__ __forceinline__ void d_mainloop(DSmem<NA, NB>& sm, int64_t kb0, int64_t kb1, Load load, AOf a_of,
                                           float (&S)[NT][2][2], float (&s)[NT][2][2], int tx, int ty) {
  if (kb0 < kb1) load(0, kb0);
  ptx::cp_async_commit();
  for (int64_t kt = kb0; kt < kb1; ++kt) {
    const int st = (int)((kt - kb0) & 1);
    if (kt + 1 < kb1) load(st ^ 1, kt + 1);
    ptx::cp_async_commit();
    ptx::cp_async_wait<1>();  // tile kt has landed (this thread's copies) ...
    __syncthreads();          // ... and every thread's
#pragma unroll 2  // (rolled, the accumulators would be copied back every k)
    for (int k = 0; k < D_BK; ++k) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int ta = a_of(t);
        const float2 ah = *reinterpret_cast<const float2*>(&sm.a[st][ta][0][k][ty * 2]);
        const float2 al = *reinterpret_cast<const float2*>(&sm.a[st][ta][1][k][ty * 2]);
        const float2 bh = *reinterpret_cast<const float2*>(&sm.b[st][t][0][k][tx * 2]);
        const float2 bl = *reinterpret_cast<const float2*>(&sm.b[st][t][1][k][tx * 2]);
        ds_mac(ah.x, al.x, bh.x, bl.x, S[t][0][0], s[t][0][0]);
        ds_mac(ah.x, al.x, bh.y, bl.y, S[t][0][1], s[t][0][1]);
        ds_mac(ah.y, al.y, bh.x, bl.x, S[t][1][0], s[t][1][0]);
        ds_mac(ah.y, al.y, bh.y, bl.y, S[t][1][1], s[t][1][1]);
      }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) ds_renorm(S[t][x][y], s[t][x][y]);
    __syncthreads();  // stage st is refilled by the next iteration's copies
  }
}

// Projections: rows b (the states, one term), columns r (NF factors in the
// order fb, fc, fa: P, Q, S).  Grid (rq / 32, bq / 32, ks).
template <int NF>
__global__ void __launch_bounds__(256, 4) k3d_project(const DDims d, const float* fc, const float* xh, float* hbuf,
                                                   const DSplit sp) {
  __shared__ __align__(16) DSmem<1, NF> sm;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t b0 = (int64_t)blockIdx.y * D_T, r0 = (int64_t)blockIdx.x * D_T;
  const int64_t fpl = d_fplane(d), xpl = d.kp * d.bq;
  float S[NF][2][2], s[NF][2][2];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) S[f][x][y] = s[f][x][y] = 0.f;
  // 16-byte chunk tid of a K tile's (hi, lo) pair of planes: plane tid / 128,
  // row (tid % 128) / 8, columns 4 (tid % 8) .. + 3
  const int hl = tid >> 7, kk = (tid & 127) >> 3, q4 = (tid & 7) * 4;
  auto load = [&](int st, int64_t kt) {
    const int64_t k = kt * D_BK + kk;
    ptx::cp_async16(&sm.a[st][0][hl][kk][q4], xh + hl * xpl + k * d.bq + b0 + q4);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int q = f == 0 ? 1 : f == 1 ? 2 : 0;  // fb, fc, fa
      ptx::cp_async16(&sm.b[st][f][hl][kk][q4], fc + (2 * q + hl) * fpl + k * d.rq + r0 + q4);
    }
  };
  const int64_t nk = d.kp / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  d_mainloop<1, NF, NF>(sm, kb0, kb1, load, [](int) { return 0; }, S, s, tx, ty);
  // epilogue through shared memory (the main loop ended on a barrier):
  // planes [q][r][b], q = H1h, H1l, H2h, H2l (one split) or the split's pairs
  constexpr int NQ = 2 * NF;
  static_assert(sizeof(float) * NQ * D_T * (D_T + 1) <= sizeof(DSmem<1, NF>), "epilogue buffer");
  float(*tp)[D_T][D_T + 1] = reinterpret_cast<float(*)[D_T][D_T + 1]>(&sm);
  int nq;
  if (sp.ks == 1) {
    nq = NF == 3 ? 4 : 2;
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int rl = tx * 2 + y, bl = ty * 2 + x;
        float h, l;
        ds_mul(S[0][x][y], s[0][x][y], S[1][x][y], s[1][x][y], h, l);
        tp[0][rl][bl] = h;
        tp[1][rl][bl] = l;
        if constexpr (NF == 3) {
          ds_mul(S[0][x][y], s[0][x][y], S[2][x][y], s[2][x][y], h, l);
          tp[2][rl][bl] = h;
          tp[3][rl][bl] = l;
        }
      }
  } else {
    nq = NQ;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          tp[2 * f][tx * 2 + y][ty * 2 + x] = S[f][x][y];
          tp[2 * f + 1][tx * 2 + y][ty * 2 + x] = s[f][x][y];
        }
  }
  __syncthreads();
  // rows of 32 b, coalesced; H planes rq x bq, partial planes likewise
  const int64_t plane = d.rq * d.bq;
  float* dst = sp.ks == 1 ? hbuf : sp.partial + (int64_t)blockIdx.z * NQ * plane;
  for (int e = tid; e < nq * D_T * D_T; e += 256) {
    const int q = e / (D_T * D_T), rl = (e / D_T) % D_T, bl = e % D_T;
    dst[q * plane + (r0 + rl) * d.bq + b0 + bl] = tp[q][rl][bl];
  }
}

// The projections' K splits summed in split order, one thread per (r, b),
// and H1 = P o Q, H2 = P o S formed from the sums.
template <int NF>
__global__ void __launch_bounds__(256) k3d_hadamard(const DDims d, const DSplit sp, float* hbuf) {
  const int64_t plane = d.rq * d.bq;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < plane; o += (int64_t)gridDim.x * blockDim.x) {
    float S[NF], s[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) S[f] = s[f] = 0.f;
#pragma unroll 1
    for (int z0 = 0; z0 < sp.ks; z0 += D_GROUP) {
      float w[D_GROUP][NF][2];
#pragma unroll
      for (int zz = 0; zz < D_GROUP; ++zz)
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (z0 + zz < sp.ks) {
            const float* src = sp.partial + (((int64_t)(z0 + zz) * NF + f) * 2) * plane + o;
            w[zz][f][0] = __ldcg(src);
            w[zz][f][1] = __ldcg(src + plane);
          }
#pragma unroll
      for (int zz = 0; zz < D_GROUP; ++zz)
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (z0 + zz < sp.ks) ds_add(S[f], s[f], w[zz][f][0], w[zz][f][1]);
    }
    float h, l;
    ds_mul(S[0], s[0], S[1], s[1], h, l);
    hbuf[o] = h;
    hbuf[plane + o] = l;
    if constexpr (NF == 3) {
      ds_mul(S[0], s[0], S[2], s[2], h, l);
      hbuf[2 * plane + o] = h;
      hbuf[3 * plane + o] = l;
    }
  }
}

// Expansion: rows b (H1, H2), columns i (fa^T, -fc^T), K = r.  Grid
// (nq / 32, bq / 32, ks).
template <int NM>
__global__ void __launch_bounds__(256) k3d_expand(const DDims d, const K3Args a, const float* fc, const float* hbuf,
                                                  const DSplit sp) {
  __shared__ __align__(16) DSmem<NM, NM> sm;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t b0 = (int64_t)blockIdx.y * D_T, i0 = (int64_t)blockIdx.x * D_T;
  const float* ft = fc + 6 * d_fplane(d);
  const int64_t tpl = d_tplane(d), hpl = d.rq * d.bq;
  float S[NM][2][2], s[NM][2][2];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) S[m][x][y] = s[m][x][y] = 0.f;
  const int hl = tid >> 7, kk = (tid & 127) >> 3, q4 = (tid & 7) * 4;
  auto load = [&](int st, int64_t kt) {
    const int64_t k = kt * D_BK + kk;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      ptx::cp_async16(&sm.a[st][m][hl][kk][q4], hbuf + (2 * m + hl) * hpl + k * d.bq + b0 + q4);
      ptx::cp_async16(&sm.b[st][m][hl][kk][q4], ft + (2 * m + hl) * tpl + k * d.nq + i0 + q4);
    }
  };
  const int64_t nk = d.rq / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  d_mainloop<NM, NM, NM>(sm, kb0, kb1, load, [](int t) { return t; }, S, s, tx, ty);
  // the two terms' sums (the second term's sign is in its factor copy)
  float T[2][2], t2[2][2];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      T[x][y] = S[0][x][y];
      t2[x][y] = s[0][x][y];
      if constexpr (NM == 2) ds_add(T[x][y], t2[x][y], S[1][x][y], s[1][x][y]);
    }
  const int64_t oplane = (int64_t)d.batch * d.n;
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const int b = (int)b0 + ty * 2 + x;
    if (b >= d.batch) continue;
    const bool on = a.active == nullptr || a.active[b];
    double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int64_t i = i0 + tx * 2 + y;
      if (i >= d.n) continue;
      if (sp.ks == 1) {
        if (on) dst[i] = (double)T[x][y] + (double)t2[x][y];
      } else {
        float* p = sp.partial + (int64_t)blockIdx.z * 2 * oplane + (int64_t)b * d.n + i;
        p[0] = T[x][y];
        p[oplane] = t2[x][y];
      }
    }
  }
}

// The expansion's K splits summed in split order, one thread per (b, i),
// into the output or the advection slot of the history ring (FP64).
__global__ void __launch_bounds__(256) k3d_finish(const DDims d, const K3Args a, const DSplit sp) {
  const int64_t oplane = (int64_t)d.batch * d.n;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < oplane; o += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(o / d.n);
    const int64_t i = o - (int64_t)b * d.n;
    if (a.active && !a.active[b]) continue;
    float S = 0.f, s = 0.f;
#pragma unroll 1
    for (int z0 = 0; z0 < sp.ks; z0 += D_GROUP) {
      float w[D_GROUP][2];
#pragma unroll
      for (int zz = 0; zz < D_GROUP; ++zz)
        if (z0 + zz < sp.ks) {
          const float* p = sp.partial + (int64_t)(z0 + zz) * 2 * oplane + o;
          w[zz][0] = __ldcg(p);
          w[zz][1] = __ldcg(p + oplane);
        }
#pragma unroll
      for (int zz = 0; zz < D_GROUP; ++zz)
        if (z0 + zz < sp.ks) ds_add(S, s, w[zz][0], w[zz][1]);
    }
    double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
    dst[i] = (double)S + (double)s;
  }
}

// K splits of one GEMM (M x N outputs in 32 x 32 tiles, K long, nf products
// per output): the count whose busiest SM has the least work, CTAs spreading
// evenly (the busiest SM runs ceil(CTAs / SMs) of them), with the split
// sums' reads and launch added; ties go to fewer splits.  (32 x 32 tiles,
// several CTAs to an SM, measured faster on GB300 than 64 x 64 tiles with
// one CTA per SM in every shape tried: N = 512-1024, 64-1024 trajectories.)
static int d_splits(int64_t m, int64_t n, int64_t K, int nf, int sm_count) {
  const int64_t nk = K / D_BK, tiles = (m / D_T) * (n / D_T);
  int best = 1;
  double best_us = 0.0;
  const int64_t kmax = std::min<int64_t>(nk, D_MAX_SPLITS);
  for (int64_t ks = 1; ks <= kmax; ++ks) {
    const int64_t busiest = (tiles * ks + sm_count - 1) / sm_count;
    const int64_t ktiles = (nk + ks - 1) / ks;
    // ~24 G double-single products per second per SM; the split sums read
    // ks x nf pairs per output at ~15 TB/s and take one more launch
    double us = (double)busiest * ktiles * D_T * D_T * nf * D_BK / 24.3e3;
    if (ks > 1) us += 2.0 + (double)ks * m * n * nf * 8.0 / 15e6;
    if (ks == 1 || us < best_us * 0.999) {
      best = (int)ks;
      best_us = us;
    }
  }
  return best;
}

// Scratch: [states hi/lo] [H1, H2 hi/lo] [project partials] [expand partials].
struct DLayout {
  int ks_p, ks_e;
  size_t x_bytes, h_bytes, pp_bytes, pe_bytes, total;
};

static size_t d_round(size_t b) { return (b + 255) / 256 * 256; }

static DLayout d_layout(const DDims& d, int sm_count) {
  DLayout L{};
  L.ks_p = d_splits(d.rq, d.bq, d.kp, d.nf, sm_count);      // columns r, rows b, K = n
  L.ks_e = d_splits(d.nq, d.bq, d.rq, d.nf - 1, sm_count);  // columns i, rows b, K = r (one or two terms)
  L.x_bytes = d_round(sizeof(float) * 2 * (size_t)d.kp * d.bq);
  L.h_bytes = d_round(sizeof(float) * 4 * (size_t)d.rq * d.bq);
  L.pp_bytes = L.ks_p > 1 ? d_round(sizeof(float) * (size_t)L.ks_p * d.nf * 2 * d.rq * d.bq) : 0;
  L.pe_bytes = L.ks_e > 1 ? d_round(sizeof(float) * (size_t)L.ks_e * 2 * d.batch * d.n) : 0;
  L.total = L.x_bytes + L.h_bytes + L.pp_bytes + L.pe_bytes;
  return L;
}

size_t k3d_factor_bytes(int64_t n, int64_t rp) {
  const DDims d = d_dims(n, rp, 1, 3);
  return sizeof(float) * (size_t)(6 * d_fplane(d) + 4 * d_tplane(d));
}

size_t k3d_scratch_bytes(int64_t n, int64_t rp, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = K3G_MIN_BATCH; b <= max_batch; ++b)
    for (int nf = 2; nf <= 3; ++nf) {  // the split counts depend on the form
      const DLayout L = d_layout(d_dims(n, rp, b, nf), sm_count);
      if (L.total > need) need = L.total;
    }
  return need;
}

cudaError_t k3d_build_factors(const uint8_t* op, size_t panel_bytes, int64_t n, int64_t rp, void* out,
                              cudaStream_t s) {
  // op holds the three FP64 panels (fa, fb, fc: n x rp each) panel_bytes apart
  const DDims d = d_dims(n, rp, 1, 3);
  const int64_t total = 6 * d_fplane(d) + 4 * d_tplane(d);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8192);
  k3d_build<<<blocks, 256, 0, s>>>(op, panel_bytes, d, static_cast<float*>(out));
  return cudaGetLastError();
}

static unsigned d_flat_blocks(int64_t count, int sm_count) {
  const int64_t b = (count + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 8 * (int64_t)sm_count));
}

struct DBufs {
  float *xh, *h, *pp, *pe;
};

static DBufs d_bufs(const DLayout& L, void* scratch) {
  uint8_t* base = static_cast<uint8_t*>(scratch);
  DBufs q;
  q.xh = reinterpret_cast<float*>(base);
  q.h = reinterpret_cast<float*>(base + L.x_bytes);
  q.pp = reinterpret_cast<float*>(base + L.x_bytes + L.h_bytes);
  q.pe = reinterpret_cast<float*>(base + L.x_bytes + L.h_bytes + L.pp_bytes);
  return q;
}

static void d_prep(const DDims& d, const K3Args& a, const DBufs& q, int sm_count, cudaStream_t s) {
  k3d_prep<<<d_flat_blocks(d.kp * d.bq, sm_count), 256, 0, s>>>(d, a, q.xh);
}

// project (+ split sums) and expand; with one expansion split the result is
// in the output or the ring, else in the expansion partials.
static void d_gemms(const DDims& d, const DLayout& L, const K3Args& a, const float* f, const DBufs& q, int sm_count,
                    cudaStream_t s) {
  const DSplit sp{L.ks_p, q.pp};
  const dim3 gp((unsigned)(d.rq / D_T), (unsigned)(d.bq / D_T), (unsigned)sp.ks);
  if (d.nf == 3)
    k3d_project<3><<<gp, 256, 0, s>>>(d, f, q.xh, q.h, sp);
  else
    k3d_project<2><<<gp, 256, 0, s>>>(d, f, q.xh, q.h, sp);
  if (sp.ks > 1) {
    const unsigned hb = d_flat_blocks(d.rq * d.bq, sm_count);
    if (d.nf == 3)
      k3d_hadamard<3><<<hb, 256, 0, s>>>(d, sp, q.h);
    else
      k3d_hadamard<2><<<hb, 256, 0, s>>>(d, sp, q.h);
  }
  const DSplit se{L.ks_e, q.pe};
  const dim3 ge((unsigned)(d.nq / D_T), (unsigned)(d.bq / D_T), (unsigned)se.ks);
  if (d.nf == 3)
    k3d_expand<2><<<ge, 256, 0, s>>>(d, a, f, q.h, se);
  else
    k3d_expand<1><<<ge, 256, 0, s>>>(d, a, f, q.h, se);
}

static DDims d_dims_of(const K3Plan& p, const K3Args& a, int batch) {
  return d_dims(p.n, p.rb, batch, a.form == GROM_FORM_CP_SKEW ? 3 : 2);
}

cudaError_t k3d_launch(const K3Plan& p, const K3Args& a, const void* factors, int batch, int max_batch,
                       void* scratch, int sm_count, cudaStream_t s) {
  (void)max_batch;
  const DDims d = d_dims_of(p, a, batch);
  const DLayout L = d_layout(d, sm_count);
  const DBufs q = d_bufs(L, scratch);
  d_prep(d, a, q, sm_count, s);
  d_gemms(d, L, a, static_cast<const float*>(factors), q, sm_count, s);
  if (L.ks_e > 1)
    k3d_finish<<<d_flat_blocks((int64_t)batch * d.n, sm_count), 256, 0, s>>>(d, a, DSplit{L.ks_e, q.pe});
  return cudaGetLastError();
}

cudaError_t k3d_launch_step(const K3Plan& p, const K3Args& a, const void* factors, int batch, void* scratch,
                            int sm_count, bool prep, const StepArgs& st, int step_index, cudaEvent_t ev0,
                            cudaEvent_t ev1, cudaStream_t s) {
  const DDims d = d_dims_of(p, a, batch);
  const DLayout L = d_layout(d, sm_count);
  const DBufs q = d_bufs(L, scratch);
  if (prep) d_prep(d, a, q, sm_count, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && ev0) e = prof_record(ev0, s);
  if (e != cudaSuccess) return e;
  d_gemms(d, L, a, static_cast<const float*>(factors), q, sm_count, s);
  e = cudaGetLastError();
  if (e == cudaSuccess && ev1) e = prof_record(ev1, s);
  if (e != cudaSuccess) return e;
  // the step kernel sums the expansion's splits and writes the next state's
  // planes [i][b] (pitch bq)
  K3TStepFuse f{};
  f.d2 = q.pe;
  f.s2 = L.ks_e;
  f.bp = batch;
  f.np = d.bq;
  f.xh = q.xh;
  f.xl = q.xh + d.kp * d.bq;
  if (f.s2 == 1) return step_diag_mc_k3d_launch(st, step_index, f, s);
  // with split sums to load, one element per thread (more threads in flight)
  StepArgs st1 = st;
  st1.ept = 1;
  st1.nblk = step_mc_blocks(d.n);
  return step_diag_mc_k3d_launch(st1, step_index, f, s);
}

}  // namespace grom
