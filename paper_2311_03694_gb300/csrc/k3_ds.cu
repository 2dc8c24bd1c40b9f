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
//   project:   P = X V, Q = X W (and S = X U for the skew form), B x rp, as
//              register-tiled double-single GEMMs over K splits; with one
//              split the epilogue forms H1 = P o Q, H2 = P o S itself.
//   hadamard:  (K splits) every (b, r) sums its splits' pairs in split
//              order and forms H1, H2 in double-single arithmetic.
//   expand:    c = H1 A^T (- H2 W^T), B x n, over K splits; with one split
//              the FP64 result goes straight to the output or to the
//              advection slot of the history ring.
//   finish:    (K splits) every (b, i) sums its splits' pairs in order.
// Output tiles are 32 x 32, 2 x 2 per thread.  The split sums run one thread
// per output over the whole GPU: a last-CTA reduction (one CTA summing a
// whole tile, one output per thread and round trip) set the time of small
// problems.  Every sum is in a fixed order (deterministic).
// The factors' hi/lo copies are made once, at create, from the FP64 panels.
#include <algorithm>

#include "ds_arith.cuh"
#include "grom_internal.h"

namespace grom {

constexpr int D_BK = 16;
constexpr int D_MAX_SPLITS = 16;
constexpr int D_GROUP = 4;  // split partials in flight per thread in the split sums

struct DDims {
  int64_t n, rp, kp;  // modes, padded rank (factor row pitch), state row pitch (n rounded up to D_BK)
  int batch, nf;
};

struct DSplit {
  int ks;
  float* partial;  // ks x nf x 2 x batch x rp (project) or ks x 2 x batch x n (expand)
};

// One FP64 factor panel (count doubles) -> its hi and lo planes.
__global__ void k3d_split_panel(const double* f, int64_t count, float* hi, float* lo) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (int64_t)gridDim.x * blockDim.x)
    ds_split(f[idx], hi[idx], lo[idx]);
}

// The states of the batch as hi/lo planes, batch x kp each (zero past n and
// for inactive trajectories).
__global__ void k3d_prep(const DDims d, const K3Args a, float* xh) {
  const int b = blockIdx.y;
  const bool on = b < d.batch && (a.active == nullptr || a.active[b]);
  const double* u = on ? (a.taken ? a.hist + b * a.hist_stride + (a.taken[b] % 3) * d.n : a.u + b * a.u_stride)
                       : nullptr;
  float* xl = xh + (int64_t)d.batch * d.kp;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.kp; k += (int64_t)gridDim.x * blockDim.x) {
    float h = 0.f, l = 0.f;
    if (on && k < d.n) ds_split(u[k], h, l);
    xh[(int64_t)b * d.kp + k] = h;
    xl[(int64_t)b * d.kp + k] = l;
  }
}

// One K tile (16) of a TB x TC output tile, TB = TC = 16 MT, 256 threads as
// 16 x 16, each owning MT x MT outputs of every term.  The operand tiles are
// staged in shared memory as hi/lo planes [k][b] and [k][column].
template <int NF, int MT>
__global__ void __launch_bounds__(256) k3d_project(const DDims d, const float* fhl, const float* xh, float* hbuf,
                                                   const DSplit sp) {
  constexpr int TB = 16 * MT, TR = 16 * MT;
  __shared__ __align__(16) float Us[2][D_BK][TB + 4];
  __shared__ __align__(16) float Xs[NF][2][D_BK][TR + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * TB;
  const int64_t r0 = (int64_t)blockIdx.x * TR;
  const int64_t fplane = d.n * d.rp;
  // factor q (0 = fa, 1 = fb, 2 = fc) hi plane at fhl + 2 q fplane, lo plane after it;
  // projections in the order (fb, fc, fa): P, Q, S
  const int fq[3] = {1, 2, 0};
  const float* xl = xh + (int64_t)d.batch * d.kp;
  float S[NF][MT][MT], s[NF][MT][MT];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
      for (int y = 0; y < MT; ++y) S[f][x][y] = s[f][x][y] = 0.f;
  const int64_t nk = (d.n + D_BK - 1) / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * D_BK; k0 < kb1 * D_BK; k0 += D_BK) {
    // states: TB rows of 16 k as float4 (k < kp always: kp is n rounded up to D_BK, zero past n)
    for (int e = tid; e < TB * 4; e += 256) {
      const int lb = e >> 2, li = (e & 3) * 4;
      const int b = b0 + lb;
      float4 vh = make_float4(0.f, 0.f, 0.f, 0.f), vl = vh;
      if (b < d.batch) {
        vh = *reinterpret_cast<const float4*>(xh + (int64_t)b * d.kp + k0 + li);
        vl = *reinterpret_cast<const float4*>(xl + (int64_t)b * d.kp + k0 + li);
      }
      Us[0][li][lb] = vh.x; Us[0][li + 1][lb] = vh.y; Us[0][li + 2][lb] = vh.z; Us[0][li + 3][lb] = vh.w;
      Us[1][li][lb] = vl.x; Us[1][li + 1][lb] = vl.y; Us[1][li + 2][lb] = vl.z; Us[1][li + 3][lb] = vl.w;
    }
    // factors: 16 rows i of TR columns as float4 (rp is a multiple of 8, so a
    // group of four columns is wholly inside or wholly outside)
    for (int e = tid; e < 4 * TR; e += 256) {
      const int xi = e / (TR / 4), xr = (e % (TR / 4)) * 4;
      const int64_t i = k0 + xi, r = r0 + xr;
      const bool ok = i < d.n && r < d.rp;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* fh = fhl + 2 * fq[f] * fplane + i * d.rp + r;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(&Xs[f][0][xi][xr]) = ok ? *reinterpret_cast<const float4*>(fh) : z;
        *reinterpret_cast<float4*>(&Xs[f][1][xi][xr]) = ok ? *reinterpret_cast<const float4*>(fh + fplane) : z;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < D_BK; ++k) {
      float uh[MT], ul[MT];
#pragma unroll
      for (int x = 0; x < MT; ++x) {
        uh[x] = Us[0][k][ty * MT + x];
        ul[x] = Us[1][k][ty * MT + x];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        float vh[MT], vl[MT];
#pragma unroll
        for (int y = 0; y < MT; ++y) {
          vh[y] = Xs[f][0][k][tx * MT + y];
          vl[y] = Xs[f][1][k][tx * MT + y];
        }
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
          for (int y = 0; y < MT; ++y) ds_mac(uh[x], ul[x], vh[y], vl[y], S[f][x][y], s[f][x][y]);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) ds_renorm(S[f][x][y], s[f][x][y]);
    __syncthreads();
  }
  const int64_t plane = (int64_t)d.batch * d.rp;
#pragma unroll
  for (int x = 0; x < MT; ++x) {
    const int b = b0 + ty * MT + x;
    if (b >= d.batch) continue;
#pragma unroll
    for (int y = 0; y < MT; ++y) {
      const int64_t r = r0 + tx * MT + y;
      if (r >= d.rp) continue;
      const int64_t o = (int64_t)b * d.rp + r;
      if (sp.ks == 1) {
        // H1 = P o Q and H2 = P o S as hi/lo planes: hbuf = [H1h | H1l | H2h | H2l], batch x rp each
        float h, l;
        ds_mul(S[0][x][y], s[0][x][y], S[1][x][y], s[1][x][y], h, l);
        hbuf[o] = h;
        hbuf[plane + o] = l;
        if constexpr (NF == 3) {
          ds_mul(S[0][x][y], s[0][x][y], S[2][x][y], s[2][x][y], h, l);
          hbuf[2 * plane + o] = h;
          hbuf[3 * plane + o] = l;
        }
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          float* dst = sp.partial + (((int64_t)blockIdx.z * NF + f) * 2) * plane + o;
          dst[0] = S[f][x][y];
          dst[plane] = s[f][x][y];
        }
      }
    }
  }
}

// The projections' K splits summed in split order, one thread per (b, r),
// and H1 = P o Q, H2 = P o S formed from the sums.
template <int NF>
__global__ void __launch_bounds__(256) k3d_hadamard(const DDims d, const DSplit sp, float* hbuf) {
  const int64_t plane = (int64_t)d.batch * d.rp;
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

template <int NM, int MT>
__global__ void __launch_bounds__(256) k3d_expand(const DDims d, const K3Args a, const float* fhl, const float* hbuf,
                                                  const DSplit sp) {
  constexpr int TB = 16 * MT, TI = 16 * MT;
  __shared__ __align__(16) float Hs[NM][2][D_BK][TB + 4];  // [term][hi/lo][r][b]
  __shared__ __align__(16) float As[NM][2][D_BK][TI + 4];  // [term][hi/lo][r][i]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * TB;
  const int64_t i0 = (int64_t)blockIdx.x * TI;
  const int64_t fplane = d.n * d.rp;
  const int64_t plane = (int64_t)d.batch * d.rp;
  // first term: A (fa); second (skew form): -W (fc)
  const float* Fm[2] = {fhl, fhl + 4 * fplane};
  float S[MT][MT], s[MT][MT];
#pragma unroll
  for (int x = 0; x < MT; ++x)
#pragma unroll
    for (int y = 0; y < MT; ++y) S[x][y] = s[x][y] = 0.f;
  const int64_t nk = (d.rp + D_BK - 1) / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * D_BK; k0 < kb1 * D_BK; k0 += D_BK) {
    // rows b of H and rows i of the factor, 16 r each as float4 (rp is a
    // multiple of 8 and k0 of 16: a group of four is wholly inside or outside)
    for (int e = tid; e < TB * 4; e += 256) {
      const int lb = e >> 2, lr = (e & 3) * 4;
      const int b = b0 + lb;
      const int64_t r = k0 + lr;
      const bool ok = b < d.batch && r < d.rp;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const float* hh = hbuf + 2 * m * plane + (int64_t)b * d.rp + r;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 vh = ok ? __ldcg(reinterpret_cast<const float4*>(hh)) : z;
        const float4 vl = ok ? __ldcg(reinterpret_cast<const float4*>(hh + plane)) : z;
        Hs[m][0][lr][lb] = vh.x; Hs[m][0][lr + 1][lb] = vh.y; Hs[m][0][lr + 2][lb] = vh.z; Hs[m][0][lr + 3][lb] = vh.w;
        Hs[m][1][lr][lb] = vl.x; Hs[m][1][lr + 1][lb] = vl.y; Hs[m][1][lr + 2][lb] = vl.z; Hs[m][1][lr + 3][lb] = vl.w;
      }
    }
    for (int e = tid; e < TI * 4; e += 256) {
      const int ai = e >> 2, ar = (e & 3) * 4;
      const int64_t i = i0 + ai, r = k0 + ar;
      const bool ok = i < d.n && r < d.rp;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const float sgn = m == 0 ? 1.f : -1.f;
        const float* fm = Fm[m] + i * d.rp + r;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 vh = ok ? *reinterpret_cast<const float4*>(fm) : z;
        const float4 vl = ok ? *reinterpret_cast<const float4*>(fm + fplane) : z;
        As[m][0][ar][ai] = sgn * vh.x; As[m][0][ar + 1][ai] = sgn * vh.y;
        As[m][0][ar + 2][ai] = sgn * vh.z; As[m][0][ar + 3][ai] = sgn * vh.w;
        As[m][1][ar][ai] = sgn * vl.x; As[m][1][ar + 1][ai] = sgn * vl.y;
        As[m][1][ar + 2][ai] = sgn * vl.z; As[m][1][ar + 3][ai] = sgn * vl.w;
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NM; ++m) {
#pragma unroll 1
      for (int k = 0; k < D_BK; ++k) {
        float hh[MT], hl[MT], ah[MT], al[MT];
#pragma unroll
        for (int x = 0; x < MT; ++x) {
          hh[x] = Hs[m][0][k][ty * MT + x];
          hl[x] = Hs[m][1][k][ty * MT + x];
        }
#pragma unroll
        for (int y = 0; y < MT; ++y) {
          ah[y] = As[m][0][k][tx * MT + y];
          al[y] = As[m][1][k][tx * MT + y];
        }
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
          for (int y = 0; y < MT; ++y) ds_mac(hh[x], hl[x], ah[y], al[y], S[x][y], s[x][y]);
      }
#pragma unroll
      for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) ds_renorm(S[x][y], s[x][y]);
    }
    __syncthreads();
  }
  const int64_t oplane = (int64_t)d.batch * d.n;
#pragma unroll
  for (int x = 0; x < MT; ++x) {
    const int b = b0 + ty * MT + x;
    if (b >= d.batch) continue;
    const bool on = a.active == nullptr || a.active[b];
    double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
#pragma unroll
    for (int y = 0; y < MT; ++y) {
      const int64_t i = i0 + tx * MT + y;
      if (i >= d.n) continue;
      if (sp.ks == 1) {
        if (on) dst[i] = (double)S[x][y] + (double)s[x][y];
      } else {
        float* p = sp.partial + (int64_t)blockIdx.z * 2 * oplane + (int64_t)b * d.n + i;
        p[0] = S[x][y];
        p[oplane] = s[x][y];
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

// Tiles and K splits of one GEMM (M x N outputs, K long, nf products per
// output).  Tiles are 32 x 32 (D_MT = 2): several CTAs share an SM, which
// hides the operand loads of one behind another's arithmetic; on GB300 the
// 64 x 64 tiles (one CTA per SM by registers) were slower in every measured
// shape (N = 512-1024, 64-1024 trajectories; 2.09 against 2.17 ms per step
// at their best for 1024 trajectories of N = R = 1024, 0.161 against 0.188
// ms for 64).  The split count is the one whose busiest SM has the least
// work, CTAs spreading evenly (the busiest SM runs ceil(CTAs / SMs) of
// them), with the split sums' reads and launch added; ties go to fewer
// splits.
constexpr int D_MT = 2;

struct DGemm {
  int ks;
  int64_t tiles_m, tiles_n;
};

static DGemm d_gemm(int64_t m, int64_t n, int64_t K, int nf, int sm_count) {
  constexpr int tile = 16 * D_MT;
  const int64_t nk = (K + D_BK - 1) / D_BK;
  const int64_t tm = (m + tile - 1) / tile, tn = (n + tile - 1) / tile;
  DGemm best{1, tm, tn};
  double best_us = 0.0;
  const int64_t kmax = std::min<int64_t>(nk, D_MAX_SPLITS);
  for (int64_t ks = 1; ks <= kmax; ++ks) {
    const int64_t busiest = (tm * tn * ks + sm_count - 1) / sm_count;
    const int64_t ktiles = (nk + ks - 1) / ks;
    // ~24 G double-single products per second per SM; the split sums read
    // ks x nf pairs per output at ~15 TB/s and take one more launch
    double us = (double)busiest * ktiles * tile * tile * nf * D_BK / 24.3e3;
    if (ks > 1) us += 2.0 + (double)ks * m * n * nf * 8.0 / 15e6;
    if (ks == 1 || us < best_us * 0.999) {
      best.ks = (int)ks;
      best_us = us;
    }
  }
  return best;
}

// Scratch: [states hi/lo] [H1, H2 hi/lo] [project partials] [expand partials].
struct DLayout {
  DGemm gp, ge;
  size_t x_bytes, h_bytes, pp_bytes, pe_bytes, total;
};

static int64_t d_kp(int64_t n) { return (n + D_BK - 1) / D_BK * D_BK; }

static DLayout d_layout(int64_t n, int64_t rp, int batch, int nf, int sm_count) {
  DLayout L{};
  L.gp = d_gemm(rp, batch, n, nf, sm_count);      // columns r (grid x), rows b (grid y), K = n
  L.ge = d_gemm(n, batch, rp, nf - 1, sm_count);  // columns i, rows b, K = rp (one or two terms)
  L.x_bytes = ((size_t)2 * batch * d_kp(n) * sizeof(float) + 255) / 256 * 256;
  L.h_bytes = ((size_t)4 * batch * rp * sizeof(float) + 255) / 256 * 256;
  L.pp_bytes = L.gp.ks > 1 ? (sizeof(float) * (size_t)L.gp.ks * 3 * 2 * (size_t)batch * (size_t)rp + 255) / 256 * 256 : 0;
  L.pe_bytes = L.ge.ks > 1 ? sizeof(float) * (size_t)L.ge.ks * 2 * (size_t)batch * (size_t)n : 0;
  L.total = L.x_bytes + L.h_bytes + L.pp_bytes + L.pe_bytes;
  return L;
}

size_t k3d_factor_bytes(int64_t n, int64_t rp) { return (size_t)6 * n * rp * sizeof(float); }

size_t k3d_scratch_bytes(int64_t n, int64_t rp, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = K3G_MIN_BATCH; b <= max_batch; ++b)
    for (int nf = 2; nf <= 3; ++nf) {  // the split counts depend on the form
      const DLayout L = d_layout(n, rp, b, nf, sm_count);
      if (L.total > need) need = L.total;
    }
  return need;
}

cudaError_t k3d_build_factors(const uint8_t* op, size_t panel_bytes, int64_t n, int64_t rp, void* out,
                              cudaStream_t s) {
  // op holds the three FP64 panels (fa, fb, fc: n x rp each) panel_bytes apart;
  // out gets [fa hi | fa lo | fb hi | fb lo | fc hi | fc lo], n x rp floats each
  float* o = static_cast<float*>(out);
  const int64_t count = n * rp;
  const unsigned blocks = (unsigned)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
  for (int q = 0; q < 3; ++q) {
    const double* f = reinterpret_cast<const double*>(op + q * panel_bytes);
    k3d_split_panel<<<blocks, 256, 0, s>>>(f, count, o + 2 * q * count, o + (2 * q + 1) * count);
  }
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

static void d_prep(const DDims& d, const K3Args& a, const DBufs& q, cudaStream_t s) {
  dim3 gx((unsigned)((d.kp + 255) / 256), (unsigned)d.batch);
  k3d_prep<<<gx, 256, 0, s>>>(d, a, q.xh);
}

// project (+ split sums) and expand; with one expansion split the result is
// in the output or the ring, else in the expansion partials.
static void d_gemms(const DDims& d, const DLayout& L, const K3Args& a, const float* f, const DBufs& q, int sm_count,
                    cudaStream_t s) {
  const DSplit sp{L.gp.ks, q.pp};
  const dim3 gp((unsigned)L.gp.tiles_m, (unsigned)L.gp.tiles_n, (unsigned)sp.ks);
  if (d.nf == 3)
    k3d_project<3, D_MT><<<gp, 256, 0, s>>>(d, f, q.xh, q.h, sp);
  else
    k3d_project<2, D_MT><<<gp, 256, 0, s>>>(d, f, q.xh, q.h, sp);
  if (sp.ks > 1) {
    const unsigned hb = d_flat_blocks((int64_t)d.batch * d.rp, sm_count);
    if (d.nf == 3)
      k3d_hadamard<3><<<hb, 256, 0, s>>>(d, sp, q.h);
    else
      k3d_hadamard<2><<<hb, 256, 0, s>>>(d, sp, q.h);
  }
  const DSplit se{L.ge.ks, q.pe};
  const dim3 ge((unsigned)L.ge.tiles_m, (unsigned)L.ge.tiles_n, (unsigned)se.ks);
  if (d.nf == 3)
    k3d_expand<2, D_MT><<<ge, 256, 0, s>>>(d, a, f, q.h, se);
  else
    k3d_expand<1, D_MT><<<ge, 256, 0, s>>>(d, a, f, q.h, se);
}

static DDims d_dims(const K3Plan& p, const K3Args& a, int batch) {
  return DDims{p.n, p.rb, d_kp(p.n), batch, a.form == GROM_FORM_CP_SKEW ? 3 : 2};
}

cudaError_t k3d_launch(const K3Plan& p, const K3Args& a, const void* factors, int batch, int max_batch,
                       void* scratch, int sm_count, cudaStream_t s) {
  (void)max_batch;
  const DDims d = d_dims(p, a, batch);
  const DLayout L = d_layout(d.n, d.rp, batch, d.nf, sm_count);
  const DBufs q = d_bufs(L, scratch);
  d_prep(d, a, q, s);
  d_gemms(d, L, a, static_cast<const float*>(factors), q, sm_count, s);
  if (L.ge.ks > 1)
    k3d_finish<<<d_flat_blocks((int64_t)batch * d.n, sm_count), 256, 0, s>>>(d, a, DSplit{L.ge.ks, q.pe});
  return cudaGetLastError();
}

cudaError_t k3d_launch_step(const K3Plan& p, const K3Args& a, const void* factors, int batch, void* scratch,
                            int sm_count, bool prep, const StepArgs& st, int step_index, cudaEvent_t ev0,
                            cudaEvent_t ev1, cudaStream_t s) {
  const DDims d = d_dims(p, a, batch);
  const DLayout L = d_layout(d.n, d.rp, batch, d.nf, sm_count);
  const DBufs q = d_bufs(L, scratch);
  if (prep) d_prep(d, a, q, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && ev0) e = prof_record(ev0, s);
  if (e != cudaSuccess) return e;
  d_gemms(d, L, a, static_cast<const float*>(factors), q, sm_count, s);
  e = cudaGetLastError();
  if (e == cudaSuccess && ev1) e = prof_record(ev1, s);
  if (e != cudaSuccess) return e;
  K3TStepFuse f{};
  f.d2 = q.pe;
  f.s2 = L.ge.ks;
  f.bp = batch;
  f.np = d.kp;
  f.xh = q.xh;
  f.xl = q.xh + (int64_t)batch * d.kp;
  return step_diag_mc_k3d_launch(st, step_index, f, s);
}

}  // namespace grom
