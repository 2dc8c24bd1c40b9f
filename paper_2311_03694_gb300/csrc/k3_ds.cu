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
//   prep:     the states of the batch as hi/lo planes (FP64 -> two floats).
//   project:  P = X V, Q = X W (and S = X U for the skew form), B x rp, as
//             64 x 64 register-tiled double-single GEMMs; epilogue
//             H1 = P o Q, H2 = P o S in double-single arithmetic.
//   expand:   c = H1 A^T (- H2 W^T), B x n; the FP64 result goes to the
//             output or to the advection slot of the history ring.
// The factors' hi/lo copies are made once, at create, from the FP64 panels.
// Split K and the last-CTA reduction follow K3g (deterministic).
#include "ds_arith.cuh"
#include "grom_internal.h"

namespace grom {

constexpr int D_BM = 64, D_BN = 64, D_BK = 16;
constexpr int D_FAST_SPLITS = 8;  // split counts whose partials the last CTA loads all at once

struct DDims {
  int64_t n, rp, kp;  // modes, padded rank (factor row pitch), state row pitch (n rounded up to D_BK)
  int batch, nf;
};

struct DSplit {
  int ks;
  float* partial;     // ks x nf x 2 x batch x rp (project) or ks x 2 x batch x n (expand)
  unsigned int* cnt;  // one counter per output tile
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

__global__ void __launch_bounds__(256) k3d_project(const DDims d, const float* fhl, const float* xh, float* hbuf,
                                                   const DSplit sp) {
  __shared__ float Us[2][D_BK][D_BM + 4];
  __shared__ float Xs[3][2][D_BK][D_BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * D_BM;
  const int64_t r0 = (int64_t)blockIdx.x * D_BN;
  const int64_t fplane = d.n * d.rp;
  // factor q (0 = fa, 1 = fb, 2 = fc) hi plane at fhl + 2 q fplane, lo plane after it;
  // projections in the order (fb, fc, fa): P, Q, S
  const int fq[3] = {1, 2, 0};
  const float* xl = xh + (int64_t)d.batch * d.kp;
  float S[3][4][4], s[3][4][4];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) S[f][x][y] = s[f][x][y] = 0.f;
  const int lb = tid >> 2, li = (tid & 3) * 4;   // state tile: 64 b x (4 x 4) k
  const int xi = tid >> 4, xr = (tid & 15) * 4;  // factor tile: 16 k x (16 x 4) r
  const int bl = b0 + lb;
  const int64_t nk = (d.n + D_BK - 1) / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * D_BK; k0 < kb1 * D_BK; k0 += D_BK) {
    // states: k < kp always (kp is n rounded up to D_BK), zero past n
    if (bl < d.batch) {
      const float4 vh = *reinterpret_cast<const float4*>(xh + (int64_t)bl * d.kp + k0 + li);
      const float4 vl = *reinterpret_cast<const float4*>(xl + (int64_t)bl * d.kp + k0 + li);
      Us[0][li][lb] = vh.x; Us[0][li + 1][lb] = vh.y; Us[0][li + 2][lb] = vh.z; Us[0][li + 3][lb] = vh.w;
      Us[1][li][lb] = vl.x; Us[1][li + 1][lb] = vl.y; Us[1][li + 2][lb] = vl.z; Us[1][li + 3][lb] = vl.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) Us[0][li + q][lb] = Us[1][li + q][lb] = 0.f;
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (f < d.nf) {
        const int64_t i = k0 + xi;
        const float* fh = fhl + 2 * fq[f] * fplane;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = r0 + xr + q;
          const bool ok = i < d.n && r < d.rp;
          Xs[f][0][xi][xr + q] = ok ? fh[i * d.rp + r] : 0.f;
          Xs[f][1][xi][xr + q] = ok ? fh[fplane + i * d.rp + r] : 0.f;
        }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < D_BK; ++k) {
      float uh[4], ul[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        uh[x] = Us[0][k][ty * 4 + x];
        ul[x] = Us[1][k][ty * 4 + x];
      }
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (f < d.nf) {
          float vh[4], vl[4];
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            vh[y] = Xs[f][0][k][tx * 4 + y];
            vl[y] = Xs[f][1][k][tx * 4 + y];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) ds_mac(uh[x], ul[x], vh[y], vl[y], S[f][x][y], s[f][x][y]);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) ds_renorm(S[f][x][y], s[f][x][y]);
    __syncthreads();
  }
  // H1 = P o Q and H2 = P o S as hi/lo planes: hbuf = [H1h | H1l | H2h | H2l], batch x rp each
  const int64_t plane = (int64_t)d.batch * d.rp;
  auto write_h = [&](int b, int64_t r, const float* Sv, const float* sv) {
    float h, l;
    ds_mul(Sv[0], sv[0], Sv[1], sv[1], h, l);
    hbuf[(int64_t)b * d.rp + r] = h;
    hbuf[plane + (int64_t)b * d.rp + r] = l;
    if (d.nf == 3) {
      ds_mul(Sv[0], sv[0], Sv[2], sv[2], h, l);
      hbuf[2 * plane + (int64_t)b * d.rp + r] = h;
      hbuf[3 * plane + (int64_t)b * d.rp + r] = l;
    }
  };
  if (sp.ks == 1) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int b = b0 + ty * 4 + x;
      if (b >= d.batch) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int64_t r = r0 + tx * 4 + y;
        if (r >= d.rp) continue;
        const float Sv[3] = {S[0][x][y], S[1][x][y], S[2][x][y]};
        const float sv[3] = {s[0][x][y], s[1][x][y], s[2][x][y]};
        write_h(b, r, Sv, sv);
      }
    }
    return;
  }
  // split K: this split's partial pairs, the last split of the tile sums them in order
  float* part = sp.partial;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int b = b0 + ty * 4 + x;
    if (b >= d.batch) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t r = r0 + tx * 4 + y;
      if (r >= d.rp) continue;
#pragma unroll
      for (int f = 0; f < 3; ++f)
        if (f < d.nf) {
          float* dst = part + (((int64_t)blockIdx.z * d.nf + f) * 2) * plane + (int64_t)b * d.rp + r;
          dst[0] = S[f][x][y];
          dst[plane] = s[f][x][y];
        }
    }
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid == 0) last = atomicAdd(&sp.cnt[tile], 1u) == (unsigned)(sp.ks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int b = b0 + ty * 4 + x;
    if (b >= d.batch) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t r = r0 + tx * 4 + y;
      if (r >= d.rp) continue;
      float Sv[3] = {0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f};
      const float* src0 = part + (int64_t)b * d.rp + r;
      if (sp.ks <= D_FAST_SPLITS) {
        // every split's pair loaded before the sums (the L2 reads in flight
        // together), then summed in split order as below
        float w[D_FAST_SPLITS][3][2];
#pragma unroll
        for (int z = 0; z < D_FAST_SPLITS; ++z)
#pragma unroll
          for (int f = 0; f < 3; ++f)
            if (z < sp.ks && f < d.nf) {
              const float* src = src0 + (((int64_t)z * d.nf + f) * 2) * plane;
              w[z][f][0] = __ldcg(src);
              w[z][f][1] = __ldcg(src + plane);
            }
#pragma unroll
        for (int z = 0; z < D_FAST_SPLITS; ++z)
#pragma unroll
          for (int f = 0; f < 3; ++f)
            if (z < sp.ks && f < d.nf) ds_add(Sv[f], sv[f], w[z][f][0], w[z][f][1]);
      } else {
        for (int z = 0; z < sp.ks; ++z)
#pragma unroll
          for (int f = 0; f < 3; ++f)
            if (f < d.nf) {
              const float* src = src0 + (((int64_t)z * d.nf + f) * 2) * plane;
              ds_add(Sv[f], sv[f], __ldcg(src), __ldcg(src + plane));
            }
      }
      write_h(b, r, Sv, sv);
    }
  }
  if (tid == 0) sp.cnt[tile] = 0u;
}

__global__ void __launch_bounds__(256) k3d_expand(const DDims d, const K3Args a, const float* fhl, const float* hbuf,
                                                  const DSplit sp) {
  __shared__ float Hs[2][2][D_BK][D_BM + 4];  // [term][hi/lo][r][b]
  __shared__ float As[2][2][D_BK][D_BN + 4];  // [term][hi/lo][r][i]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * D_BM;
  const int64_t i0 = (int64_t)blockIdx.x * D_BN;
  const int64_t fplane = d.n * d.rp;
  const int64_t plane = (int64_t)d.batch * d.rp;
  const int nm = d.nf == 3 ? 2 : 1;
  // first term: A (fa); second (skew form): -W (fc)
  const float* Fm[2] = {fhl, fhl + 4 * fplane};
  float S[4][4], s[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) S[x][y] = s[x][y] = 0.f;
  const int lb = tid >> 2, lr = (tid & 3) * 4;  // H tile 64 b x 16 r
  const int ai = tid >> 2, ar = (tid & 3) * 4;  // factor tile 64 i x 16 r (stored transposed)
  const int64_t nk = (d.rp + D_BK - 1) / D_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * D_BK; k0 < kb1 * D_BK; k0 += D_BK) {
    const int b = b0 + lb;
    const int64_t i = i0 + ai;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m < nm) {
        const float* hh = hbuf + 2 * m * plane;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = k0 + lr + q;
          const bool ok = b < d.batch && r < d.rp;
          Hs[m][0][lr + q][lb] = ok ? hh[(int64_t)b * d.rp + r] : 0.f;
          Hs[m][1][lr + q][lb] = ok ? hh[plane + (int64_t)b * d.rp + r] : 0.f;
        }
        const float sgn = m == 0 ? 1.f : -1.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = k0 + ar + q;
          const bool ok = i < d.n && r < d.rp;
          As[m][0][ar + q][ai] = ok ? sgn * Fm[m][i * d.rp + r] : 0.f;
          As[m][1][ar + q][ai] = ok ? sgn * Fm[m][fplane + i * d.rp + r] : 0.f;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m < nm) {
#pragma unroll 4
        for (int k = 0; k < D_BK; ++k) {
          float hh[4], hl[4], ah[4], al[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            hh[x] = Hs[m][0][k][ty * 4 + x];
            hl[x] = Hs[m][1][k][ty * 4 + x];
          }
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            ah[y] = As[m][0][k][tx * 4 + y];
            al[y] = As[m][1][k][tx * 4 + y];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) ds_mac(hh[x], hl[x], ah[y], al[y], S[x][y], s[x][y]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) ds_renorm(S[x][y], s[x][y]);
      }
    }
    __syncthreads();
  }
  auto dst_of = [&](int b) -> double* {
    return a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
  };
  if (sp.ks == 1) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int b = b0 + ty * 4 + x;
      if (b >= d.batch || (a.active && !a.active[b])) continue;
      double* dst = dst_of(b);
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int64_t i = i0 + tx * 4 + y;
        if (i < d.n) dst[i] = (double)S[x][y] + (double)s[x][y];
      }
    }
    return;
  }
  float* part = sp.partial;
  const int64_t oplane = (int64_t)d.batch * d.n;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int b = b0 + ty * 4 + x;
    if (b >= d.batch) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + tx * 4 + y;
      if (i >= d.n) continue;
      float* p = part + (int64_t)blockIdx.z * 2 * oplane + (int64_t)b * d.n + i;
      p[0] = S[x][y];
      p[oplane] = s[x][y];
    }
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid == 0) last = atomicAdd(&sp.cnt[tile], 1u) == (unsigned)(sp.ks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int b = b0 + ty * 4 + x;
    if (b >= d.batch || (a.active && !a.active[b])) continue;
    double* dst = dst_of(b);
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + tx * 4 + y;
      if (i >= d.n) continue;
      float Sv = 0.f, sv = 0.f;
      const float* p0 = part + (int64_t)b * d.n + i;
      if (sp.ks <= D_FAST_SPLITS) {
        float w[D_FAST_SPLITS][2];
#pragma unroll
        for (int z = 0; z < D_FAST_SPLITS; ++z)
          if (z < sp.ks) {
            w[z][0] = __ldcg(p0 + (int64_t)z * 2 * oplane);
            w[z][1] = __ldcg(p0 + (int64_t)z * 2 * oplane + oplane);
          }
#pragma unroll
        for (int z = 0; z < D_FAST_SPLITS; ++z)
          if (z < sp.ks) ds_add(Sv, sv, w[z][0], w[z][1]);
      } else {
        for (int z = 0; z < sp.ks; ++z) {
          const float* p = p0 + (int64_t)z * 2 * oplane;
          ds_add(Sv, sv, __ldcg(p), __ldcg(p + oplane));
        }
      }
      dst[i] = (double)Sv + (double)sv;
    }
  }
  if (tid == 0) sp.cnt[tile] = 0u;
}

// K splits so that the grid covers about two waves of the GPU; each split
// keeps at least 128 elements of the K range, or for short ranges one K
// tile (up to 8 splits), so that small problems (a serving pool of a small
// ROM: one output tile) still spread over several SMs.  (A 64-element floor
// measured slower at N = 1024 with 16-64 trajectories: the last CTA's sum of
// 16 splits costs more than the extra parallelism gains.)
static int d_splits(int64_t tiles, int64_t K, int sm_count) {
  int64_t ks = (2 * sm_count + tiles - 1) / tiles;
  const int64_t kshort = K / D_BK < 8 ? K / D_BK : 8;
  const int64_t kmax = K / 128 > kshort ? K / 128 : kshort;
  if (ks > kmax) ks = kmax;
  if (ks < 1) ks = 1;
  return (int)ks;
}

// Scratch: [tile counters, sized for the largest batch] [states hi/lo]
// [H1, H2 hi/lo] [project partials] [expand partials].
struct DLayout {
  int ks_p, ks_e;
  size_t cnt_bytes, x_bytes, h_bytes, pp_bytes, pe_bytes, total;
  size_t tiles_cap;
};

static int64_t d_kp(int64_t n) { return (n + D_BK - 1) / D_BK * D_BK; }

static DLayout d_layout(int64_t n, int64_t rp, int batch, int max_batch, int sm_count) {
  DLayout L{};
  const int64_t bt = (batch + D_BM - 1) / D_BM;
  L.ks_p = d_splits(bt * ((rp + D_BN - 1) / D_BN), n, sm_count);
  L.ks_e = d_splits(bt * ((n + D_BN - 1) / D_BN), rp, sm_count);
  L.tiles_cap = (size_t)((max_batch + D_BM - 1) / D_BM) * (size_t)(((rp > n ? rp : n) + D_BN - 1) / D_BN);
  L.cnt_bytes = (2 * L.tiles_cap * sizeof(unsigned int) + 255) / 256 * 256;
  L.x_bytes = ((size_t)2 * batch * d_kp(n) * sizeof(float) + 255) / 256 * 256;
  L.h_bytes = ((size_t)4 * batch * rp * sizeof(float) + 255) / 256 * 256;
  L.pp_bytes = L.ks_p > 1 ? sizeof(float) * (size_t)L.ks_p * 3 * 2 * (size_t)batch * (size_t)rp : 0;
  L.pe_bytes = L.ks_e > 1 ? sizeof(float) * (size_t)L.ks_e * 2 * (size_t)batch * (size_t)n : 0;
  L.total = L.cnt_bytes + L.x_bytes + L.h_bytes + L.pp_bytes + L.pe_bytes;
  return L;
}

size_t k3d_factor_bytes(int64_t n, int64_t rp) { return (size_t)6 * n * rp * sizeof(float); }

size_t k3d_scratch_bytes(int64_t n, int64_t rp, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = K3G_MIN_BATCH; b <= max_batch; ++b) {
    const DLayout L = d_layout(n, rp, b, max_batch, sm_count);
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

cudaError_t k3d_launch(const K3Plan& p, const K3Args& a, const void* factors, int batch, int max_batch,
                       void* scratch, int sm_count, cudaStream_t s) {
  DDims d{p.n, p.rb, d_kp(p.n), batch, a.form == GROM_FORM_CP_SKEW ? 3 : 2};
  const DLayout L = d_layout(d.n, d.rp, batch, max_batch, sm_count);
  uint8_t* base = static_cast<uint8_t*>(scratch);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(base);
  float* xh = reinterpret_cast<float*>(base + L.cnt_bytes);
  float* h = reinterpret_cast<float*>(base + L.cnt_bytes + L.x_bytes);
  float* pp = reinterpret_cast<float*>(base + L.cnt_bytes + L.x_bytes + L.h_bytes);
  float* pe = reinterpret_cast<float*>(base + L.cnt_bytes + L.x_bytes + L.h_bytes + L.pp_bytes);
  const float* f = static_cast<const float*>(factors);
  dim3 gx((unsigned)((d.kp + 255) / 256), (unsigned)batch);
  k3d_prep<<<gx, 256, 0, s>>>(d, a, xh);
  DSplit sp{L.ks_p, pp, cnt};
  DSplit se{L.ks_e, pe, cnt + L.tiles_cap};
  dim3 gp((unsigned)((d.rp + D_BN - 1) / D_BN), (unsigned)((batch + D_BM - 1) / D_BM), (unsigned)sp.ks);
  k3d_project<<<gp, 256, 0, s>>>(d, f, xh, h, sp);
  dim3 ge((unsigned)((d.n + D_BN - 1) / D_BN), (unsigned)((batch + D_BM - 1) / D_BM), (unsigned)se.ks);
  k3d_expand<<<ge, 256, 0, s>>>(d, a, f, h, se);
  return cudaGetLastError();
}

}  // namespace grom
