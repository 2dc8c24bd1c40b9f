// K3 for batches: the CP-form advection term (Sec. 3.1, eq. tc_ap; skew
// structure Sec. 3.3) of B trajectories as register-tiled GEMMs.
//
//   project:  P = U_B X_b, Q = U_B X_c (and S = U_B X_a for the skew form),
//             U_B the B x n states, X n x rp factors; epilogue H1 = P o Q,
//             H2 = P o S, written as B x rp.
//   expand:   C_out = H1 A^T (- H2 W^T), B x n, written in FP64 to the output
//             or to the advection slot of the history ring.
//
// CTA tile 64 x 64 (trajectories x columns), K step 16, 256 threads with a
// 4 x 4 register micro-tile each; the three projections share the state tile.
// Arithmetic in FP32 for FP32/BF16 storage, FP64 for FP64 storage.  Used for
// batches of 16 or more trajectories.  When the output tiles alone cannot
// fill the GPU the K range is split across CTAs; each split writes a partial
// tile and the last CTA of the tile to arrive (arrival counter, no waiting)
// sums the splits in order, so results stay deterministic.
#include "grom_internal.h"

namespace grom {

constexpr int G_BM = 64, G_BN = 64, G_BK = 16;

template <int ST>
struct GT;
template <>
struct GT<GROM_F64> {
  using acc_t = double;
  static __device__ __forceinline__ double ld(const uint8_t* p, int64_t idx) {
    return reinterpret_cast<const double*>(p)[idx];
  }
  static __device__ __forceinline__ double cu(double v) { return v; }
};
template <>
struct GT<GROM_F32> {
  using acc_t = float;
  static __device__ __forceinline__ float ld(const uint8_t* p, int64_t idx) {
    return reinterpret_cast<const float*>(p)[idx];
  }
  static __device__ __forceinline__ float cu(double v) { return __double2float_rn(v); }
};
template <>
struct GT<GROM_BF16> {
  using acc_t = float;
  static __device__ __forceinline__ float ld(const uint8_t* p, int64_t idx) {
    return __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(p)[idx] << 16);
  }
  static __device__ __forceinline__ float cu(double v) { return __double2float_rn(v); }
};

struct GDims {
  int64_t n, rp;
  int batch, nf;
};

__device__ __forceinline__ const double* g_state(const K3Args& a, int b, int64_t n) {
  return a.taken ? a.hist + b * a.hist_stride + (a.taken[b] % 3) * n : a.u + b * a.u_stride;
}

struct GSplit {
  int ks;                 // K splits
  void* partial;          // ks x nf x batch x rp (project) or ks x batch x n (expand)
  unsigned int* cnt;      // one counter per output tile
};

template <int ST>
__global__ void __launch_bounds__(256) k3g_project(const GDims d, const K3Args a, void* hbuf, const GSplit sp) {
  using T = GT<ST>;
  using acc_t = typename T::acc_t;
  __shared__ acc_t Us[G_BK][G_BM + 4];
  __shared__ acc_t Xs[3][G_BK][G_BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * G_BM;
  const int64_t r0 = (int64_t)blockIdx.x * G_BN;
  const uint8_t* F[3] = {a.fb, a.fc, a.fa};
  acc_t acc[3][4][4];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[f][x][y] = acc_t(0);
  // per-thread load coordinates: state tile (64 b x 16 i), factor tiles (16 i x 64 r)
  const int lb = tid >> 2, li = (tid & 3) * 4;   // 64 x (4 x 4)
  const int xi = tid >> 4, xr = (tid & 15) * 4;  // 16 x (16 x 4)
  const int bl = b0 + lb;
  const bool b_on = bl < d.batch && (a.active == nullptr || a.active[bl]);
  const double* urow = b_on ? g_state(a, bl, d.n) : nullptr;
  const int64_t nk = (d.n + G_BK - 1) / G_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * G_BK; k0 < kb1 * G_BK; k0 += G_BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = k0 + li + q;
      Us[li + q][lb] = (b_on && i < d.n) ? T::cu(urow[i]) : acc_t(0);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (f < d.nf) {
        const int64_t i = k0 + xi;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = r0 + xr + q;
          Xs[f][xi][xr + q] = (i < d.n && r < d.rp) ? T::ld(F[f], i * d.rp + r) : acc_t(0);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G_BK; ++k) {
      acc_t ub[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) ub[x] = Us[k][ty * 4 + x];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (f < d.nf) {
          acc_t xv[4];
#pragma unroll
          for (int y = 0; y < 4; ++y) xv[y] = Xs[f][k][tx * 4 + y];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[f][x][y] = fma(ub[x], xv[y], acc[f][x][y]);
        }
      }
    }
    __syncthreads();
  }
  acc_t* h1 = reinterpret_cast<acc_t*>(hbuf);
  acc_t* h2 = h1 + (int64_t)d.batch * d.rp;
  if (sp.ks == 1) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int b = b0 + ty * 4 + x;
      if (b >= d.batch) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int64_t r = r0 + tx * 4 + y;
        if (r >= d.rp) continue;
        h1[(int64_t)b * d.rp + r] = acc[0][x][y] * acc[1][x][y];
        if (d.nf == 3) h2[(int64_t)b * d.rp + r] = acc[0][x][y] * acc[2][x][y];
      }
    }
    return;
  }
  // split K: write this split's partial tile, the last split of the tile sums them
  acc_t* part = reinterpret_cast<acc_t*>(sp.partial);
  const int64_t plane = (int64_t)d.batch * d.rp;
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
        if (f < d.nf) part[((int64_t)blockIdx.z * d.nf + f) * plane + (int64_t)b * d.rp + r] = acc[f][x][y];
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
      acc_t v[3] = {acc_t(0), acc_t(0), acc_t(0)};
      for (int z = 0; z < sp.ks; ++z)
#pragma unroll
        for (int f = 0; f < 3; ++f)
          if (f < d.nf) v[f] += __ldcg(part + ((int64_t)z * d.nf + f) * plane + (int64_t)b * d.rp + r);
      h1[(int64_t)b * d.rp + r] = v[0] * v[1];
      if (d.nf == 3) h2[(int64_t)b * d.rp + r] = v[0] * v[2];
    }
  }
  if (tid == 0) sp.cnt[tile] = 0u;
}

template <int ST>
__global__ void __launch_bounds__(256) k3g_expand(const GDims d, const K3Args a, const void* hbuf, const GSplit sp) {
  using T = GT<ST>;
  using acc_t = typename T::acc_t;
  __shared__ acc_t Hs[2][G_BK][G_BM + 4];
  __shared__ acc_t As[2][G_BK][G_BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int b0 = blockIdx.y * G_BM;
  const int64_t i0 = (int64_t)blockIdx.x * G_BN;
  const acc_t* h1 = reinterpret_cast<const acc_t*>(hbuf);
  const acc_t* h2 = h1 + (int64_t)d.batch * d.rp;
  const int nm = d.nf == 3 ? 2 : 1;
  acc_t acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = acc_t(0);
  const int lb = tid >> 2, lr = (tid & 3) * 4;  // H tile 64 b x 16 r
  const int ai = tid >> 2, ar = (tid & 3) * 4;  // A tile 64 i x 16 r (stored transposed)
  const uint8_t* Fm[2] = {a.fa, a.fc};
  const int64_t nk = (d.rp + G_BK - 1) / G_BK;
  const int64_t kb0 = (int64_t)blockIdx.z * nk / sp.ks, kb1 = ((int64_t)blockIdx.z + 1) * nk / sp.ks;
  for (int64_t k0 = kb0 * G_BK; k0 < kb1 * G_BK; k0 += G_BK) {
    const int b = b0 + lb;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m < nm) {
        const acc_t* hm = m == 0 ? h1 : h2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = k0 + lr + q;
          Hs[m][lr + q][lb] = (b < d.batch && r < d.rp) ? hm[(int64_t)b * d.rp + r] : acc_t(0);
        }
        const int64_t i = i0 + ai;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t r = k0 + ar + q;
          const acc_t v = (i < d.n && r < d.rp) ? T::ld(Fm[m], i * d.rp + r) : acc_t(0);
          As[m][ar + q][ai] = m == 0 ? v : -v;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m < nm) {
#pragma unroll
        for (int k = 0; k < G_BK; ++k) {
          acc_t hv[4], av[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) hv[x] = Hs[m][k][ty * 4 + x];
#pragma unroll
          for (int y = 0; y < 4; ++y) av[y] = As[m][k][tx * 4 + y];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(hv[x], av[y], acc[x][y]);
        }
      }
    }
    __syncthreads();
  }
  if (sp.ks == 1) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int b = b0 + ty * 4 + x;
      if (b >= d.batch || (a.active && !a.active[b])) continue;
      double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int64_t i = i0 + tx * 4 + y;
        if (i < d.n) dst[i] = (double)acc[x][y];
      }
    }
    return;
  }
  acc_t* part = reinterpret_cast<acc_t*>(sp.partial);
  const int64_t plane = (int64_t)d.batch * d.n;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int b = b0 + ty * 4 + x;
    if (b >= d.batch) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + tx * 4 + y;
      if (i < d.n) part[(int64_t)blockIdx.z * plane + (int64_t)b * d.n + i] = acc[x][y];
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
    double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + tx * 4 + y;
      if (i >= d.n) continue;
      acc_t v = acc_t(0);
      for (int z = 0; z < sp.ks; ++z) v += __ldcg(part + (int64_t)z * plane + (int64_t)b * d.n + i);
      dst[i] = (double)v;
    }
  }
  if (tid == 0) sp.cnt[tile] = 0u;
}

// K splits so that the grid covers about two waves of the GPU; each split
// keeps at least 128 elements of the K range, or for short ranges one K
// tile (up to 8 splits), so that a small problem (one output tile: 64
// trajectories of an N = 128 ROM) spreads over several SMs instead of one.
static int g_splits(int64_t tiles, int64_t K, int sm_count) {
  int64_t ks = (2 * sm_count + tiles - 1) / tiles;
  const int64_t kshort = K / G_BK < 8 ? K / G_BK : 8;
  const int64_t kmax = K / 128 > kshort ? K / 128 : kshort;
  if (ks > kmax) ks = kmax;
  if (ks < 1) ks = 1;
  return (int)ks;
}

// Scratch layout: [tile counters, sized for the largest batch, fixed offset]
// [H1 H2] [project partials] [expand partials].  The counters never move, so
// partial sums of one batch size cannot land on the counters of another.
struct GLayout {
  int ks_p, ks_e;
  size_t cnt_bytes, h_bytes, pp_bytes, pe_bytes, total;
  size_t tiles_cap;
};

static GLayout g_layout(int64_t n, int64_t rp, int batch, int max_batch, int storage, int sm_count) {
  GLayout L{};
  const size_t es = storage == GROM_F64 ? 8 : 4;
  const int64_t bt = (batch + G_BM - 1) / G_BM;
  L.ks_p = g_splits(bt * ((rp + G_BN - 1) / G_BN), n, sm_count);
  L.ks_e = g_splits(bt * ((n + G_BN - 1) / G_BN), rp, sm_count);
  L.tiles_cap = (size_t)((max_batch + G_BM - 1) / G_BM) * (size_t)(((rp > n ? rp : n) + G_BN - 1) / G_BN);
  L.cnt_bytes = (2 * L.tiles_cap * sizeof(unsigned int) + 255) / 256 * 256;
  L.h_bytes = 2 * es * (size_t)rp * (size_t)batch;
  L.pp_bytes = L.ks_p > 1 ? es * (size_t)L.ks_p * 3 * (size_t)batch * (size_t)rp : 0;
  L.pe_bytes = L.ks_e > 1 ? es * (size_t)L.ks_e * (size_t)batch * (size_t)n : 0;
  L.total = L.cnt_bytes + L.h_bytes + L.pp_bytes + L.pe_bytes;
  return L;
}

// Scratch for every batch size up to max_batch (the split count, and with it
// the partial buffers, is not monotonic in the batch size).
size_t k3g_scratch_bytes(int64_t n, int64_t rp, int max_batch, int storage, int sm_count) {
  size_t need = 0;
  for (int b = K3G_MIN_BATCH; b <= max_batch; ++b) {
    const GLayout L = g_layout(n, rp, b, max_batch, storage, sm_count);
    if (L.total > need) need = L.total;
  }
  return need;
}

template <int ST>
static cudaError_t k3g_run(const GDims& d, const K3Args& a, void* scratch, int max_batch, int sm_count,
                           cudaStream_t s) {
  const GLayout L = g_layout(d.n, d.rp, d.batch, max_batch, ST, sm_count);
  uint8_t* base = reinterpret_cast<uint8_t*>(scratch);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(base);
  uint8_t* h = base + L.cnt_bytes;
  GSplit sp{L.ks_p, h + L.h_bytes, cnt};
  GSplit se{L.ks_e, h + L.h_bytes + L.pp_bytes, cnt + L.tiles_cap};
  dim3 gp((unsigned)((d.rp + G_BN - 1) / G_BN), (unsigned)((d.batch + G_BM - 1) / G_BM), (unsigned)sp.ks);
  k3g_project<ST><<<gp, 256, 0, s>>>(d, a, h, sp);
  dim3 ge((unsigned)((d.n + G_BN - 1) / G_BN), (unsigned)((d.batch + G_BM - 1) / G_BM), (unsigned)se.ks);
  k3g_expand<ST><<<ge, 256, 0, s>>>(d, a, h, se);
  return cudaGetLastError();
}

cudaError_t k3g_launch(const K3Plan& p, int storage, const K3Args& a, int batch, int max_batch, void* scratch,
                       int sm_count, cudaStream_t s) {
  GDims d{p.n, p.rb, batch, a.form == GROM_FORM_CP_SKEW ? 3 : 2};
  switch (storage) {
    case GROM_F64: return k3g_run<GROM_F64>(d, a, scratch, max_batch, sm_count, s);
    case GROM_F32: return k3g_run<GROM_F32>(d, a, scratch, max_batch, sm_count, s);
    case GROM_BF16: return k3g_run<GROM_BF16>(d, a, scratch, max_batch, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace grom
