// K2: batched dense contraction on the tcgen05 tensor cores (BF16 storage).
//
// For B trajectories the contraction is one GEMM (Sec. 2.2, eq. Cu, written
// with the mode-1 matricisation of C):
//   Cout[i, b] = sum_{(j,k)} C_(1)[i, (j,k)] * KR[(j,k), b],  KR[(j,k), b] = u_bj u_bk
// with M = n (test index), N = B, K = n * np.  KR, the Khatri-Rao product of
// the states, is never materialised: each K-tile of 64 covers one advecting
// index j and 64 advected indices k, so its KR tile is u_bj * u_b[k0:k0+64],
// generated in registers (FP32 products) and written into shared memory in the
// 128-byte swizzled K-major layout the tensor core reads.  Each product p is
// stored as two BF16 tiles hi = rn(p), lo = rn(p - hi) and both are
// multiplied (two MMAs per K step): rounding p to BF16 alone would add an
// error of the size of the tensor's own BF16 rounding, which on
// cancellation-heavy states pushes the result past the BF16 tolerance; with
// the split the Khatri-Rao operand is exact to ~2^-17.
//
// CTA (10 warps): warp 0 issues TMA loads of 256 x 64 BF16 tiles of C (two
// 128-row halves), either from the row layout of the stored tensor (rows
// (i, j) of np values: a tile is 256 segments of 128 bytes, n*np*2 bytes
// apart) or, when the ROM keeps one, from a tile-major copy in which every
// 256 x 64 tile is one contiguous 32 KB block (full DRAM bursts, which the
// small-batch, bandwidth-bound regime needs); warp 1 owns the tensor memory and issues tcgen05.mma
// (M=128, N=btile, K=16) into two FP32 accumulators in TMEM, one per half,
// both fed by the same KR tile, which halves KR generation per flop; warps 2-9
// generate the KR tiles (one row b each, u_bj prefetched eight tiles ahead)
// and afterwards read the accumulators back (tcgen05.ld) and store FP32
// partial sums.  Stages are recycled through mbarriers signalled by
// tcgen05.commit.  The K range is split across CTAs by ranges of j; a reduce
// kernel sums the splits in a fixed order (deterministic) into FP64.
// K-tiles are ordered with the advected block outer and j inner, so each
// generator thread keeps its 64 u_bk values in registers across j.
//
// The same kernel computes the MTTKRP of CP fitting (Sec. 2.3, eq. cp_als):
// with KR[(j,k), b] = P_jb Q_kb for two factor matrices P and Q (column b a
// rank component) instead of u_bj u_bk, Cout = X_(1) (P kr Q).
#include <cudaTypedefs.h>

#include <algorithm>

#include "grom_internal.h"
#include "tc.cuh"

namespace grom {

constexpr int K2_THREADS = 320;
constexpr int K2_GEN_WARPS = 8;
constexpr int K2_MT = 2;                         // 128-row accumulators per CTA
constexpr int K2_A_TILE = 128 * 128;             // 128 rows x 64 bf16
constexpr int K2_A_BYTES = K2_MT * K2_A_TILE;    // one TMA box of 256 rows
constexpr int K2_PF = 8;                         // u_bj prefetch distance (tiles)

struct K2Dev {
  int64_t n, np;
  int btile, col_tiles, i_tiles, splits, stages_a, stages_b, tmem_cols;
  int64_t bp;  // padded batch = col_tiles * btile
  int tiled;   // 1: the tensor map covers the tile-major copy
  float* pb;   // bp x np FP32 weights of the middle index j (u, or factor P^T)
  float* qb;   // bp x np FP32 weights of the inner index k (u, or factor Q^T), zero padded
  float* part; // splits x n x bp FP32 partials
  int* err;
};

__device__ __forceinline__ void k2_abort(volatile int* abort_flag, int* err) {
  *abort_flag = 1;
  atomicOr(err, DEV_ERR_TIMEOUT);
}

// K-tile t of a CTA: advected block kb = t / nj (outer), advecting index j0 + t % nj (inner).
__device__ __forceinline__ int64_t k2_j(int64_t t, int64_t nj, int64_t j0) { return j0 + t % nj; }

// TPR generator threads share a Khatri-Rao row (each writes 8 / TPR of its
// eight 16-byte swizzle chunks), so narrow column tiles still keep all eight
// generator warps busy: TPR = min(8, 256 / btile).
template <int TPR>
__global__ void __launch_bounds__(K2_THREADS, 1) k2_tc_kernel(const __grid_constant__ CUtensorMap tmap, const K2Dev p) {
  // btile <= 128 (TPR >= 2): one MMA of N = 2 btile multiplies the hi and lo
  // KR tiles together
  constexpr bool MERGED = TPR > 1;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int SA = p.stages_a, SB = p.stages_b;
  const int half_bytes = p.btile * 128;   // one BF16 KR tile (hi or lo)
  const int b_bytes = 2 * half_bytes;      // hi tile, then lo tile
  uint8_t* sa = smem;                                  // SA x (2 x 128 rows x 128 B)
  uint8_t* sb = smem + (size_t)SA * K2_A_BYTES;        // SB x (hi | lo)
  uint64_t* full_a = reinterpret_cast<uint64_t*>(sb + (size_t)SB * b_bytes);
  uint64_t* empty_a = full_a + SA;
  uint64_t* full_b = empty_a + SA;
  uint64_t* empty_b = full_b + SB;
  uint64_t* accum = empty_b + SB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile coordinates: a pair of 128-row tiles of the test index, a column tile, a K split
  const int split = blockIdx.x % p.splits;
  const int rest = blockIdx.x / p.splits;
  const int col_tile = rest % p.col_tiles;
  const int i_pair = rest / p.col_tiles;
  const int64_t j0 = (int64_t)split * p.n / p.splits, j1 = ((int64_t)split + 1) * p.n / p.splits;
  const int64_t nj = j1 - j0;
  const int64_t kblocks = p.np / 64;
  const int64_t T = nj * kblocks;  // K-tiles of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      ptx::mbar_init(&full_a[s], 1);
      ptx::mbar_init(&empty_a[s], 1);
    }
    for (int s = 0; s < SB; ++s) {
      ptx::mbar_init(&full_b[s], K2_GEN_WARPS);
      ptx::mbar_init(&empty_b[s], 1);
    }
    ptx::mbar_init(accum, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmap);
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, (uint32_t)p.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int64_t t = 0;
      for (; t < T; ++t) {
        const int s = (int)(t % SA);
        const uint32_t ph = (uint32_t)((t / SA) & 1);
        if (t >= SA && !ptx::mbar_wait(&empty_a[s], ph ^ 1u, abort_flag)) {
          k2_abort(abort_flag, p.err);
          break;
        }
        const int64_t kb = t / nj, j = j0 + (t - kb * nj);
        ptx::mbar_arrive_expect_tx(&full_a[s], K2_A_BYTES);
        if (p.tiled)
          tc::tma_load_2d(sa + (size_t)s * K2_A_BYTES, &tmap, 0,
                          (int32_t)((((int64_t)i_pair * p.n + j) * kblocks + kb) * 256), &full_a[s]);
        else
          tc::tma_load_2d(sa + (size_t)s * K2_A_BYTES, &tmap, (int32_t)(j * p.np + kb * 64), i_pair * 256, &full_a[s]);
      }
      for (int64_t q = t > SA ? t - SA : 0; q < t; ++q)
        if (!ptx::mbar_wait(&full_a[q % SA], (uint32_t)((q / SA) & 1), nullptr)) atomicOr(p.err, DEV_ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // merged: the hi and lo KR tiles are adjacent in shared memory, so one
      // MMA of N = 2 btile covers both (half the instructions); the
      // accumulator of each 128-row half holds A hi^T | A lo^T side by side
      const uint32_t idesc = tc::idesc_bf16_f32(128, MERGED ? 2 * p.btile : p.btile);
      const uint32_t acc1 = tmem + (uint32_t)(MERGED ? 2 * p.btile : p.btile);
      for (int64_t t = 0; t < T; ++t) {
        const int s = (int)(t % SA), r = (int)(t % SB);
        if (!ptx::mbar_wait(&full_a[s], (uint32_t)((t / SA) & 1), abort_flag) ||
            !ptx::mbar_wait(&full_b[r], (uint32_t)((t / SB) & 1), abort_flag)) {
          k2_abort(abort_flag, p.err);
          break;
        }
        tc::fence_after_sync();
        const uint64_t a0 = tc::sw128_kmajor_desc(sa + (size_t)s * K2_A_BYTES);
        const uint64_t a1 = tc::sw128_kmajor_desc(sa + (size_t)s * K2_A_BYTES + K2_A_TILE);
        const uint64_t bh = tc::sw128_kmajor_desc(sb + (size_t)r * b_bytes);
        const uint64_t bl = tc::sw128_kmajor_desc(sb + (size_t)r * b_bytes + half_bytes);
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // 4 x K=16 inside the 128-byte swizzle span
          const uint32_t first = (t > 0 || k > 0) ? 1u : 0u;
          if constexpr (MERGED) {
            tc::mma_bf16(tmem, a0 + 2 * k, bh + 2 * k, idesc, first);
            tc::mma_bf16(acc1, a1 + 2 * k, bh + 2 * k, idesc, first);
            continue;
          }
          tc::mma_bf16(tmem, a0 + 2 * k, bh + 2 * k, idesc, first);
          tc::mma_bf16(tmem, a0 + 2 * k, bl + 2 * k, idesc, 1u);
          tc::mma_bf16(acc1, a1 + 2 * k, bh + 2 * k, idesc, first);
          tc::mma_bf16(acc1, a1 + 2 * k, bl + 2 * k, idesc, 1u);
        }
        tc::commit(&empty_a[s]);
        tc::commit(&empty_b[r]);
      }
      tc::commit(accum);  // arrives once every issued MMA has completed
    }
  } else {
    // ------------------------------------------------ KR generators (8 warps)
    constexpr int CPT = 8 / TPR;          // 16-byte chunks (8 columns each) per thread
    const int gt = threadIdx.x - 64;
    const int g = gt / TPR;               // row b of the KR tile
    const int part = gt - g * TPR;        // this thread's chunks: part*CPT .. part*CPT + CPT-1
    const bool row_on = g < p.btile;
    const int64_t bglob = (int64_t)col_tile * p.btile + (row_on ? g : 0);
    const float* prow = p.pb + bglob * p.np;
    const float* urow = p.qb + bglob * p.np + part * CPT * 8;
    float uk[8 * CPT];
    int64_t cur_kb = -1;
    // u_bj of the next K2_PF K-tiles, in a ring indexed by t mod K2_PF
    float ring[K2_PF];
#pragma unroll
    for (int q = 0; q < K2_PF; ++q) ring[q] = (row_on && q < T) ? prow[k2_j(q, nj, j0)] : 0.f;
    bool stop = false;
    for (int64_t t0 = 0; t0 < T && !stop; t0 += K2_PF) {
#pragma unroll
      for (int q = 0; q < K2_PF; ++q) {
        const int64_t t = t0 + q;
        if (t >= T) break;
        const int r = (int)(t % SB);
        const uint32_t ph = (uint32_t)((t / SB) & 1);
        const int64_t kb = t / nj;
        const float uj = ring[q];
        if (row_on && t + K2_PF < T) ring[q] = prow[k2_j(t + K2_PF, nj, j0)];
        if (row_on && kb != cur_kb) {
          const float4* src = reinterpret_cast<const float4*>(urow + kb * 64);
#pragma unroll
          for (int v = 0; v < 2 * CPT; ++v) {
            const float4 x = src[v];
            uk[4 * v] = x.x; uk[4 * v + 1] = x.y; uk[4 * v + 2] = x.z; uk[4 * v + 3] = x.w;
          }
          cur_kb = kb;
        }
        // warp-uniform (the warp stores and arrives together)
        if (t >= SB && !__all_sync(0xffffffffu, ptx::mbar_wait(&empty_b[r], ph ^ 1u, abort_flag))) {
          if (lane == 0) k2_abort(abort_flag, p.err);
          stop = true;
          break;
        }
        if (row_on) {
          uint8_t* row_hi = sb + (size_t)r * b_bytes + (size_t)g * 128;
          uint8_t* row_lo = row_hi + half_bytes;
#pragma unroll
          for (int cc = 0; cc < CPT; ++cc) {
            const int c = part * CPT + cc;  // chunk of the row
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float p0 = uk[8 * cc + 2 * h] * uj, p1 = uk[8 * cc + 2 * h + 1] * uj;
              const __nv_bfloat162 hi = __floats2bfloat162_rn(p0, p1);
              const float2 hf = __bfloat1622float2(hi);
              const __nv_bfloat162 lo = __floats2bfloat162_rn(p0 - hf.x, p1 - hf.y);
              wh[h] = *reinterpret_cast<const uint32_t*>(&hi);
              wl[h] = *reinterpret_cast<const uint32_t*>(&lo);
            }
            const int off = (c ^ (g & 7)) << 4;
            *reinterpret_cast<uint4*>(row_hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4*>(row_lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
          }
        }
        ptx::fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&full_b[r]);
      }
    }
    // -------------------------------------------------------------- epilogue
    if (warp >= 2 && warp < 6) {
      // warp-uniform: the tensor-memory loads below are collective
      const bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(accum, 0, nullptr));
      if (!ok && lane == 0) atomicOr(p.err, DEV_ERR_TIMEOUT);
      tc::fence_after_sync();
      const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 are readable by this warp
      if (ok && !__any_sync(0xffffffffu, *abort_flag != 0)) {
        for (int m = 0; m < K2_MT; ++m) {
          const int64_t i = (int64_t)i_pair * 256 + m * 128 + 32 * q + lane;
          for (int c0 = 0; c0 < p.btile; c0 += 32) {
            uint32_t rr[32];
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            if constexpr (!MERGED) {
              tc::tmem_ld_32x32b_x32(tmem + lanes + (uint32_t)(m * p.btile + c0), rr);
              tc::tmem_ld_wait();
            } else if (p.btile >= 32) {
              // hi part + lo part of columns c0 .. c0+31
              uint32_t rl[32];
              const uint32_t base = tmem + lanes + (uint32_t)(m * 2 * p.btile);
              tc::tmem_ld_32x32b_x32(base + (uint32_t)c0, rr);
              tc::tmem_ld_32x32b_x32(base + (uint32_t)(p.btile + c0), rl);
              tc::tmem_ld_wait();
#pragma unroll
              for (int v = 0; v < 32; ++v) rr[v] = __float_as_uint(__uint_as_float(rr[v]) + __uint_as_float(rl[v]));
            } else {
              // btile = 16: one load holds the hi (0..15) and lo (16..31) columns
              tc::tmem_ld_32x32b_x32(tmem + lanes + (uint32_t)(m * 2 * p.btile), rr);
              tc::tmem_ld_wait();
#pragma unroll
              for (int v = 0; v < 16; ++v) rr[v] = __float_as_uint(__uint_as_float(rr[v]) + __uint_as_float(rr[16 + v]));
            }
            if (i < p.n) {
              float* dst = p.part + ((int64_t)split * p.n + i) * p.bp + (int64_t)col_tile * p.btile + c0;
              const int mm = p.btile - c0 < 32 ? p.btile - c0 : 32;
              if (mm == 32) {
#pragma unroll
                for (int v = 0; v < 8; ++v)
                  reinterpret_cast<float4*>(dst)[v] =
                      make_float4(__uint_as_float(rr[4 * v]), __uint_as_float(rr[4 * v + 1]),
                                  __uint_as_float(rr[4 * v + 2]), __uint_as_float(rr[4 * v + 3]));
              } else {
#pragma unroll
                for (int v = 0; v < 32; ++v)
                  if (v < mm) dst[v] = __uint_as_float(rr[v]);
              }
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
  }
}

// qb[b][k] = u_b[k] (FP32), zero for padding rows/columns and inactive
// trajectories; with factors, pb[b][k] = P[k][b] and qb[b][k] = Q[k][b]
// (P, Q row-major n x f_stride).
__global__ void k2_prep_kernel(const K2Dev p, const double* u, int64_t u_stride, const double* hist,
                               const int64_t* taken, int64_t hist_stride, const int32_t* active, int batch,
                               const double* fp, const double* fq, int64_t f_stride) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.bp * p.np) return;
  const int64_t b = t / p.np, k = t - b * p.np;
  const bool in = b < batch && k < p.n;
  if (fq) {
    p.qb[t] = in ? __double2float_rn(fq[k * f_stride + b]) : 0.f;
    p.pb[t] = in ? __double2float_rn(fp[k * f_stride + b]) : 0.f;
    return;
  }
  float v = 0.f;
  if (in && (active == nullptr || active[b])) {
    const double* ub = taken ? hist + b * hist_stride + (taken[b] % 3) * p.n : u + b * u_stride;
    v = __double2float_rn(ub[k]);
  }
  p.qb[t] = v;
}

// c[b][i] = sum over splits of the FP32 partials, in split order, in FP64.
__global__ void k2_reduce_kernel(const K2Dev p, double* c, int64_t c_stride, double* hist, const int64_t* taken,
                                 int64_t hist_stride, const int32_t* active, int batch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * p.n) return;
  const int64_t i = t / batch, b = t - i * batch;  // consecutive threads: consecutive b (coalesced reads)
  if (active && !active[b]) return;
  // loads issued eight at a time, added in split order
  const float* src = p.part + i * p.bp + b;
  const int64_t stride = p.n * p.bp;
  double s = 0.0;
  int q = 0;
  for (; q + 8 <= p.splits; q += 8) {
    float v[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) v[x] = src[(q + x) * stride];
#pragma unroll
    for (int x = 0; x < 8; ++x) s += (double)v[x];
  }
  for (; q < p.splits; ++q) s += (double)src[q * stride];
  double* dst = taken ? hist + b * hist_stride + (3 + taken[b] % 3) * p.n : c + b * c_stride;
  dst[i] = s;
}

// ------------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// Tile-major copy: tile t = (i_pair * n + j) * (np / 64) + kb holds rows
// i_pair*256 .. +255 of columns j*np + kb*64 .. +63 of C_(1), 256 rows of 128
// bytes, contiguous (rows past n are zero).
__global__ void k_k2_tiles(const __nv_bfloat16* __restrict__ rows, int64_t n, int64_t np, int64_t tiles,
                           __nv_bfloat16* __restrict__ out) {
  const int64_t total = tiles * 256 * 8;  // 16-byte vectors
  const int64_t kblocks = np / 64;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = v / (256 * 8), r = (v / 8) % 256, c = v % 8;
    const int64_t kb = t % kblocks, j = (t / kblocks) % n, ip = t / (kblocks * n);
    const int64_t i = ip * 256 + r;
    uint4 x = make_uint4(0, 0, 0, 0);
    if (i < n) x = *reinterpret_cast<const uint4*>(rows + (i * n + j) * np + kb * 64 + c * 8);
    *reinterpret_cast<uint4*>(out + (t * 256 + r) * 64 + c * 8) = x;
  }
}

size_t k2_tiles_bytes(int64_t n) {
  const int64_t np = padded_n(n), i_tiles = (n + 255) / 256;
  return (size_t)(i_tiles * n * (np / 64)) * 256 * 64 * sizeof(__nv_bfloat16);
}

cudaError_t k2_build_tiles(const void* rows, int64_t n, void* tiles, cudaStream_t s) {
  const int64_t np = padded_n(n), i_tiles = (n + 255) / 256;
  const int64_t nt = i_tiles * n * (np / 64);
  const int64_t total = nt * 256 * 8;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  k_k2_tiles<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(rows), n, np, nt,
                                               reinterpret_cast<__nv_bfloat16*>(tiles));
  return cudaGetLastError();
}

bool k2_make_tmap_tiled(CUtensorMap* m, const void* tiles, int64_t n) {
  auto fn = tmap_encode_fn();
  if (!fn) return false;
  const int64_t np = padded_n(n), i_tiles = (n + 255) / 256;
  cuuint64_t dims[2] = {64, (cuuint64_t)(i_tiles * n * (np / 64) * 256)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {64, 256};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(tiles), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool k2_make_tmap(CUtensorMap* m, const void* tensor, int64_t n, int64_t np) {
  auto fn = tmap_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(n * np), (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)(n * np * 2)};
  cuuint32_t box[2] = {64, 256};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(tensor), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

K2Plan k2_plan(int64_t n, int batch, int sm_count, int splits_force) {
  K2Plan p{};
  p.n = n;
  p.np = padded_n(n);
  int btile = (batch + 15) / 16 * 16;
  if (btile > 256) btile = 256;
  p.btile = btile;
  p.col_tiles = (batch + btile - 1) / btile;
  p.i_tiles = (int)((n + 255) / 256);  // pairs of 128-row tiles
  const int tiles = p.col_tiles * p.i_tiles;
  int splits = sm_count / tiles;
  if (splits < 1) splits = 1;
  if (splits_force > 0) splits = splits_force;
  if (splits > n) splits = (int)n;
  p.splits = splits;
  const int b_bytes = 2 * btile * 128;  // hi and lo KR tiles
  p.stages_b = btile >= 128 ? 2 : 4;
  int sa = (int)((200 * 1024 - p.stages_b * b_bytes) / K2_A_BYTES);
  if (sa > 6) sa = 6;
  if (sa < 2) sa = 2;
  p.stages_a = sa;
  int cols = 32;
  const int acc_cols = btile <= 128 ? 4 * btile : 2 * btile;  // two accumulators (hi|lo side by side when merged)
  while (cols < acc_cols) cols <<= 1;
  p.tmem_cols = cols;
  p.smem = 1024 + (size_t)sa * K2_A_BYTES + (size_t)p.stages_b * b_bytes + (size_t)(2 * sa + 2 * p.stages_b + 1) * 8 + 16;
  p.bp = (int64_t)p.col_tiles * btile;
  return p;
}

// FP32 operand rows (two arrays, the second used for factor pairs) and the
// split-K partials.
size_t k2_scratch_bytes(const K2Plan& p) {
  return 4 * (2 * (size_t)p.bp * p.np + (size_t)p.splits * p.n * p.bp);
}

size_t k2_scratch_need(int64_t n, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = 16; b - 16 < max_batch; b += 16)
    need = std::max(need, k2_scratch_bytes(k2_plan(n, b < max_batch ? b : max_batch, sm_count)));
  return need;
}

cudaError_t k2_launch(const K2Plan& p, const CUtensorMap* tmap, const K2Args& a, cudaStream_t s) {
  K2Dev d{};
  d.tiled = a.tiled;
  d.n = p.n;
  d.np = p.np;
  d.btile = p.btile;
  d.col_tiles = p.col_tiles;
  d.i_tiles = p.i_tiles;
  d.splits = p.splits;
  d.stages_a = p.stages_a;
  d.stages_b = p.stages_b;
  d.tmem_cols = p.tmem_cols;
  d.bp = p.bp;
  d.qb = reinterpret_cast<float*>(a.scratch);
  d.pb = a.fq ? d.qb + p.bp * p.np : d.qb;
  d.part = d.qb + 2 * p.bp * p.np;
  d.err = a.err;
  const int64_t prep = p.bp * p.np;
  k2_prep_kernel<<<(unsigned)((prep + 255) / 256), 256, 0, s>>>(d, a.u, a.u_stride, a.hist, a.taken, a.hist_stride,
                                                                a.active, a.batch, a.fp, a.fq, a.f_stride);
  int tpr = 1;  // largest power of two <= 256 / btile, at most 8
  while (tpr < 8 && 2 * tpr * p.btile <= 256) tpr *= 2;
  auto kern = tpr == 8 ? k2_tc_kernel<8> : tpr == 4 ? k2_tc_kernel<4> : tpr == 2 ? k2_tc_kernel<2> : k2_tc_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  if (a.ev0) prof_record(a.ev0, s);
  kern<<<(unsigned)(p.i_tiles * p.col_tiles * p.splits), K2_THREADS, p.smem, s>>>(*tmap, d);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.ev1) prof_record(a.ev1, s);
  const int64_t red = (int64_t)a.batch * p.n;
  k2_reduce_kernel<<<(unsigned)((red + 255) / 256), 256, 0, s>>>(d, a.c, a.c_stride, a.hist, a.taken, a.hist_stride,
                                                                 a.active, a.batch);
  return cudaGetLastError();
}

}  // namespace grom
