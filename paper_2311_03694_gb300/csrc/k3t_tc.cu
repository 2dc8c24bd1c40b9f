// K3T: the CP-form advection term of a batch of trajectories on the tcgen05
// tensor cores (BF16 factor storage).
//
//   general:  [P; Q]    = [B C]^T X,     Z = P o Q,              c = A Z
//   skew:     [P; Q; S] = [V W U]^T X,   Z = [P o Q; P o S],     c = [U, -W] Z
//
// (Sec. 3.1, eq. tc_ap; the skew structure of Sec. 3.3, eq. skew_abc_struct,
// evaluated without its repeated blocks), X = [u_1 .. u_B].  Both
// contractions run on one GEMM kernel D = A_op (B_hi + B_lo)^T:
//   * A_op is BF16 and K-major: for the projections FT, the transposed factors
//     stacked (nseg * Rp rows of Np), for the expansion AE = A or [U | -W]
//     (n rows of nz * Rp); both are gathered once from the stored BF16
//     factors, so they hold the same values the SIMT kernels read;
//   * B_op is the states (then the Hadamard products) split into BF16 hi and
//     lo parts, side by side in shared memory, so one MMA of N = 2 btile
//     multiplies both (the operand exact to ~2^-17);
//   * FP32 accumulation in tensor memory; the epilogue adds the hi and lo
//     halves and stores FP32 rows (split-K partials when the output tiles
//     alone cannot fill the GPU).
// A Hadamard kernel sums the projection splits, forms Z and transposes it
// into hi/lo rows; a finish kernel sums the expansion splits in a fixed
// order in FP64 into the output or the advection slot of the history ring.
//
// CTA (6 warps): warp 0 issues the TMA loads (a 128 x 64 A box, two btile x
// 64 B boxes per K step), warp 1 owns the tensor memory and issues
// tcgen05.mma (M = 128, N = 2 btile, K = 16), warps 2-5 read the accumulator
// back.
#include <cudaTypedefs.h>

#include <algorithm>

#include "grom_internal.h"
#include "tc.cuh"

namespace grom {

constexpr int K3T_THREADS = 192;
constexpr int K3T_A_BYTES = 128 * 64 * 2;  // 128 rows x 64 K
constexpr int K3T_SMEM_MAX = 232448;

struct K3TGemm {
  int64_t M, K, bp;  // A rows, contraction length (multiple of 64), padded batch
  int btile, mtiles, ctiles, splits, stages, tmem_cols;
  float* out;        // splits x M x bp
  int* err;
};

__device__ __forceinline__ void k3t_abort(volatile int* abort_flag, int* err) {
  *abort_flag = 1;
  atomicOr(err, DEV_ERR_TIMEOUT);
}

__global__ void __launch_bounds__(K3T_THREADS, 1)
    k3t_gemm(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_bh,
             const __grid_constant__ CUtensorMap tmap_bl, const K3TGemm g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int S = g.stages;
  const int b_half = g.btile * 128;
  const int stage_b = 2 * b_half;
  uint8_t* sa = smem;
  uint8_t* sb = sa + (size_t)S * K3T_A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sb + (size_t)S * stage_b);
  uint64_t* empty = full + S;
  uint64_t* accum = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x % g.splits;
  const int rest = blockIdx.x / g.splits;
  const int ct = rest % g.ctiles, mt = rest / g.ctiles;
  const int64_t kblocks = g.K / 64;
  const int64_t kb0 = (int64_t)split * kblocks / g.splits, kb1 = ((int64_t)split + 1) * kblocks / g.splits;
  const int64_t T = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(accum, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_bh);
    tc::prefetch_tmap(&tmap_bl);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, (uint32_t)g.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int64_t t = 0;
      for (; t < T; ++t) {
        const int s = (int)(t % S);
        if (t >= S && !ptx::mbar_wait(&empty[s], (uint32_t)(((t / S) & 1) ^ 1), abort_flag)) {
          k3t_abort(abort_flag, g.err);
          break;
        }
        const int32_t x = (int32_t)((kb0 + t) * 64);
        ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)(K3T_A_BYTES + stage_b));
        tc::tma_load_2d(sa + (size_t)s * K3T_A_BYTES, &tmap_a, x, mt * 128, &full[s]);
        uint8_t* b = sb + (size_t)s * stage_b;
        tc::tma_load_2d(b, &tmap_bh, x, ct * g.btile, &full[s]);
        tc::tma_load_2d(b + b_half, &tmap_bl, x, ct * g.btile, &full[s]);
      }
      for (int64_t q = t > S ? t - S : 0; q < t; ++q)
        if (!ptx::mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), nullptr)) atomicOr(g.err, DEV_ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(128, 2 * g.btile);  // hi | lo
      for (int64_t t = 0; t < T; ++t) {
        const int s = (int)(t % S);
        if (!ptx::mbar_wait(&full[s], (uint32_t)((t / S) & 1), abort_flag)) {
          k3t_abort(abort_flag, g.err);
          break;
        }
        tc::fence_after_sync();
        const uint64_t ad = tc::sw128_kmajor_desc(sa + (size_t)s * K3T_A_BYTES);
        const uint64_t bd = tc::sw128_kmajor_desc(sb + (size_t)s * stage_b);  // 2 btile rows
#pragma unroll
        for (int k = 0; k < 4; ++k) tc::mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (t > 0 || k > 0) ? 1u : 0u);
        tc::commit(&empty[s]);
      }
      tc::commit(accum);  // arrives once every issued MMA has completed
    }
  } else {
    // ----------------------------------------------------- epilogue (warps 2-5)
    const bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(accum, 0, nullptr));
    if (!ok && lane == 0) atomicOr(g.err, DEV_ERR_TIMEOUT);
    tc::fence_after_sync();
    const int q = warp & 3;
    if (ok && T > 0 && !__any_sync(0xffffffffu, *abort_flag != 0)) {
      const int64_t m = (int64_t)mt * 128 + 32 * q + lane;
      const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16);
      float* dst = g.out + ((int64_t)split * g.M + m) * g.bp + (int64_t)ct * g.btile;
      for (int c0 = 0; c0 < g.btile; c0 += 32) {
        uint32_t v[32], w[32];
        if (g.btile == 16) {
          tc::tmem_ld_32x32b_x32(acc, v);  // hi 0..15 | lo 16..31
#pragma unroll
          for (int c = 0; c < 32; ++c) w[c] = v[(c + 16) & 31];
        } else {
          tc::tmem_ld_32x32b_x32(acc + (uint32_t)c0, v);
          tc::tmem_ld_32x32b_x32(acc + (uint32_t)(g.btile + c0), w);
        }
        tc::tmem_ld_wait();
        if (m < g.M) {
          const int nb = g.btile - c0 < 32 ? g.btile - c0 : 32;
          if (nb == 32) {
#pragma unroll
            for (int c = 0; c < 32; c += 4)
              *reinterpret_cast<float4*>(dst + c0 + c) = make_float4(
                  __uint_as_float(v[c]) + __uint_as_float(w[c]), __uint_as_float(v[c + 1]) + __uint_as_float(w[c + 1]),
                  __uint_as_float(v[c + 2]) + __uint_as_float(w[c + 2]),
                  __uint_as_float(v[c + 3]) + __uint_as_float(w[c + 3]));
          } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) dst[c0 + c] = __uint_as_float(v[c]) + __uint_as_float(w[c]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)g.tmem_cols);
  }
}

// States into BF16 hi/lo rows xh, xl (bp x np), zero for padding and inactive
// trajectories; grid (np / 256, bp).
__global__ void k3t_prep(const K3Args a, int64_t n, int64_t np, int64_t bp, int batch, __nv_bfloat16* xh,
                         __nv_bfloat16* xl) {
  const int64_t b = blockIdx.y, k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int64_t t = b * np + k;
  float v = 0.f;
  if (b < batch && k < n && (a.active == nullptr || a.active[b])) {
    const double* ub = a.taken ? a.hist + b * a.hist_stride + (a.taken[b] % 3) * n : a.u + b * a.u_stride;
    v = __double2float_rn(ub[k]);
  }
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  xh[t] = hi;
  xl[t] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Z[b][j] (BF16 hi/lo, bp x kz) from the projection partials d1 (s1 x m1 x
// bp, rows P | Q | S of rp each): Z[b][j] = P_j Q_j for j < rp and, in the
// skew form (kz = 2 rp), Z[b][rp + j] = P_j S_j; 32 x 32 tiles through shared
// memory (coalesced reads along b, writes along j).
__global__ void k3t_hadamard(const float* __restrict__ d1, int s1, int64_t m1, int64_t rp, int64_t bp, int64_t kz,
                             __nv_bfloat16* zh, __nv_bfloat16* zl) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t j0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
  for (int jj = ty; jj < 32; jj += 8) {
    const int64_t j = j0 + jj, b = b0 + tx;
    float z = 0.f;
    if (j < kz && b < bp) {
      const int64_t jp = j < rp ? j : j - rp;            // column of P
      const int64_t jo = j < rp ? rp + j : 2 * rp + jp;   // row of Q, or of S (skew, second half)
      float p = 0.f, o = 0.f;
      for (int s = 0; s < s1; ++s) {
        p += d1[((int64_t)s * m1 + jp) * bp + b];
        o += d1[((int64_t)s * m1 + jo) * bp + b];
      }
      z = p * o;
    }
    tile[jj][tx] = z;
  }
  __syncthreads();
  for (int bb = ty; bb < 32; bb += 8) {
    const int64_t b = b0 + bb, j = j0 + tx;
    if (b < bp && j < kz) {
      const float z = tile[tx][bb];
      const __nv_bfloat16 hi = __float2bfloat16_rn(z);
      zh[b * kz + j] = hi;
      zl[b * kz + j] = __float2bfloat16_rn(z - __bfloat162float(hi));
    }
  }
}

// c[b][i] = sum over splits of d2[split][i][b], in split order, in FP64.
// Consecutive threads take consecutive b: the reads are coalesced, the
// writes land 6 n doubles apart (a 32 x 32 shared-memory transpose for
// coalesced writes was measured slower: a quarter of the threads).
__global__ void k3t_finish(const float* __restrict__ d2, int s2, int64_t n, int64_t m2, int64_t bp, const K3Args a,
                           int batch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * n) return;
  const int64_t i = t / batch, b = t - i * batch;
  if (a.active && !a.active[b]) return;
  double s = 0.0;
  for (int q = 0; q < s2; ++q) s += (double)d2[((int64_t)q * m2 + i) * bp + b];
  double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * n : a.c + b * a.c_stride;
  dst[i] = s;
}

// FT and AE from the stored BF16 factors fa, fb, fc (row-major n x rb).
__global__ void k3t_build(const __nv_bfloat16* __restrict__ fa, const __nv_bfloat16* __restrict__ fb,
                          const __nv_bfloat16* __restrict__ fc, int64_t n, int64_t rb, int64_t R, int64_t rp,
                          int64_t np, int skew, __nv_bfloat16* __restrict__ ft, __nv_bfloat16* __restrict__ ae) {
  const int nseg = skew ? 3 : 2, nz = skew ? 2 : 1;
  const int64_t kz = nz * rp, nft = nseg * rp * np, nae = n * kz;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nft + nae; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nft) {
      const int64_t row = t / np, k = t - row * np, seg = row / rp, q = row - seg * rp;
      // projection rows: general B^T, C^T; skew V^T, W^T, U^T
      const __nv_bfloat16* f = seg == 0 ? fb : seg == 1 ? fc : fa;
      ft[t] = (q < R && k < n) ? f[k * rb + q] : zero;
    } else {
      const int64_t e = t - nft, i = e / kz, j = e - i * kz;
      __nv_bfloat16 v = zero;
      if (j < rp) {
        if (j < R) v = fa[i * rb + j];                   // A, or U
      } else if (j - rp < R) {
        v = __hneg(fc[i * rb + (j - rp)]);               // -W
      }
      ae[e] = v;
    }
  }
}

// ------------------------------------------------------------------- host
// rows x cols BF16, row-major, boxes of box_rows x 64.
static bool k3t_tmap(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int box_rows) {
  auto fn = tmap_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Largest split of a K range of kblocks 64-wide blocks: at least 4 K steps per split.
static int k3t_split_max(int64_t kblocks) { return (int)(kblocks / 4 > 1 ? kblocks / 4 : 1); }

// Splits of one GEMM: enough CTAs to cover the SMs, within k3t_split_max;
// `force` in [1, k3t_split_max] replaces the rule.
static int k3t_splits(int64_t tiles, int64_t kblocks, int sm_count, int force) {
  const int kmax = k3t_split_max(kblocks);
  if (force >= 1 && force <= kmax) return force;
  int s = (int)(sm_count / (tiles > 0 ? tiles : 1));
  if (s > kmax) s = kmax;
  return s < 1 ? 1 : s;
}

K3TPlan k3t_plan(int64_t n, int64_t r, int form, int batch, int sm_count, int s1_force, int s2_force) {
  K3TPlan p{};
  p.n = n;
  p.np = padded_n(n);
  p.r = r;
  p.rp = (r + 63) / 64 * 64;
  const bool skew = form == GROM_FORM_CP_SKEW;
  p.nseg = skew ? 3 : 2;
  p.nz = skew ? 2 : 1;
  p.m1 = p.nseg * p.rp;
  p.k1 = p.np;
  p.m2 = n;
  p.k2 = p.nz * p.rp;
  int btile = (batch + 15) / 16 * 16;
  if (btile > 128) btile = 128;
  p.btile = btile;
  p.ctiles = (batch + btile - 1) / btile;
  p.bp = (int64_t)p.ctiles * btile;
  const int64_t mt1 = (p.m1 + 127) / 128, mt2 = (p.m2 + 127) / 128;
  p.s1 = k3t_splits(mt1 * p.ctiles, p.k1 / 64, sm_count, s1_force);
  p.s2 = k3t_splits(mt2 * p.ctiles, p.k2 / 64, sm_count, s2_force);
  p.s1_max = k3t_split_max(p.k1 / 64);
  p.s2_max = k3t_split_max(p.k2 / 64);
  const int stage = K3T_A_BYTES + 2 * btile * 128;
  int st = (int)((K3T_SMEM_MAX - 1024 - 256) / stage);
  if (st > 6) st = 6;
  p.stages = st;
  p.smem = 1024 + (size_t)st * stage + (size_t)(2 * st + 1) * 8 + 16;
  int cols = 32;
  while (cols < 2 * btile) cols <<= 1;
  p.tmem_cols = cols;
  return p;
}

// xh | xl | d1 partials | zh | zl | d2 partials
size_t k3t_scratch_bytes(const K3TPlan& p) {
  return 2 * (size_t)p.bp * p.np * 2 + 4 * (size_t)p.s1 * p.m1 * p.bp + 2 * (size_t)p.bp * p.k2 * 2 +
         4 * (size_t)p.s2 * p.m2 * p.bp;
}

size_t k3t_scratch_need(int64_t n, int64_t r, int form, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = 16; b - 16 < max_batch; b += 16)
    need = std::max(need, k3t_scratch_bytes(k3t_plan(n, r, form, b < max_batch ? b : max_batch, sm_count)));
  return need;
}

size_t k3t_factor_bytes(int64_t n, int64_t r, int form) {
  const K3TPlan p = k3t_plan(n, r, form, 16, 1);
  return ((size_t)p.m1 * p.np + (size_t)n * p.k2) * 2;
}

cudaError_t k3t_build_factors(const void* fa, const void* fb, const void* fc, int64_t n, int64_t rb, int64_t r,
                              int form, void* ft, void* ae, cudaStream_t s) {
  const K3TPlan p = k3t_plan(n, r, form, 16, 1);
  const int64_t total = p.m1 * p.np + n * p.k2;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  k3t_build<<<(unsigned)blocks, 256, 0, s>>>(
      reinterpret_cast<const __nv_bfloat16*>(fa), reinterpret_cast<const __nv_bfloat16*>(fb),
      reinterpret_cast<const __nv_bfloat16*>(fc), n, rb, r, p.rp, p.np, form == GROM_FORM_CP_SKEW ? 1 : 0,
      reinterpret_cast<__nv_bfloat16*>(ft), reinterpret_cast<__nv_bfloat16*>(ae));
  return cudaGetLastError();
}

bool k3t_make_tmaps(CUtensorMap* m_ft, CUtensorMap* m_ae, const void* ft, const void* ae, int64_t n, int64_t r,
                    int form) {
  const K3TPlan p = k3t_plan(n, r, form, 16, 1);
  return k3t_tmap(m_ft, ft, p.np, p.m1, 128) && k3t_tmap(m_ae, ae, p.k2, n, 128);
}

static cudaError_t k3t_gemm_launch(const K3TPlan& p, const CUtensorMap* ma, const void* bh, const void* bl,
                                   int64_t M, int64_t K, int splits, float* out, int* err, cudaStream_t s) {
  CUtensorMap mh, ml;
  if (!k3t_tmap(&mh, bh, K, p.bp, p.btile) || !k3t_tmap(&ml, bl, K, p.bp, p.btile)) return cudaErrorInvalidValue;
  K3TGemm g{};
  g.M = M;
  g.K = K;
  g.bp = p.bp;
  g.btile = p.btile;
  g.mtiles = (int)((M + 127) / 128);
  g.ctiles = p.ctiles;
  g.splits = splits;
  g.stages = p.stages;
  g.tmem_cols = p.tmem_cols;
  g.out = out;
  g.err = err;
  cudaError_t e = cudaFuncSetAttribute(k3t_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  k3t_gemm<<<(unsigned)(g.mtiles * g.ctiles * splits), K3T_THREADS, p.smem, s>>>(*ma, mh, ml, g);
  return cudaGetLastError();
}

cudaError_t k3t_launch(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a, int batch,
                       void* scratch, int* err, cudaStream_t s) {
  __nv_bfloat16* xh = reinterpret_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* xl = xh + p.bp * p.np;
  float* d1 = reinterpret_cast<float*>(xl + p.bp * p.np);
  __nv_bfloat16* zh = reinterpret_cast<__nv_bfloat16*>(d1 + (size_t)p.s1 * p.m1 * p.bp);
  __nv_bfloat16* zl = zh + p.bp * p.k2;
  float* d2 = reinterpret_cast<float*>(zl + p.bp * p.k2);
  k3t_prep<<<dim3((unsigned)((p.np + 255) / 256), (unsigned)p.bp), 256, 0, s>>>(a, p.n, p.np, p.bp, batch, xh, xl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = k3t_gemm_launch(p, m_ft, xh, xl, p.m1, p.k1, p.s1, d1, err, s)) != cudaSuccess) return e;
  dim3 hg((unsigned)((p.bp + 31) / 32), (unsigned)((p.k2 + 31) / 32));
  k3t_hadamard<<<hg, 256, 0, s>>>(d1, p.s1, p.m1, p.rp, p.bp, p.k2, zh, zl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = k3t_gemm_launch(p, m_ae, zh, zl, p.m2, p.k2, p.s2, d2, err, s)) != cudaSuccess) return e;
  const int64_t fin = (int64_t)batch * p.n;
  k3t_finish<<<(unsigned)((fin + 255) / 256), 256, 0, s>>>(d2, p.s2, p.n, p.m2, p.bp, a, batch);
  return cudaGetLastError();
}

}  // namespace grom
