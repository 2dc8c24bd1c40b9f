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
// The projections run as one fused kernel (k3t_proj): a CTA owns 128 rank
// indices j and one column tile of trajectories and issues the P, Q (and S)
// MMAs of those j into separate tensor-memory accumulators that share the
// state tile, so its epilogue forms Z = P o Q (and P o S) itself and writes
// the hi/lo rows of the expansion's B operand (with split K, the last CTA of
// a tile to arrive sums the splits' partials in split order).  The expansion
// (k3t_gemm) writes its partials trajectory-major, and the step kernel sums
// them in FP64 in split order while it steps (k_step_diag_mc, K3T mode),
// writing the next state's BF16 hi/lo rows as it goes; a finish kernel does
// the same sum for the plain evaluation (grom_nonlinear).  Per step: the
// projection kernel, the expansion and the step; the state prep runs once
// per call.
//
// CTA (6 warps): warp 0 issues the TMA loads (128 x 64 A boxes, two btile x
// 64 B boxes per K step), warp 1 owns the tensor memory and issues
// tcgen05.mma (M = 128, N = 2 btile, K = 16), warps 2-5 read the
// accumulators back.
#include <cudaTypedefs.h>

#include <algorithm>

#include "grom_internal.h"
#include "step_mc.cuh"
#include "tc.cuh"

namespace grom {

constexpr int K3T_THREADS = 192;
constexpr int K3T_PROJ_MAX_SPLITS = 8;  // K splits of the projection kernel (its last-CTA reduction holds them all)
constexpr int K3T_A_BYTES = 128 * 64 * 2;  // 128 rows x 64 K
constexpr int K3T_SMEM_MAX = 232448;

struct K3TGemm {
  int64_t M, K, bp;  // A rows, contraction length (multiple of 64), padded batch
  int btile, mtiles, ctiles, splits, stages, tmem_cols;
  float* out;        // splits x bp x M (trajectory-major)
  int* err;
};

struct K3TProj {
  int64_t rp, bp, kz, K;  // padded rank, padded batch, Z row length (nz rp), K = np
  int nseg, btile, jtiles, ctiles, splits, stages, tmem_cols;
  float* part;            // splits > 1: one block per (split, rank tile, column tile) of btile x 3 x 128 floats
  unsigned int* cnt;      // jtiles x ctiles arrival counters, zero between launches
  __nv_bfloat16* zh;      // bp x kz hi rows of Z
  __nv_bfloat16* zl;      // lo rows
  int* err;
};

__device__ __forceinline__ void k3t_abort(volatile int* abort_flag, int* err) {
  *abort_flag = 1;
  atomicOr(err, DEV_ERR_TIMEOUT);
}

// One pipeline ring of a tcgen05 GEMM: S stage slots, each stage_a bytes of
// A boxes and stage_b bytes of the hi/lo B boxes, with full/empty barriers
// and the accumulator barrier.  The roles count the K steps they have
// handled (`it`) across tiles, so a CTA can run several tiles, and the
// persistent stepper several phases, on one ring without re-arming it.
struct K3TRing {
  uint8_t* sa;
  uint8_t* sb;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* accum;
  int S, stage_a, stage_b;
};

__device__ __forceinline__ K3TRing k3t_ring(uint8_t* base, uint64_t* bars, int S, int na, int btile) {
  K3TRing R;
  R.S = S;
  R.stage_a = na * K3T_A_BYTES;
  R.stage_b = 2 * btile * 128;
  R.sa = base;
  R.sb = base + (size_t)S * R.stage_a;
  R.full = bars;
  R.empty = bars + S;
  R.accum = bars + 2 * S;
  return R;
}

__device__ __forceinline__ void k3t_ring_init(const K3TRing& R) {
  for (int s = 0; s < R.S; ++s) {
    ptx::mbar_init(&R.full[s], 1);
    ptx::mbar_init(&R.empty[s], 1);
  }
  ptx::mbar_init(R.accum, 1);
}

// TMA producer of one tile (one thread): T K steps of na A boxes (rows
// a_row + seg a_step of ta) and the hi/lo B boxes (rows b_row).
__device__ __forceinline__ void k3t_produce(const K3TRing& R, const CUtensorMap* ta, const CUtensorMap* tbh,
                                            const CUtensorMap* tbl, int na, int32_t a_row, int32_t a_step,
                                            int32_t b_row, int64_t kb0, int64_t T, uint32_t& it,
                                            volatile int* abort_flag, int* err) {
  const int b_half = R.stage_b / 2;
  for (int64_t t = 0; t < T; ++t) {
    const uint32_t s = it % (uint32_t)R.S;
    if (it >= (uint32_t)R.S && !ptx::mbar_wait(&R.empty[s], ((it / R.S) & 1u) ^ 1u, abort_flag)) {
      k3t_abort(abort_flag, err);
      return;
    }
    const int32_t x = (int32_t)((kb0 + t) * 64);
    ptx::mbar_arrive_expect_tx(&R.full[s], (uint32_t)(R.stage_a + R.stage_b));
    uint8_t* a = R.sa + (size_t)s * R.stage_a;
    for (int seg = 0; seg < na; ++seg) tc::tma_load_2d(a + seg * K3T_A_BYTES, ta, x, a_row + seg * a_step, &R.full[s]);
    uint8_t* b = R.sb + (size_t)s * R.stage_b;
    tc::tma_load_2d(b, tbh, x, b_row, &R.full[s]);
    tc::tma_load_2d(b + b_half, tbl, x, b_row, &R.full[s]);
    ++it;
  }
}

// The last min(S, issued) loads of the ring have landed (before the CTA
// exits: no copy may still be writing its shared memory).  it0: the count
// when this CTA's producer started.
__device__ __forceinline__ void k3t_drain(const K3TRing& R, uint32_t it0, uint32_t it, int* err) {
  const uint32_t lo = it - it0 > (uint32_t)R.S ? it - (uint32_t)R.S : it0;
  for (uint32_t q = lo; q < it; ++q)
    if (!ptx::mbar_wait(&R.full[q % R.S], (q / R.S) & 1u, nullptr)) atomicOr(err, DEV_ERR_TIMEOUT);
}

// MMA issuer of one tile (one thread): per K step, each of the na A boxes
// times the B boxes (M = 128, N = 2 btile: hi | lo) into the accumulator at
// tmem + seg acc_step columns; then the accumulator barrier.
__device__ __forceinline__ void k3t_mma(const K3TRing& R, uint32_t tmem, int na, uint32_t acc_step, uint32_t idesc,
                                        int64_t T, uint32_t& it, volatile int* abort_flag, int* err) {
  for (int64_t t = 0; t < T; ++t) {
    const uint32_t s = it % (uint32_t)R.S;
    if (!ptx::mbar_wait(&R.full[s], (it / R.S) & 1u, abort_flag)) {
      k3t_abort(abort_flag, err);
      break;
    }
    tc::fence_after_sync();
    const uint64_t bd = tc::sw128_kmajor_desc(R.sb + (size_t)s * R.stage_b);  // 2 btile rows
    for (int seg = 0; seg < na; ++seg) {
      const uint64_t ad = tc::sw128_kmajor_desc(R.sa + (size_t)s * R.stage_a + seg * K3T_A_BYTES);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tc::mma_bf16(tmem + (uint32_t)seg * acc_step, ad + 2 * k, bd + 2 * k, idesc, (t > 0 || k > 0) ? 1u : 0u);
    }
    tc::commit(&R.empty[s]);
    ++it;
  }
  tc::commit(R.accum);  // arrives once every issued MMA has completed
}

// Epilogue warps (2-5) wait for the tile's accumulator; parity: the tile's
// index among the ring's tiles in this CTA.
__device__ __forceinline__ bool k3t_wait_accum(const K3TRing& R, uint32_t parity, int* err) {
  const bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(R.accum, parity, nullptr));
  if (!ok && (threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_TIMEOUT);
  tc::fence_after_sync();
  return ok;
}

// Tile coordinates of a flattened tile index: split fastest, then the column tile.
struct K3TTile {
  int split, ct, mt;
  int64_t kb0, T;
};

__device__ __forceinline__ K3TTile k3t_tile(int idx, int splits, int ctiles, int64_t K) {
  K3TTile t;
  t.split = idx % splits;
  const int rest = idx / splits;
  t.ct = rest % ctiles;
  t.mt = rest / ctiles;
  const int64_t kblocks = K / 64;
  t.kb0 = (int64_t)t.split * kblocks / splits;
  t.T = ((int64_t)t.split + 1) * kblocks / splits - t.kb0;
  return t;
}

// Expansion epilogue: lane = output row m, column = trajectory; for each
// column the 32 lanes store 32 consecutive m of that trajectory's row.
__device__ __forceinline__ void k3t_gemm_epilogue(const K3TGemm& g, uint32_t tmem, const K3TTile& tl, bool run) {
  const int q = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  if (!run) return;
  const int64_t m = (int64_t)tl.mt * 128 + 32 * q + lane;
  const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16);
  float* dst = g.out + ((int64_t)tl.split * g.bp + (int64_t)tl.ct * g.btile) * g.M + m;
  for (int c0 = 0; c0 < g.btile; c0 += 16) {
    uint32_t v[16], w[16];
    tc::tmem_ld_32x32b_x16(acc + (uint32_t)c0, v);
    tc::tmem_ld_32x32b_x16(acc + (uint32_t)(g.btile + c0), w);
    tc::tmem_ld_wait();
    if (m < g.M) {
#pragma unroll
      for (int c = 0; c < 16; ++c) dst[(int64_t)(c0 + c) * g.M] = __uint_as_float(v[c]) + __uint_as_float(w[c]);
    }
  }
}

__global__ void __launch_bounds__(K3T_THREADS, 1)
    k3t_gemm(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_bh,
             const __grid_constant__ CUtensorMap tmap_bl, const K3TGemm g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)g.stages * (K3T_A_BYTES + 2 * g.btile * 128));
  const K3TRing R = k3t_ring(smem, bars, g.stages, 1, g.btile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(R.accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const K3TTile tl = k3t_tile(blockIdx.x, g.splits, g.ctiles, g.K);

  if (threadIdx.x == 0) {
    k3t_ring_init(R);
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
    if (lane == 0) {
      uint32_t it = 0;
      k3t_produce(R, &tmap_a, &tmap_bh, &tmap_bl, 1, tl.mt * 128, 0, tl.ct * g.btile, tl.kb0, tl.T, it, abort_flag,
                  g.err);
      k3t_drain(R, 0, it, g.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0;
      k3t_mma(R, tmem, 1, 0, tc::idesc_bf16_f32(128, 2 * g.btile), tl.T, it, abort_flag, g.err);
    }
  } else {
    const bool ok = k3t_wait_accum(R, 0, g.err);
    k3t_gemm_epilogue(g, tmem, tl, ok && tl.T > 0 && !__any_sync(0xffffffffu, *abort_flag != 0));
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)g.tmem_cols);
  }
}

// K3O (k3_oz.cu): D = A B^T for the sliced FP64 CP form, in 128 x 128
// tiles.  A holds `slices` slices of mslice rows, B `slices` slices of
// nslice rows (K-major BF16 integer digits); D[col][m] is stored raw (FP32,
// exact: every product of two digits and every partial sum is an integer
// below 2^24).  Only the tiles that hold a slice pair (p, q) of the kept
// triangle p + q < slices are computed.  CTAs are persistent over tiles: the
// producer streams the next tiles' K steps through the ring while the MMAs
// fill one of two tensor-memory accumulators and the epilogue warps store
// the other.  The B tile is two 64-row boxes in the ring's hi and lo slots,
// one MMA of N = BT (128, or 256 for wide problems: half the state bytes per
// product, which the L2 has to deliver to every SM).
struct K3OGemm {
  int64_t M, K, mslice, nslice;
  int slices, mtiles, ctiles, stages;
  float* out;  // ncols x M
  int* err;
};
template <int BT>
__device__ __forceinline__ bool k3o_tile(const K3OGemm& g, int tile, int& mt, int& ct) {
  mt = tile % g.mtiles;
  ct = tile / g.mtiles;
  const int sp = (int)((int64_t)mt * 128 / g.mslice), sq = (int)((int64_t)ct * BT / g.nslice);
  return sp + sq < g.slices;
}

template <int BT>
__global__ void __launch_bounds__(K3T_THREADS, 1)
    k3o_gemm(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b0,
             const __grid_constant__ CUtensorMap tmap_b1, const K3OGemm g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)g.stages * (K3T_A_BYTES + BT * 128));
  const K3TRing R = k3t_ring(smem, bars, g.stages, 1, BT / 2);
  uint64_t* accf = R.accum;  // accumulator b holds a finished tile (accf[0] is the ring's own barrier)
  uint64_t* acce = accf + 2; // accumulator b has been stored
  uint64_t* drain = acce + 2;  // every issued MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t T = g.K / 64;
  const int tiles = g.mtiles * g.ctiles;

  if (threadIdx.x == 0) {
    k3t_ring_init(R);  // full, empty and accf[0]
    ptx::mbar_init(&accf[1], 1);
    ptx::mbar_init(&acce[0], 4);  // the four epilogue warps
    ptx::mbar_init(&acce[1], 4);
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_a);
    tc::prefetch_tmap(&tmap_b0);
    tc::prefetch_tmap(&tmap_b1);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, (uint32_t)(2 * BT));
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x) {
        int mt, ct;
        if (!k3o_tile<BT>(g, tile, mt, ct)) continue;
        k3t_produce(R, &tmap_a, &tmap_b0, &tmap_b1, 1, mt * 128, 0, ct * BT, 0, T, it, abort_flag, g.err);
      }
      k3t_drain(R, 0, it, g.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(128, BT);
      uint32_t it = 0;
      int n = 0;  // tiles of this CTA so far
      for (int tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x) {
        int mt, ct;
        if (!k3o_tile<BT>(g, tile, mt, ct)) continue;
        const int ab = n & 1;
        if (n >= 2 && !ptx::mbar_wait(&acce[ab], (uint32_t)(((n >> 1) - 1) & 1), abort_flag)) {
          k3t_abort(abort_flag, g.err);
          break;
        }
        tc::fence_after_sync();
        K3TRing Rb = R;
        Rb.accum = &accf[ab];
        k3t_mma(Rb, tmem + (uint32_t)(ab * BT), 1, 0, idesc, T, it, abort_flag, g.err);
        ++n;
      }
      // the tensor memory is freed below only after every MMA has completed
      tc::commit(drain);
      if (!ptx::mbar_wait(drain, 0, nullptr)) atomicOr(g.err, DEV_ERR_TIMEOUT);
    }
  } else {
    const int q = warp & 3;  // tensor-memory lanes 32q .. 32q + 31
    int n = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      int mt, ct;
      if (!k3o_tile<BT>(g, tile, mt, ct)) continue;
      const int ab = n & 1;
      const bool got = __all_sync(0xffffffffu, ptx::mbar_wait(&accf[ab], (uint32_t)((n >> 1) & 1), abort_flag));
      if (!got) {
        if (lane == 0) k3t_abort(abort_flag, g.err);
        break;
      }
      tc::fence_after_sync();
      if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
        const int64_t m = (int64_t)mt * 128 + 32 * q + lane;
        const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * BT);
        float* dst = g.out + (int64_t)ct * BT * g.M + m;
        for (int c0 = 0; c0 < BT; c0 += 16) {
          uint32_t v[16];
          tc::tmem_ld_32x32b_x16(acc + (uint32_t)c0, v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < 16; ++c) dst[(int64_t)(c0 + c) * g.M] = __uint_as_float(v[c]);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acce[ab]);
      ++n;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)(2 * BT));
  }
}

// Z[b][j] = P_j Q_j (and Z[b][rp + j] = P_j S_j) into BF16 hi/lo rows.
__device__ __forceinline__ void k3t_store_z(const K3TProj& g, int64_t b, int64_t j, float p, float q, float s) {
  const float z1 = p * q;
  const __nv_bfloat16 h1 = __float2bfloat16_rn(z1);
  g.zh[b * g.kz + j] = h1;
  g.zl[b * g.kz + j] = __float2bfloat16_rn(z1 - __bfloat162float(h1));
  if (g.nseg == 3) {
    const float z2 = p * s;
    const __nv_bfloat16 h2 = __float2bfloat16_rn(z2);
    g.zh[b * g.kz + g.rp + j] = h2;
    g.zl[b * g.kz + g.rp + j] = __float2bfloat16_rn(z2 - __bfloat162float(h2));
  }
}

// The FP32 partial block of split z of tile (jt, ct): btile columns x 3
// segments x 128 rank rows, so that inside a block every offset of a
// column group is a constant.
__device__ __forceinline__ float* k3t_part_block(const K3TProj& g, int z, int jt, int ct) {
  return g.part + (((int64_t)z * g.jtiles + jt) * g.ctiles + ct) * ((int64_t)g.btile * 384);
}

// The last split CTA of a tile: Z of rank row jl (index j) for the tile's
// columns from the splits' partials, summed in split order.  Four columns
// at a time, every split's partials are loaded before they are summed, so
// the L2 reads are in flight together.
__device__ __forceinline__ void k3t_reduce_splits(const K3TProj& g, int jt, int ct, int jl, int64_t j) {
#pragma unroll 1
  for (int c0 = 0; c0 < g.btile; c0 += 4) {
    float w[K3T_PROJ_MAX_SPLITS][3][4];
#pragma unroll
    for (int z = 0; z < K3T_PROJ_MAX_SPLITS; ++z)
      if (z < g.splits) {
        const float* blk = k3t_part_block(g, z, jt, ct) + c0 * 384 + jl;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int seg = 0; seg < 3; ++seg) w[z][seg][c] = __ldcg(blk + (c * 3 + seg) * 128);
      }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int z = 0; z < K3T_PROJ_MAX_SPLITS; ++z)
        if (z < g.splits)
#pragma unroll
          for (int seg = 0; seg < 3; ++seg) v[seg] += w[z][seg][c];
      k3t_store_z(g, (int64_t)ct * g.btile + c0 + c, j, v[0], v[1], v[2]);
    }
  }
}

// Projection epilogue of tile (jt = tl.mt, ct, split): Z rows of rank
// indices j0 = 128 jt .. j0 + 127 (lane = row), or with split K this
// split's partials and, for the last split of the tile to arrive, their sum
// in split order.  Rows past rp belong to the next segment or lie past the
// factor copy (zero-filled); they are not stored.
__device__ __forceinline__ void k3t_proj_epilogue(const K3TProj& g, uint32_t tmem, const K3TTile& tl, bool run,
                                                  volatile int* abort_flag, volatile int* last_flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;
  const int jt = tl.mt, ct = tl.ct, split = tl.split;
  const int64_t j = (int64_t)jt * 128 + 32 * q + lane;
  const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16);
  if (run) {
    for (int c0 = 0; c0 < g.btile; c0 += 16) {
      float pv[3][16];
#pragma unroll
      for (int seg = 0; seg < 3; ++seg) {
        if (seg < g.nseg) {
          uint32_t v[16], w[16];
          tc::tmem_ld_32x32b_x16(acc + (uint32_t)(seg * 2 * g.btile + c0), v);
          tc::tmem_ld_32x32b_x16(acc + (uint32_t)(seg * 2 * g.btile + g.btile + c0), w);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < 16; ++c) pv[seg][c] = __uint_as_float(v[c]) + __uint_as_float(w[c]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) pv[seg][c] = 0.f;
        }
      }
      if (j < g.rp) {
        const int64_t b0 = (int64_t)ct * g.btile + c0;
        if (g.splits == 1) {
#pragma unroll
          for (int c = 0; c < 16; ++c) k3t_store_z(g, b0 + c, j, 0.f + pv[0][c], 0.f + pv[1][c], 0.f + pv[2][c]);
        } else {
          // this split's partials (all three segments; zero where the form has two)
          float* blk = k3t_part_block(g, split, jt, ct) + c0 * 384 + 32 * q + lane;
#pragma unroll
          for (int seg = 0; seg < 3; ++seg)
#pragma unroll
            for (int c = 0; c < 16; ++c) blk[(c * 3 + seg) * 128] = pv[seg][c];
        }
      }
    }
  }
  if (g.splits > 1) {
    // the last split of the tile to arrive sums the partials in split order
    const int tile = jt * g.ctiles + ct;
    __threadfence();
    ptx::named_sync(1, 128);
    if (warp == 2 && lane == 0) *last_flag = atomicAdd(&g.cnt[tile], 1u) == (unsigned)(g.splits - 1);
    ptx::named_sync(1, 128);
    if (*last_flag) {
      __threadfence();
      if (j < g.rp && !*abort_flag) k3t_reduce_splits(g, jt, ct, 32 * q + lane, j);
      if (warp == 2 && lane == 0) g.cnt[tile] = 0u;
    }
  }
}

// The projections and the Hadamard products of one tile: rank indices
// j0 = 128 jt .. j0 + 127 and trajectories of column tile ct.  Per K step the
// producer loads the nseg A boxes (rows seg rp + j0 of FT: V^T, W^T, U^T for
// the skew form, B^T, C^T for the general one) and the hi/lo state boxes; the
// MMA warp multiplies each A box with the shared state tile into its own
// accumulator (tensor-memory columns seg 2 btile .. +2 btile: hi | lo).
__global__ void __launch_bounds__(K3T_THREADS, 1)
    k3t_proj(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_bh,
             const __grid_constant__ CUtensorMap tmap_bl, const K3TProj g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + (size_t)g.stages * (g.nseg * K3T_A_BYTES + 2 * g.btile * 128));
  const K3TRing R = k3t_ring(smem, bars, g.stages, g.nseg, g.btile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(R.accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* last_flag = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const K3TTile tl = k3t_tile(blockIdx.x, g.splits, g.ctiles, g.K);

  if (threadIdx.x == 0) {
    k3t_ring_init(R);
    *abort_flag = 0;
    *last_flag = 0;
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
    if (lane == 0) {
      uint32_t it = 0;
      k3t_produce(R, &tmap_a, &tmap_bh, &tmap_bl, g.nseg, tl.mt * 128, (int32_t)g.rp, tl.ct * g.btile, tl.kb0, tl.T,
                  it, abort_flag, g.err);
      k3t_drain(R, 0, it, g.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0;
      k3t_mma(R, tmem, g.nseg, (uint32_t)(2 * g.btile), tc::idesc_bf16_f32(128, 2 * g.btile), tl.T, it, abort_flag,
              g.err);
    }
  } else {
    const bool ok = k3t_wait_accum(R, 0, g.err);
    k3t_proj_epilogue(g, tmem, tl, ok && tl.T > 0 && !__any_sync(0xffffffffu, *abort_flag != 0), abort_flag,
                      last_flag);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)g.tmem_cols);
  }
}

// ------------------------------------------------------------------------
// Persistent batched stepper: every step of a grom_step call on a batch of
// trajectories (a serving pool, with its masks and step budgets) in one
// cooperative launch of one CTA per SM.  Per step:
//   projections (the tiles of k3t_proj)    -> grid barrier
//   expansion   (the tiles of k3t_gemm)    -> grid barrier
//   step        (the elements of k_step_diag_mc)  -> grid barrier
// Each GEMM phase keeps its own ring, whose roles count K steps across tiles,
// phases and steps, and the tensor memory is allocated once.  Rows a later
// phase reads with TMA (Z, the next state's BF16 rows) are written through
// the generic proxy, so the writers fence the async proxy before the barrier.
// The tiles, the split sums and the step's arithmetic are those of the
// per-step kernels, so the states are bitwise the same.  The step phase runs
// the standalone kernel's blocks (same energy/invariant bits) when sums or
// non-identity operators are asked for; in the plain case it spreads the
// elements over all threads and advances each trajectory's step count (and
// serving budget) after the next grid barrier.
struct K3TPersist {
  StepArgs st;
  K3TStepFuse kf;
  K3Args ka;             // the pool's states for the prep at the start of the call
  int batch, nsteps;
  int tiles_p, tiles_g;  // tiles of the two GEMM phases
  int plain;             // 1: flat step phase (no sums, identity mass, no L or f)
  int64_t np, bp;
  unsigned int* bar;     // grid barrier word (zero at create; every barrier adds 2^31 in total)
  uint32_t tmem_cols;
};

__device__ __forceinline__ void k3tp_grid_sync(unsigned int* bar, int* err, volatile int* abort_flag, bool proxy) {
  if (proxy) asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, inc);
    const uint64_t t0 = ptx::globaltimer();
    for (uint32_t spin = 0;; ++spin) {
      const unsigned int now = *reinterpret_cast<volatile unsigned int*>(bar);
      if ((now ^ old) & 0x80000000u) break;
      if ((spin & 255u) == 255u && ptx::globaltimer() - t0 > ptx::WAIT_LIMIT_NS) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (proxy) asm volatile("fence.proxy.async.global;" ::: "memory");
}

__global__ void __launch_bounds__(K3T_THREADS, 1)
    k3tp_kernel(const __grid_constant__ CUtensorMap tmap_ft, const __grid_constant__ CUtensorMap tmap_xh,
                const __grid_constant__ CUtensorMap tmap_xl, const __grid_constant__ CUtensorMap tmap_ae,
                const __grid_constant__ CUtensorMap tmap_zh, const __grid_constant__ CUtensorMap tmap_zl,
                const K3TProj gp, const K3TGemm gg, const K3TPersist pp) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const size_t area_p = (size_t)gp.stages * (gp.nseg * K3T_A_BYTES + 2 * gp.btile * 128);
  const size_t area_g = (size_t)gg.stages * (K3T_A_BYTES + 2 * gg.btile * 128);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (area_p > area_g ? area_p : area_g));
  const K3TRing RP = k3t_ring(smem, bars, gp.stages, gp.nseg, gp.btile);
  const K3TRing RG = k3t_ring(smem, bars + 2 * gp.stages + 1, gg.stages, 1, gg.btile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * gp.stages + 1 + 2 * gg.stages + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* last_flag = abort_flag + 1;
  volatile int* bad_sh = abort_flag + 2;
  volatile int* last_sh = abort_flag + 3;
  double* sh = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(tmem_slot) + 24);  // 64 doubles

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int G = gridDim.x, g = blockIdx.x;
  const StepArgs& st = pp.st;
  int* err = gp.err;

  if (tid == 0) {
    k3t_ring_init(RP);
    k3t_ring_init(RG);
    *abort_flag = 0;
    *last_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_ft);
    tc::prefetch_tmap(&tmap_ae);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, pp.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // the state prep of the call (the rows k3t_prep writes)
  {
    __nv_bfloat16* xh = static_cast<__nv_bfloat16*>(pp.kf.xh);
    __nv_bfloat16* xl = static_cast<__nv_bfloat16*>(pp.kf.xl);
    const K3Args& a = pp.ka;
    for (int64_t t = (int64_t)g * K3T_THREADS + tid; t < pp.bp * pp.np; t += (int64_t)G * K3T_THREADS) {
      const int64_t b = t / pp.np, k = t - b * pp.np;
      float v = 0.f;
      if (b < pp.batch && k < st.n && (a.active == nullptr || a.active[b])) {
        const double* ub = a.hist + b * a.hist_stride + (a.taken[b] % 3) * st.n;
        v = __double2float_rn(ub[k]);
      }
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      xh[t] = hi;
      xl[t] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
  k3tp_grid_sync(pp.bar, err, abort_flag, true);

  uint32_t itp = 0, itg = 0;           // K steps of each ring (producer and MMA keep their own copy)
  uint32_t nt_p = 0, nt_g = 0;         // tiles of each ring in this CTA (accumulator parity)
  const uint32_t idesc = tc::idesc_bf16_f32(128, 2 * gp.btile);
  for (int step = 0; step < pp.nsteps; ++step) {
    if (pp.plain && step > 0 && tid == 0) {
      // the previous step's counts: every element of it is done (grid barrier)
      for (int b = g; b < pp.batch; b += G)
        if (!st.active || st.active[b]) step_done(st, b, st.taken[b]);
    }
    // ---------------------------------------------------------- projections
    for (int tile = g; tile < pp.tiles_p; tile += G, ++nt_p) {
      const K3TTile tl = k3t_tile(tile, gp.splits, gp.ctiles, gp.K);
      if (warp == 0) {
        if (lane == 0)
          k3t_produce(RP, &tmap_ft, &tmap_xh, &tmap_xl, gp.nseg, tl.mt * 128, (int32_t)gp.rp, tl.ct * gp.btile, tl.kb0,
                      tl.T, itp, abort_flag, err);
      } else if (warp == 1) {
        if (lane == 0) k3t_mma(RP, tmem, gp.nseg, (uint32_t)(2 * gp.btile), idesc, tl.T, itp, abort_flag, err);
      } else {
        const bool ok = k3t_wait_accum(RP, nt_p & 1u, err);
        k3t_proj_epilogue(gp, tmem, tl, ok && tl.T > 0 && !__any_sync(0xffffffffu, *abort_flag != 0), abort_flag,
                          last_flag);
      }
      tc::fence_before_sync();
      __syncthreads();  // the accumulator is free for the next tile
      tc::fence_after_sync();
    }
    k3tp_grid_sync(pp.bar, err, abort_flag, true);
    // ------------------------------------------------------------ expansion
    for (int tile = g; tile < pp.tiles_g; tile += G, ++nt_g) {
      const K3TTile tl = k3t_tile(tile, gg.splits, gg.ctiles, gg.K);
      if (warp == 0) {
        if (lane == 0)
          k3t_produce(RG, &tmap_ae, &tmap_zh, &tmap_zl, 1, tl.mt * 128, 0, tl.ct * gg.btile, tl.kb0, tl.T, itg,
                      abort_flag, err);
      } else if (warp == 1) {
        if (lane == 0) k3t_mma(RG, tmem, 1, 0, idesc, tl.T, itg, abort_flag, err);
      } else {
        const bool ok = k3t_wait_accum(RG, nt_g & 1u, err);
        k3t_gemm_epilogue(gg, tmem, tl, ok && tl.T > 0 && !__any_sync(0xffffffffu, *abort_flag != 0));
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
    k3tp_grid_sync(pp.bar, err, abort_flag, false);
    // ----------------------------------------------------------------- step
    if (!pp.plain) {
      // the standalone kernel's blocks, run by the first STEP_MC_THREADS threads
      const int nvb = st.nblk * pp.batch;
      if (tid < STEP_MC_THREADS)
        for (int vb = g; vb < nvb; vb += G)
          step_mc_block<false>(st, step, K1Plan{}, K1Args{}, 2, 0, 1, pp.kf, vb % st.nblk, vb / st.nblk, tid,
                               [] { ptx::named_sync(2, STEP_MC_THREADS); }, sh, bad_sh, last_sh);
    } else {
      // four elements per round: every operand of the four is loaded before
      // any is stepped (the stores of a step could alias the next loads as
      // far as the compiler knows, which would serialise the rounds)
      const int64_t n = st.n;
      __nv_bfloat16* xh = static_cast<__nv_bfloat16*>(pp.kf.xh);
      __nv_bfloat16* xl = static_cast<__nv_bfloat16*>(pp.kf.xl);
      const int64_t total = (int64_t)pp.batch * n, stride = (int64_t)G * K3T_THREADS;
      for (int64_t t0 = (int64_t)g * K3T_THREADS + tid; t0 < total; t0 += 4 * stride) {
        double uq[4][3], nq[4][3], hd[4], nl[4];
        int64_t lq[4], iq[4];
        int bq[4], kq[4];
        bool on[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t t = t0 + e * stride;
          on[e] = t < total;
          const int b = on[e] ? (int)(t / n) : 0;
          bq[e] = b;
          iq[e] = t - (int64_t)b * n;
          on[e] = on[e] && (!st.active || st.active[b]);
          lq[e] = on[e] ? st.taken[b] : 0;
          kq[e] = (int)(lq[e] + 1 < st.order ? lq[e] + 1 : st.order);
          nl[e] = 0.0;
          hd[e] = 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) uq[e][q] = nq[e][q] = 0.0;
          if (on[e]) {
            const double* h = st.hist + bq[e] * st.hist_stride;
            const int m0 = (int)(lq[e] % 3);
            for (int q = 0; q < pp.kf.s2; ++q) nl[e] += (double)pp.kf.d2[((int64_t)q * pp.kf.bp + b) * n + iq[e]];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const int m = m0 - q < 0 ? m0 - q + 3 : m0 - q;
              if (q < kq[e]) {
                uq[e][q] = h[m * n + iq[e]];
                if (q > 0) nq[e][q] = h[(3 + m) * n + iq[e]];
              }
            }
            hd[e] = st.hdiag[kq[e] - 1][iq[e]];
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (!on[e]) continue;
          // the plain diagonal step (step_elem with PLAIN), from the loaded operands
          const int k = kq[e];
          double ext = 0.0, bdf = 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if (q < k) {
              const double gq = q == 0 ? nl[e] : nq[e][q];
              ext = fma(c_alpha[k - 1][q], gq, ext);
              bdf = fma(st.bdt[k - 1][q], uq[e][q], bdf);
            }
          }
          const double un = -(ext + bdf) * hd[e];
          double* h = st.hist + bq[e] * st.hist_stride;
          h[(3 + lq[e] % 3) * n + iq[e]] = nl[e];
          h[((lq[e] + 1) % 3) * n + iq[e]] = un;
          const float v = __double2float_rn(un);
          const __nv_bfloat16 hi = __float2bfloat16_rn(v);
          xh[(int64_t)bq[e] * pp.np + iq[e]] = hi;
          xl[(int64_t)bq[e] * pp.np + iq[e]] = __float2bfloat16_rn(v - __bfloat162float(hi));
          if (((__double_as_longlong(un) >> 52) & 0x7FF) == 0x7FF) report_nonfinite(st, bq[e]);
        }
      }
    }
    k3tp_grid_sync(pp.bar, err, abort_flag, true);
  }
  if (pp.plain && pp.nsteps > 0 && tid == 0)
    for (int b = g; b < pp.batch; b += G)
      if (!st.active || st.active[b]) step_done(st, b, st.taken[b]);
  if (warp == 0 && lane == 0) {
    k3t_drain(RP, 0, itp, err);
    k3t_drain(RG, 0, itg, err);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, pp.tmem_cols);
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

// c[b][i] = sum over splits of d2[split][b][i], in split order, in FP64
// (the plain evaluation; stepping does this sum inside the step kernel).
// Consecutive threads take consecutive i: reads and writes are coalesced.
__global__ void k3t_finish(const float* __restrict__ d2, int s2, int64_t n, int64_t bp, const K3Args a, int batch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * n) return;
  const int64_t b = t / n, i = t - b * n;
  if (a.active && !a.active[b]) return;
  double s = 0.0;
  for (int q = 0; q < s2; ++q) s += (double)d2[((int64_t)q * bp + b) * n + i];
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
  // the projection kernel keeps nseg accumulators of 2 btile columns (hi |
  // lo) in tensor memory: 3 x 128 (skew) or 2 x 256 columns at most
  const int bmax = skew ? 64 : 128;
  int btile = (batch + 15) / 16 * 16;
  if (btile > bmax) btile = bmax;
  p.btile = btile;
  p.ctiles = (batch + btile - 1) / btile;
  p.bp = (int64_t)p.ctiles * btile;
  p.jtiles = (int)((p.rp + 127) / 128);
  const int64_t mt2 = (p.m2 + 127) / 128;
  p.s1_max = std::min(k3t_split_max(p.k1 / 64), K3T_PROJ_MAX_SPLITS);
  p.s1 = std::min(k3t_splits((int64_t)p.jtiles * p.ctiles, p.k1 / 64, sm_count, s1_force), p.s1_max);
  p.s2 = k3t_splits(mt2 * p.ctiles, p.k2 / 64, sm_count, s2_force);
  p.s2_max = k3t_split_max(p.k2 / 64);
  // projections: nseg A boxes and the hi/lo state boxes per stage
  const int stage_p = p.nseg * K3T_A_BYTES + 2 * btile * 128;
  int stp = (int)((K3T_SMEM_MAX - 1024 - 256) / stage_p);
  if (stp > 6) stp = 6;
  p.stages_p = stp;
  p.smem_p = 1024 + (size_t)stp * stage_p + (size_t)(2 * stp + 1) * 8 + 16;
  int cols_p = 32;
  while (cols_p < p.nseg * 2 * btile) cols_p <<= 1;
  p.tmem_p = cols_p;
  // expansion: one A box and the hi/lo Z boxes per stage
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

// Scratch: [arrival counters of the projection tiles, a fixed region per
// (n, r) so that no batch size moves them] xh | xl | projection partials |
// zh | zl | expansion partials.  The counters are zeroed at create and reset
// by the last CTA of each tile.
size_t k3t_counter_bytes(const K3TPlan& p) {
  // 256 bytes for the persistent stepper's grid-barrier word, then the counters
  return 256 + ((size_t)p.jtiles * K3T_MAX_CTILES * sizeof(unsigned int) + 255) / 256 * 256;
}

size_t k3t_scratch_bytes(const K3TPlan& p) {
  const size_t part = p.s1 > 1 ? 4 * (size_t)p.s1 * p.jtiles * p.bp * 384 : 0;
  return k3t_counter_bytes(p) + 2 * (size_t)p.bp * p.np * 2 + part + 2 * (size_t)p.bp * p.k2 * 2 +
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

// D = A B^T of the sliced FP64 CP form; M, mslice multiples of 128, ncols and
// nslice multiples of 64 with ncols a multiple of 128, K a multiple of 64.
template <int BT>
static cudaError_t k3o_gemm_run(const void* A, int64_t M, int64_t mslice, const void* B, int64_t ncols,
                                int64_t nslice, int64_t K, int slices, float* out, int* err, int sm_count,
                                cudaStream_t s) {
  if (M % 128 || mslice % 128 || ncols % BT || nslice % 64 || K % 64 || K <= 0) return cudaErrorInvalidValue;
  CUtensorMap ma, mb0, mb1;
  const __nv_bfloat16* b1 = static_cast<const __nv_bfloat16*>(B) + (BT / 2) * K;  // the tile's second half
  if (!k3t_tmap(&ma, A, K, M, 128) || !k3t_tmap(&mb0, B, K, ncols, BT / 2) ||
      !k3t_tmap(&mb1, b1, K, ncols - BT / 2, BT / 2))
    return cudaErrorInvalidValue;
  K3OGemm g{};
  g.M = M;
  g.K = K;
  g.mslice = mslice;
  g.nslice = nslice;
  g.slices = slices;
  g.mtiles = (int)(M / 128);
  g.ctiles = (int)(ncols / BT);
  const int stage = K3T_A_BYTES + BT * 128;
  int st = (int)((K3T_SMEM_MAX - 1024 - 256) / stage);
  if (st > 6) st = 6;
  g.stages = st;
  g.out = out;
  g.err = err;
  // ring barriers, accf[2], acce[2], drain, the tensor-memory slot and the abort flag
  const size_t smem = 1024 + (size_t)st * stage + (size_t)(2 * st + 5) * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(k3o_gemm<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = g.mtiles * g.ctiles;
  const int grid = tiles < sm_count ? tiles : sm_count;
  k3o_gemm<BT><<<(unsigned)grid, K3T_THREADS, smem, s>>>(ma, mb0, mb1, g);
  return cudaGetLastError();
}

cudaError_t k3o_gemm_launch(const void* A, int64_t M, int64_t mslice, const void* B, int64_t ncols,
                            int64_t nslice, int64_t K, int slices, float* out, int* err, int sm_count,
                            cudaStream_t s) {
  if (ncols % 256 == 0 && ncols >= 512)
    return k3o_gemm_run<256>(A, M, mslice, B, ncols, nslice, K, slices, out, err, sm_count, s);
  return k3o_gemm_run<128>(A, M, mslice, B, ncols, nslice, K, slices, out, err, sm_count, s);
}

// The pieces of the scratch for plan p.
struct K3TBufs {
  unsigned int* bar;
  unsigned int* cnt;
  __nv_bfloat16 *xh, *xl, *zh, *zl;
  float *d1, *d2;
};

static K3TBufs k3t_bufs(const K3TPlan& p, void* scratch) {
  K3TBufs q{};
  uint8_t* base = static_cast<uint8_t*>(scratch);
  q.bar = reinterpret_cast<unsigned int*>(base);
  q.cnt = reinterpret_cast<unsigned int*>(base + 256);
  q.xh = reinterpret_cast<__nv_bfloat16*>(base + k3t_counter_bytes(p));
  q.xl = q.xh + p.bp * p.np;
  q.d1 = reinterpret_cast<float*>(q.xl + p.bp * p.np);
  q.zh = reinterpret_cast<__nv_bfloat16*>(q.d1 + (p.s1 > 1 ? (size_t)p.s1 * p.jtiles * p.bp * 384 : 0));
  q.zl = q.zh + p.bp * p.k2;
  q.d2 = reinterpret_cast<float*>(q.zl + p.bp * p.k2);
  return q;
}

// States into the BF16 hi/lo rows of the projections' B operand.
static cudaError_t k3t_prep_launch(const K3TPlan& p, const K3Args& a, int batch, const K3TBufs& q, cudaStream_t s) {
  k3t_prep<<<dim3((unsigned)((p.np + 255) / 256), (unsigned)p.bp), 256, 0, s>>>(a, p.n, p.np, p.bp, batch, q.xh, q.xl);
  return cudaGetLastError();
}

// Projections with the Hadamard products, then the expansion into the
// trajectory-major partials d2.
static cudaError_t k3t_gemms(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3TBufs& q,
                             int* err, cudaStream_t s) {
  if (p.ctiles > K3T_MAX_CTILES) return cudaErrorInvalidValue;
  CUtensorMap mh, ml;
  if (!k3t_tmap(&mh, q.xh, p.k1, p.bp, p.btile) || !k3t_tmap(&ml, q.xl, p.k1, p.bp, p.btile))
    return cudaErrorInvalidValue;
  K3TProj g{};
  g.rp = p.rp;
  g.bp = p.bp;
  g.kz = p.k2;
  g.K = p.k1;
  g.nseg = p.nseg;
  g.btile = p.btile;
  g.jtiles = p.jtiles;
  g.ctiles = p.ctiles;
  g.splits = p.s1;
  g.stages = p.stages_p;
  g.tmem_cols = p.tmem_p;
  g.part = q.d1;
  g.cnt = q.cnt;
  g.zh = q.zh;
  g.zl = q.zl;
  g.err = err;
  cudaError_t e = cudaFuncSetAttribute(k3t_proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem_p);
  if (e != cudaSuccess) return e;
  k3t_proj<<<(unsigned)(p.jtiles * p.ctiles * p.s1), K3T_THREADS, p.smem_p, s>>>(*m_ft, mh, ml, g);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return k3t_gemm_launch(p, m_ae, q.zh, q.zl, p.m2, p.k2, p.s2, q.d2, err, s);
}

cudaError_t k3t_launch(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a, int batch,
                       void* scratch, int* err, cudaStream_t s) {
  const K3TBufs q = k3t_bufs(p, scratch);
  cudaError_t e = k3t_prep_launch(p, a, batch, q, s);
  if (e == cudaSuccess) e = k3t_gemms(p, m_ft, m_ae, q, err, s);
  if (e != cudaSuccess) return e;
  const int64_t fin = (int64_t)batch * p.n;
  k3t_finish<<<(unsigned)((fin + 255) / 256), 256, 0, s>>>(q.d2, p.s2, p.n, p.bp, a, batch);
  return cudaGetLastError();
}

cudaError_t k3t_launch_step(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a,
                            int batch, void* scratch, int* err, bool prep, const StepArgs& st, int step_index,
                            cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t s) {
  const K3TBufs q = k3t_bufs(p, scratch);
  cudaError_t e = prep ? k3t_prep_launch(p, a, batch, q, s) : cudaSuccess;
  if (e == cudaSuccess && ev0) e = prof_record(ev0, s);
  if (e == cudaSuccess) e = k3t_gemms(p, m_ft, m_ae, q, err, s);
  if (e == cudaSuccess && ev1) e = prof_record(ev1, s);
  if (e != cudaSuccess) return e;
  K3TStepFuse f{};
  f.d2 = q.d2;
  f.s2 = p.s2;
  f.bp = p.bp;
  f.np = p.np;
  f.xh = q.xh;
  f.xl = q.xl;
  return step_diag_mc_k3t_launch(st, step_index, f, s);
}

size_t k3tp_smem(const K3TPlan& p) {
  const size_t area_p = (size_t)p.stages_p * (p.nseg * K3T_A_BYTES + 2 * p.btile * 128);
  const size_t area_g = (size_t)p.stages * (K3T_A_BYTES + 2 * p.btile * 128);
  return 1024 + std::max(area_p, area_g) + (size_t)(2 * p.stages_p + 1 + 2 * p.stages + 1) * 8 + 24 + 64 * 8;
}

cudaError_t k3tp_launch(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a,
                        int batch, void* scratch, int* err, const StepArgs& st, int nsteps, int sm_count,
                        cudaStream_t s) {
  const size_t smem = k3tp_smem(p);
  if (p.ctiles > K3T_MAX_CTILES || smem > (size_t)K3T_SMEM_MAX || nsteps < 1) return cudaErrorInvalidValue;
  const K3TBufs q = k3t_bufs(p, scratch);
  CUtensorMap mft = *m_ft, mae = *m_ae, mxh, mxl, mzh, mzl;
  if (!k3t_tmap(&mxh, q.xh, p.k1, p.bp, p.btile) || !k3t_tmap(&mxl, q.xl, p.k1, p.bp, p.btile) ||
      !k3t_tmap(&mzh, q.zh, p.k2, p.bp, p.btile) || !k3t_tmap(&mzl, q.zl, p.k2, p.bp, p.btile))
    return cudaErrorInvalidValue;
  K3TProj gp{};
  gp.rp = p.rp;
  gp.bp = p.bp;
  gp.kz = p.k2;
  gp.K = p.k1;
  gp.nseg = p.nseg;
  gp.btile = p.btile;
  gp.jtiles = p.jtiles;
  gp.ctiles = p.ctiles;
  gp.splits = p.s1;
  gp.stages = p.stages_p;
  gp.tmem_cols = p.tmem_p;
  gp.part = q.d1;
  gp.cnt = q.cnt;
  gp.zh = q.zh;
  gp.zl = q.zl;
  gp.err = err;
  K3TGemm gg{};
  gg.M = p.m2;
  gg.K = p.k2;
  gg.bp = p.bp;
  gg.btile = p.btile;
  gg.mtiles = (int)((p.m2 + 127) / 128);
  gg.ctiles = p.ctiles;
  gg.splits = p.s2;
  gg.stages = p.stages;
  gg.tmem_cols = p.tmem_cols;
  gg.out = q.d2;
  gg.err = err;
  K3TPersist pp{};
  pp.st = st;
  pp.kf.d2 = q.d2;
  pp.kf.s2 = p.s2;
  pp.kf.bp = p.bp;
  pp.kf.np = p.np;
  pp.kf.xh = q.xh;
  pp.kf.xl = q.xl;
  pp.ka = a;
  pp.batch = batch;
  pp.nsteps = nsteps;
  pp.tiles_p = p.jtiles * p.ctiles * p.s1;
  pp.tiles_g = gg.mtiles * p.ctiles * p.s2;
  pp.plain = !st.mass_diag && !st.lin_diag && !st.forcing && !st.energy && !st.invariant;
  pp.np = p.np;
  pp.bp = p.bp;
  pp.bar = q.bar;
  pp.tmem_cols = (uint32_t)std::max(p.tmem_p, p.tmem_cols);
  cudaError_t e = cudaFuncSetAttribute(k3tp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3tp_kernel, K3T_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  // one CTA per SM at most, and not many more CTAs than the phases have work
  // for, so a small ROM's pool leaves SMs to the other pools' kernels (64 at
  // least: with fewer the barriers and the step phase took longer, measured
  // on a 128-mode pool of 64 trajectories)
  const int64_t step_units = pp.plain ? ((int64_t)batch * p.n + 4 * K3T_THREADS - 1) / (4 * K3T_THREADS)
                                      : (int64_t)st.nblk * batch;
  int64_t grid = std::max<int64_t>({(int64_t)pp.tiles_p, (int64_t)pp.tiles_g, step_units, 64});
  if (grid > sm_count) grid = sm_count;
  void* args[] = {&mft, &mxh, &mxl, &mae, &mzh, &mzl, &gp, &gg, &pp};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k3tp_kernel), dim3((unsigned)grid),
                                     dim3(K3T_THREADS), args, smem, s);
}

}  // namespace grom
