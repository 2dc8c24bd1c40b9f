// K2P: batched contraction on the tcgen05 tensor cores for the skew-packed
// BF16 layout (the factored form of the batched contraction).
//
// The skew-packed layout keeps one entry of each pair C_ijk = -C_kji: row
// (i, j) holds P[i][j][p] = C[i][j][(i+1+p) mod n] for p < h (Sec. 2.2,
// skew-symmetry of the advection tensor).  For B states the contraction is
// factored through
//   D_i[p, b] = sum_j P[i][j][p] u_bj                       (one GEMM per i)
// after which every stored entry feeds both halves of its pair:
//   c_ib     += D_i[p, b] u_b,k      k = (i+1+p) mod n       (direct entry)
//   c_kb     -= D_i[p, b] u_bi                               (mirrored entry)
// The GEMM is M = packed position p (128 per tile), N = trajectories, K = j.
// The stored rows have p contiguous, so A is read MN-major straight from the
// stored tensor (two 64-position TMA boxes per K step); B is U^T split into
// BF16 hi and lo parts, side by side in shared memory, so one MMA of
// N = 2 btile multiplies both (the states exact to ~2^-17); the epilogue adds
// the hi and lo halves of the accumulator.
// Both halves of a pair use the same FP32 D and the same FP32 state, so
// u^T c(u) vanishes up to FP32 rounding of the sums.  Against the dense K2
// this reads half the tensor bytes and issues half the MMA work, and needs no
// Khatri-Rao generation.
//
// A CTA tile is (m consecutive test indices i, one 128-position block, one
// column tile of trajectories); CTAs are persistent over tiles.  Warp 0
// issues the TMA loads, warp 1 owns the tensor memory and issues
// tcgen05.mma into two FP32 accumulators of 2 btile columns (double buffered
// over i), warps 2-9 read each accumulator back (tcgen05.ld, lane = position
// p; two warps per lane quadrant, splitting the 32-column chunks):
//   * the direct entries are weighted with u_b,k (a coalesced gather) and
//     summed over the 32 lanes of the warp (transpose-reduce with shuffles);
//     the four lane quadrants' sums are added in shared memory, in a fixed
//     order, and written once per (i, b);
//   * the mirrored entries D u_bi are added into a shared-memory window
//     indexed by k - (i0+1+p0): lane p of index i writes row (i-i0) + p, so a
//     tile touches m + 127 rows, conflict-free with an odd row pitch.  The
//     window is written out once per tile.
// A finish kernel adds, for every (k, b), the direct partials and subtracts
// the window rows that cover k, in a fixed order (deterministic), in FP64.
// Where a stored row has two or more position blocks the plans run the
// SM-pair variant (k2p_pair_kernel, below): one 256-row MMA over a cluster of
// two CTAs, each with its own block and half of the states operand; the same
// epilogue, finish and bits.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "grom_internal.h"
#include "tc.cuh"
#include "tc_pair.cuh"

namespace grom {

constexpr int K2P_THREADS = 320;                 // TMA warp, MMA warp, 8 epilogue warps
constexpr int K2P_EPI = 256;                     // epilogue threads
constexpr int K2P_A_BYTES = 128 * 64 * 2;        // 128 positions x 64 advecting indices (two boxes)
constexpr int K2P_SMEM_MAX = 232448;             // opt-in shared memory per CTA

struct K2PDev {
  int64_t n, np, lp, bp;
  int btile, col_tiles, pblks, pbs, m, ranges, tiles, stages, tmem_cols, wrows, wpitch;
  // pbs: position blocks in the tile and scratch numbering (pblks, or pblks
  // rounded up to even for SM pairs; a block past pblks is all padding)
  const float* uf;  // bp x np FP32 states (zero padded)
  float* cdp;       // pbs x n x bp direct partials (per position block)
  float* ep;        // tiles x wrows x btile mirrored-entry windows
  int* err;
};

__device__ __forceinline__ void k2p_tile(const K2PDev& p, int tile, int& ct, int& pb, int64_t& i0, int64_t& i1) {
  ct = tile % p.col_tiles;
  const int rest = tile / p.col_tiles;
  pb = rest % p.pbs;
  const int r = rest / p.pbs;
  i0 = (int64_t)r * p.m;
  i1 = i0 + p.m < p.n ? i0 + p.m : p.n;
}

__device__ __forceinline__ void k2p_abort(volatile int* abort_flag, int* err) {
  *abort_flag = 1;
  atomicOr(err, DEV_ERR_TIMEOUT);
}

// One chunk of NB (32 or 16) trajectory columns of an accumulator, for the
// 32 positions of this warp's lanes: the direct entries D u_k summed over the
// lanes into cdst[0 .. NB) (shared memory), the mirrored entries D u_i added into this lane's
// window row.  acc_hi / acc_lo address the hi and lo products of the chunk,
// ucol the FP32 states of its first column (row stride np).
template <int NB>
__device__ __forceinline__ void k2p_chunk(uint32_t acc_hi, uint32_t acc_lo, const float* __restrict__ ucol,
                                          int64_t np, int64_t k, int64_t i, float* wrow, float* cdst, int lane) {
  uint32_t v[NB], w[NB];
  if constexpr (NB == 32) {
    tc::tmem_ld_32x32b_x32(acc_hi, v);
    tc::tmem_ld_32x32b_x32(acc_lo, w);
  } else {
    tc::tmem_ld_32x32b_x16(acc_hi, v);
    tc::tmem_ld_32x32b_x16(acc_lo, w);
  }
  // lane l holds u_{c0+l, i}; u_{b, k} is gathered per column (consecutive
  // lanes read consecutive k)
  const float ui_l = lane < NB ? __ldg(ucol + lane * np + i) : 0.f;
  float uk[NB];
  const float* pk = ucol + k;
#pragma unroll
  for (int cc = 0; cc < NB; ++cc, pk += np) uk[cc] = __ldg(pk);
  tc::tmem_ld_wait();
  float t[32];
#pragma unroll
  for (int cc = 0; cc < NB; ++cc) {
    const float d = __uint_as_float(v[cc]) + __uint_as_float(w[cc]);
    t[cc] = d * uk[cc];
    wrow[cc] = fmaf(d, __shfl_sync(0xffffffffu, ui_l, cc), wrow[cc]);
  }
#pragma unroll
  for (int cc = NB; cc < 32; ++cc) t[cc] = 0.f;
  // transpose-reduce: afterwards lane l holds the sum over the warp's 32
  // positions of column l
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int cc = 0; cc < s; ++cc) {
      const float send = up ? t[cc] : t[cc + s];
      const float keep = up ? t[cc + s] : t[cc];
      t[cc] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  if (lane < NB) cdst[lane] = t[0];
}

__global__ void __launch_bounds__(K2P_THREADS, 1)
    k2p_tc_kernel(const __grid_constant__ CUtensorMap tmap_c, const __grid_constant__ CUtensorMap tmap_uh,
                  const __grid_constant__ CUtensorMap tmap_ul, const K2PDev p) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned, kept as an offset into the shared array so that the
  // compiler sees shared-memory accesses (not generic ones) in the epilogue
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int S = p.stages;
  const int b_half = p.btile * 128;  // one BF16 tile of U^T (hi or lo)
  const int stage_b = 2 * b_half;
  uint8_t* sa = smem;                                   // S x (128 positions x 64 j)
  uint8_t* sb = sa + (size_t)S * K2P_A_BYTES;           // S x (hi | lo)
  float* win = reinterpret_cast<float*>(sb + (size_t)S * stage_b);
  const size_t wbytes = ((size_t)p.wrows * p.wpitch * 4 + 15) / 16 * 16;
  float* red = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(win) + wbytes);  // 4 quadrants x 128 columns
  uint64_t* full = reinterpret_cast<uint64_t*>(red + 4 * 128);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;  // accumulator b holds a finished D_i
  uint64_t* acce = accf + 2;   // accumulator b has been read back
  uint64_t* drain = acce + 2;  // every issued MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* ep_abort = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jblocks = (int)((p.n + 63) / 64);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], K2P_EPI / 32);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    *ep_abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_c);
    tc::prefetch_tmap(&tmap_uh);
    tc::prefetch_tmap(&tmap_ul);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, (uint32_t)p.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int64_t q = 0;  // K steps issued
      bool run = true;
      for (int tile = blockIdx.x; run && tile < p.tiles; tile += gridDim.x) {
        int ct, pb;
        int64_t i0, i1;
        k2p_tile(p, tile, ct, pb, i0, i1);
        for (int64_t i = i0; run && i < i1; ++i) {
          for (int jb = 0; jb < jblocks; ++jb, ++q) {
            const int s = (int)(q % S);
            if (q >= S && !ptx::mbar_wait(&empty[s], (uint32_t)(((q / S) & 1) ^ 1), abort_flag)) {
              k2p_abort(abort_flag, p.err);
              run = false;
              break;
            }
            ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)(K2P_A_BYTES + stage_b));
            uint8_t* a = sa + (size_t)s * K2P_A_BYTES;
            tc::tma_load_3d(a, &tmap_c, pb * 128, jb * 64, (int32_t)i, &full[s]);
            tc::tma_load_3d(a + K2P_A_BYTES / 2, &tmap_c, pb * 128 + 64, jb * 64, (int32_t)i, &full[s]);
            uint8_t* b = sb + (size_t)s * stage_b;
            tc::tma_load_2d(b, &tmap_uh, jb * 64, ct * p.btile, &full[s]);
            tc::tma_load_2d(b + b_half, &tmap_ul, jb * 64, ct * p.btile, &full[s]);
          }
        }
      }
      // the copies still in flight land before the CTA exits
      for (int64_t x = q > S ? q - S : 0; x < q; ++x)
        if (!ptx::mbar_wait(&full[x % S], (uint32_t)((x / S) & 1), nullptr)) atomicOr(p.err, DEV_ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32_amn(128, 2 * p.btile);  // hi | lo
      int64_t q = 0, icnt = 0;
      bool run = true;
      for (int tile = blockIdx.x; run && tile < p.tiles; tile += gridDim.x) {
        int ct, pb;
        int64_t i0, i1;
        k2p_tile(p, tile, ct, pb, i0, i1);
        for (int64_t i = i0; run && i < i1; ++i, ++icnt) {
          const int bi = (int)(icnt & 1);
          if (icnt >= 2 && !ptx::mbar_wait(&acce[bi], (uint32_t)(((icnt >> 1) - 1) & 1), abort_flag)) {
            k2p_abort(abort_flag, p.err);
            run = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)(bi * 2 * p.btile);
          for (int jb = 0; jb < jblocks; ++jb, ++q) {
            const int s = (int)(q % S);
            if (!ptx::mbar_wait(&full[s], (uint32_t)((q / S) & 1), abort_flag)) {
              k2p_abort(abort_flag, p.err);
              run = false;
              break;
            }
            tc::fence_after_sync();
            // A: two 64-position boxes 8 KB apart along M, 8-row K atoms 1 KB apart
            const uint64_t a0 = tc::sw128_mnmajor_desc(sa + (size_t)s * K2P_A_BYTES, K2P_A_BYTES / 2, 1024);
            const uint64_t bhl = tc::sw128_kmajor_desc(sb + (size_t)s * stage_b);  // 2 btile rows
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // K = 16: two 8-row atoms of A, 32 bytes of B
              const uint32_t accum = (jb > 0 || k > 0) ? 1u : 0u;
              tc::mma_bf16(acc, a0 + (uint64_t)(128 * k), bhl + 2 * k, idesc, accum);
            }
            tc::commit(&empty[s]);
          }
          if (run) tc::commit(&accf[bi]);
        }
      }
      tc::commit(drain);
      if (!ptx::mbar_wait(drain, 0, nullptr)) atomicOr(p.err, DEV_ERR_TIMEOUT);
    }
  } else {
    // ----------------------------------------------- epilogue (warps 2-9)
    const int q = warp & 3;             // tensor-memory lanes 32q .. 32q+31 belong to this warp
    const int half = (warp - 2) >> 2;   // the pair of a quadrant takes alternate 32-column chunks
    const int et = threadIdx.x - 64;
    for (int x = et; x < p.wrows * p.wpitch; x += K2P_EPI) win[x] = 0.f;
    ptx::named_sync(1, K2P_EPI);
    int64_t icnt = 0;
    bool run = true;
    for (int tile = blockIdx.x; run && tile < p.tiles; tile += gridDim.x) {
      int ct, pb;
      int64_t i0, i1;
      k2p_tile(p, tile, ct, pb, i0, i1);
      const int64_t pp = (int64_t)pb * 128 + 32 * q + lane;  // this lane's packed position
      const float* ut = p.uf + (int64_t)ct * p.btile * p.np;
      float* cd = p.cdp + (int64_t)pb * p.n * p.bp + (int64_t)ct * p.btile;
      for (int64_t i = i0; i < i1; ++i, ++icnt) {
        const int bi = (int)(icnt & 1);
        // warp-uniform: the tensor-memory loads below are collective
        const bool got = __all_sync(0xffffffffu, ptx::mbar_wait(&accf[bi], (uint32_t)((icnt >> 1) & 1), abort_flag));
        if (!got && lane == 0) {
          *ep_abort = 1;
          k2p_abort(abort_flag, p.err);
        }
        ptx::named_sync(1, K2P_EPI);
        if (*ep_abort) {  // read by all epilogue warps between the same two barriers
          run = false;
          break;
        }
        tc::fence_after_sync();
        const int64_t k = (i + 1 + pp) % p.n;
        float* wrow = win + ((int)(i - i0) + 32 * q + lane) * p.wpitch;
        const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(bi * 2 * p.btile);
        for (int c0 = 32 * half; c0 < p.btile; c0 += 64) {
          const uint32_t ahi = acc + (uint32_t)c0, alo = acc + (uint32_t)(p.btile + c0);
          const float* ucol = ut + (int64_t)c0 * p.np;
          if (p.btile - c0 >= 32)
            k2p_chunk<32>(ahi, alo, ucol, p.np, k, i, wrow + c0, red + q * 128 + c0, lane);
          else  // a last half chunk (btile an odd multiple of 16)
            k2p_chunk<16>(ahi, alo, ucol, p.np, k, i, wrow + c0, red + q * 128 + c0, lane);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[bi]);
        ptx::named_sync(1, K2P_EPI);  // consecutive i of different quadrants share window rows
        // the four quadrants' direct sums (read before the next i's first barrier)
        if (et < p.btile) cd[i * p.bp + et] = ((red[et] + red[128 + et]) + red[256 + et]) + red[384 + et];
      }
      if (!run) break;
      float* dst = p.ep + (int64_t)tile * p.wrows * p.btile;
      for (int x = et; x < p.wrows * p.btile; x += K2P_EPI) {
        const int w = x / p.btile, b = x - w * p.btile;
        dst[x] = win[w * p.wpitch + b];
        win[w * p.wpitch + b] = 0.f;
      }
      ptx::named_sync(1, K2P_EPI);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
  }
}

// ------------------------------------------------------------- SM pairs
// The same contraction with one pair MMA (cta_group::2, M = 256) per K step
// over a cluster of two CTAs.  Each CTA holds the A tile of its own
// 128-position block (blocks 2q and 2q + 1 of a pair tile) and one half of
// the states operand (the leader the hi part, the peer the lo part), so a CTA
// brings in 16 KB + 128 btile bytes per K step for the same MMA work per SM
// as the single-CTA kernel's 16 KB + 256 btile bytes, and one more pipeline
// stage fits beside the window.  The leader's MMA thread writes both SMs'
// tensor memory.  Barriers: full (in the leader; both CTAs' TMA loads
// complete on it), empty and accumulator-full (in both, multicast commits),
// accumulator-empty (in the leader; the 16 epilogue warps of the pair arrive
// on it).  Each CTA's epilogue is the single-CTA one for its own block.
__device__ __forceinline__ void k2p_pair_tile(const K2PDev& p, int t2, uint32_t rank, int& ct, int& pb, int64_t& i0,
                                              int64_t& i1, int& tile) {
  k2p_pair_coords(t2, (int)rank, p.col_tiles, p.pbs, p.m, p.n, ct, pb, i0, i1, tile);
}

// Stops both CTAs of the pair: their waits return at the next check.
__device__ __forceinline__ void k2p_pair_abort(volatile int* abort_flag, uint32_t peer_abort, int* err) {
  *abort_flag = 1;
  tcp::st_cluster_u32(peer_abort, 1u);
  atomicOr(err, DEV_ERR_TIMEOUT);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(K2P_THREADS, 1)
    k2p_pair_kernel(const __grid_constant__ CUtensorMap tmap_c, const __grid_constant__ CUtensorMap tmap_uh,
                    const __grid_constant__ CUtensorMap tmap_ul, const K2PDev p) {
  extern __shared__ uint8_t smem_raw[];
  // the same 1024-byte aligned offset in both CTAs (the pair MMA reads the
  // peer's operands at the leader's offsets)
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int S = p.stages;
  const int stage_b = p.btile * 128;  // this CTA's half of U^T (hi or lo)
  uint8_t* sa = smem;                                   // S x (128 positions x 64 j)
  uint8_t* sb = sa + (size_t)S * K2P_A_BYTES;           // S x (hi or lo)
  float* win = reinterpret_cast<float*>(sb + (size_t)S * stage_b);
  const size_t wbytes = ((size_t)p.wrows * p.wpitch * 4 + 15) / 16 * 16;
  float* red = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(win) + wbytes);  // 4 quadrants x 128 columns
  uint64_t* full = reinterpret_cast<uint64_t*>(red + 4 * 128);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;  // accumulator b holds a finished D_i
  uint64_t* acce = accf + 2;   // accumulator b has been read back (leader)
  uint64_t* drain = acce + 2;  // every issued MMA has completed (leader)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* ep_abort = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = tcp::cta_rank();
  const bool leader = rank == 0;
  const int cluster = (int)(blockIdx.x >> 1), nclusters = (int)(gridDim.x >> 1);
  const int pair_tiles = p.tiles >> 1;
  const int jblocks = (int)((p.n + 63) / 64);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], 2 * K2P_EPI / 32);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    *ep_abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmap_c);
    tc::prefetch_tmap(leader ? &tmap_uh : &tmap_ul);
  }
  if (warp == 1) {
    tcp::tmem_alloc2(tmem_slot, (uint32_t)p.tmem_cols);
    tcp::tmem_relinquish2();
  }
  tc::fence_before_sync();
  __syncthreads();
  tcp::cluster_sync();  // both CTAs' barriers exist before any arrival from the other
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t peer_abort = tcp::map_shared((const void*)abort_flag, rank ^ 1u);

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      const CUtensorMap* tmap_u = leader ? &tmap_uh : &tmap_ul;
      int64_t q = 0;  // K steps issued
      bool run = true;
      for (int t2 = cluster; run && t2 < pair_tiles; t2 += nclusters) {
        int ct, pb, tile;
        int64_t i0, i1;
        k2p_pair_tile(p, t2, rank, ct, pb, i0, i1, tile);
        for (int64_t i = i0; run && i < i1; ++i) {
          for (int jb = 0; jb < jblocks; ++jb, ++q) {
            const int s = (int)(q % S);
            if (q >= S && !ptx::mbar_wait(&empty[s], (uint32_t)(((q / S) & 1) ^ 1), abort_flag)) {
              k2p_pair_abort(abort_flag, peer_abort, p.err);
              run = false;
              break;
            }
            const uint32_t fb = tcp::map_shared(&full[s], 0);
            if (leader) ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)(2 * (K2P_A_BYTES + stage_b)));
            uint8_t* a = sa + (size_t)s * K2P_A_BYTES;
            tcp::tma_load_3d_pair(a, &tmap_c, pb * 128, jb * 64, (int32_t)i, fb);
            tcp::tma_load_3d_pair(a + K2P_A_BYTES / 2, &tmap_c, pb * 128 + 64, jb * 64, (int32_t)i, fb);
            tcp::tma_load_2d_pair(sb + (size_t)s * stage_b, tmap_u, jb * 64, ct * p.btile, fb);
          }
        }
      }
      // the leader's full barriers count both CTAs' copies: the copies still
      // in flight land before the leader reaches the closing cluster barrier
      if (leader)
        for (int64_t x = q > S ? q - S : 0; x < q; ++x)
          if (!ptx::mbar_wait(&full[x % S], (uint32_t)((x / S) & 1), nullptr)) atomicOr(p.err, DEV_ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------- MMA issuer (leader)
    if (lane == 0 && leader) {
      const uint32_t idesc = tc::idesc_bf16_f32_amn(256, 2 * p.btile);  // hi (leader) | lo (peer)
      int64_t q = 0, icnt = 0;
      bool run = true;
      for (int t2 = cluster; run && t2 < pair_tiles; t2 += nclusters) {
        int ct, pb, tile;
        int64_t i0, i1;
        k2p_pair_tile(p, t2, rank, ct, pb, i0, i1, tile);
        for (int64_t i = i0; run && i < i1; ++i, ++icnt) {
          const int bi = (int)(icnt & 1);
          if (icnt >= 2 && !ptx::mbar_wait(&acce[bi], (uint32_t)(((icnt >> 1) - 1) & 1), abort_flag)) {
            k2p_pair_abort(abort_flag, peer_abort, p.err);
            run = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)(bi * 2 * p.btile);
          for (int jb = 0; jb < jblocks; ++jb, ++q) {
            const int s = (int)(q % S);
            if (!ptx::mbar_wait(&full[s], (uint32_t)((q / S) & 1), abort_flag)) {
              k2p_pair_abort(abort_flag, peer_abort, p.err);
              run = false;
              break;
            }
            tc::fence_after_sync();
            const uint64_t a0 = tc::sw128_mnmajor_desc(sa + (size_t)s * K2P_A_BYTES, K2P_A_BYTES / 2, 1024);
            const uint64_t b0 = tc::sw128_kmajor_desc(sb + (size_t)s * stage_b);  // btile rows per CTA
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t accum = (jb > 0 || k > 0) ? 1u : 0u;
              tcp::mma2_bf16(acc, a0 + (uint64_t)(128 * k), b0 + 2 * k, idesc, accum);
            }
            tcp::commit2_mc(&empty[s], 3);
          }
          if (run) tcp::commit2_mc(&accf[bi], 3);
        }
      }
      tcp::commit2_mc(drain, 3);
      if (!ptx::mbar_wait(drain, 0, nullptr)) atomicOr(p.err, DEV_ERR_TIMEOUT);
    }
  } else {
    // ----------------------------------------------- epilogue (warps 2-9)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;
    const uint32_t acce_l0 = tcp::map_shared(&acce[0], 0), acce_l1 = tcp::map_shared(&acce[1], 0);
    for (int x = et; x < p.wrows * p.wpitch; x += K2P_EPI) win[x] = 0.f;
    ptx::named_sync(1, K2P_EPI);
    int64_t icnt = 0;
    bool run = true;
    for (int t2 = cluster; run && t2 < pair_tiles; t2 += nclusters) {
      int ct, pb, tile;
      int64_t i0, i1;
      k2p_pair_tile(p, t2, rank, ct, pb, i0, i1, tile);
      const int64_t pp = (int64_t)pb * 128 + 32 * q + lane;
      const float* ut = p.uf + (int64_t)ct * p.btile * p.np;
      float* cd = p.cdp + (int64_t)pb * p.n * p.bp + (int64_t)ct * p.btile;
      for (int64_t i = i0; i < i1; ++i, ++icnt) {
        const int bi = (int)(icnt & 1);
        const bool got = __all_sync(0xffffffffu, ptx::mbar_wait(&accf[bi], (uint32_t)((icnt >> 1) & 1), abort_flag));
        if (!got && lane == 0) {
          *ep_abort = 1;
          k2p_pair_abort(abort_flag, peer_abort, p.err);
        }
        ptx::named_sync(1, K2P_EPI);
        if (*ep_abort) {
          run = false;
          break;
        }
        tc::fence_after_sync();
        const int64_t k = (i + 1 + pp) % p.n;
        float* wrow = win + ((int)(i - i0) + 32 * q + lane) * p.wpitch;
        const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(bi * 2 * p.btile);
        for (int c0 = 32 * half; c0 < p.btile; c0 += 64) {
          const uint32_t ahi = acc + (uint32_t)c0, alo = acc + (uint32_t)(p.btile + c0);
          const float* ucol = ut + (int64_t)c0 * p.np;
          if (p.btile - c0 >= 32)
            k2p_chunk<32>(ahi, alo, ucol, p.np, k, i, wrow + c0, red + q * 128 + c0, lane);
          else
            k2p_chunk<16>(ahi, alo, ucol, p.np, k, i, wrow + c0, red + q * 128 + c0, lane);
        }
        tc::fence_before_sync();
        __syncwarp();
        // the loads above are complete (tcgen05.wait::ld): the signal orders no memory access
        if (lane == 0) tcp::mbar_arrive_remote(bi ? acce_l1 : acce_l0);
        ptx::named_sync(1, K2P_EPI);
        if (et < p.btile) cd[i * p.bp + et] = ((red[et] + red[128 + et]) + red[256 + et]) + red[384 + et];
      }
      if (!run) break;
      float* dst = p.ep + (int64_t)tile * p.wrows * p.btile;
      for (int x = et; x < p.wrows * p.btile; x += K2P_EPI) {
        const int w = x / p.btile, b = x - w * p.btile;
        dst[x] = win[w * p.wpitch + b];
        win[w * p.wpitch + b] = 0.f;
      }
      ptx::named_sync(1, K2P_EPI);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tcp::cluster_sync();  // no thread of either CTA touches the other's memory or the tensor memory after this
  if (warp == 1) {
    tc::fence_after_sync();
    tcp::tmem_dealloc2(tmem, (uint32_t)p.tmem_cols);
  }
}

// uf[b][k] = u_b[k] (FP32) and its BF16 hi/lo parts, zero for padding and
// inactive trajectories.
__global__ void k2p_prep_kernel(const K2PDev p, float* uf, __nv_bfloat16* uh, __nv_bfloat16* ul, const double* u,
                                int64_t u_stride, const double* hist, const int64_t* taken, int64_t hist_stride,
                                const int32_t* active, int batch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.bp * p.np) return;
  const int64_t b = t / p.np, k = t - b * p.np;
  float v = 0.f;
  if (b < batch && k < p.n && (active == nullptr || active[b])) {
    const double* ub = taken ? hist + b * hist_stride + (taken[b] % 3) * p.n : u + b * u_stride;
    v = __double2float_rn(ub[k]);
  }
  uf[t] = v;
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  uh[t] = hi;
  ul[t] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// c[b][k] = direct partials of row k - mirrored-entry windows covering k,
// each group summed in a fixed order in FP32 (the partials are FP32 sums
// already; FP64 adds run at about two per clock per SM on this part), the
// two totals subtracted in FP64.
__global__ void k2p_finish_kernel(const K2PDev p, double* c, int64_t c_stride, double* hist, const int64_t* taken,
                                  int64_t hist_stride, const int32_t* active, int batch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * p.n) return;
  const int64_t k = t / batch, b = t - k * batch;  // consecutive threads: consecutive b
  if (active && !active[b]) return;
  const int ct = (int)(b / p.btile), bl = (int)(b - (int64_t)ct * p.btile);
  float sd = 0.f, sm = 0.f;
  for (int pb = 0; pb < p.pblks; ++pb) sd += p.cdp[((int64_t)pb * p.n + k) * p.bp + b];
  // window row w of tile (range r, block pb) holds the mirrored entries of
  // k = (r m + 1 + 128 pb + w) mod n
  for (int pb = 0; pb < p.pblks; ++pb) {
    const int64_t x = ((k - 1 - (int64_t)pb * 128) % p.n + p.n) % p.n;
    auto add = [&](int r) {
      int64_t w = x - (int64_t)r * p.m;
      if (w < 0) w += p.n;
      const float* e = p.ep + ((int64_t)(r * p.pbs + pb) * p.col_tiles + ct) * p.wrows * p.btile + bl;
      for (; w < p.wrows; w += p.n) sm += e[w * p.btile];
    };
    if (p.n <= p.wrows) {
      for (int r = 0; r < p.ranges; ++r) add(r);
    } else {
      // w = x - r m for r m <= x, w = x - r m + n for r m > x; at most one row per tile
      const int rhi = (int)(x / p.m);
      const int rlo = x - p.wrows < 0 ? 0 : (int)((x - p.wrows) / p.m) + 1;
#pragma unroll 4
      for (int r = rlo; r <= rhi; ++r) add(r);
      const int64_t y = x + p.n - p.wrows;
      int r2 = y < 0 ? 0 : (int)(y / p.m) + 1;
      if (r2 < rhi + 1) r2 = rhi + 1;
      for (int r = r2; r < p.ranges; ++r) add(r);
    }
  }
  double* dst = taken ? hist + b * hist_stride + (3 + taken[b] % 3) * p.n : c + b * c_stride;
  dst[k] = (double)sd - (double)sm;
}

// ------------------------------------------------------------------- host
// The stored rows as a 3-D tensor (p, j, i); boxes of 64 positions x 64 j.
bool k2p_make_tmap(CUtensorMap* m, const void* packed, int64_t n, int64_t lp) {
  auto fn = tmap_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)lp, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)(lp * 2), (cuuint64_t)(n * lp * 2)};
  cuuint32_t box[3] = {64, 64, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(packed), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool k2p_make_tmap_u(CUtensorMap* m, const void* u, int64_t np, int64_t bp, int btile) {
  auto fn = tmap_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)bp};
  cuuint64_t strides[1] = {(cuuint64_t)(np * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)btile};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(u), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static size_t k2p_window_bytes(int wrows, int wpitch) { return ((size_t)wrows * wpitch * 4 + 15) / 16 * 16; }

// Pipeline stages that fit beside the mirrored-entry window of an m-row tile.
static int k2p_stages_for(int m, int wpitch, int stage) {
  const size_t fixed = 1024 + k2p_window_bytes(m + 127, wpitch) + 4 * 128 * 4 + (size_t)(2 * 8 + 5) * 8 + 16;
  const int st = (int)(((size_t)K2P_SMEM_MAX - fixed) / (size_t)stage);
  return st > 8 ? 8 : st;
}

static int k2p_btile(int batch) {
  const int btile = (batch + 15) / 16 * 16;
  return btile > 128 ? 128 : btile;
}

// SM pairs need at least two position blocks (a stored row longer than
// 128 positions).
bool k2p_pair_ok(int64_t lp) { return (lp + 127) / 128 >= 2; }

// The tile heights the plan considers: m in [8, 32] that keep the deepest
// pipeline the shared memory allows at m = 8 (the window grows with m).  The
// SM-pair kernel's stages are smaller, so every height admitted here keeps at
// least as many stages there.
bool k2p_tile_m_ok(int batch, int m) {
  if (m < 8 || m > 32) return false;
  const int btile = k2p_btile(batch);
  const int stage = K2P_A_BYTES + 2 * btile * 128;
  const int s8 = k2p_stages_for(8, btile + 1, stage);
  return k2p_stages_for(m, btile + 1, stage) >= (s8 < 3 ? s8 : 3);
}

K2PPlan k2p_plan(int64_t n, int64_t lp, int batch, int sm_count, int m_force, int ctas_force) {
  K2PPlan p{};
  p.n = n;
  p.np = padded_n(n);
  p.lp = lp;
  const int btile = k2p_btile(batch);
  p.btile = btile;
  p.col_tiles = (batch + btile - 1) / btile;
  p.bp = (int64_t)p.col_tiles * btile;
  p.pblks = (int)((lp + 127) / 128);
  // SM pairs wherever a row has two blocks: measured 4-7 % faster than
  // single CTAs from 16 to 1024 trajectories at N = 512 and 1024
  const bool pair_ok = k2p_pair_ok(lp) && sm_count >= 2;
  int ctas = pair_ok ? 2 : 1;
  if (ctas_force == 1 || (ctas_force == 2 && pair_ok)) ctas = ctas_force;
  p.ctas = ctas;
  p.pbs = ctas == 2 ? (p.pblks + 1) / 2 * 2 : p.pblks;
  p.wpitch = btile + 1;  // odd pitch: the 32 lanes of a warp hit 32 banks
  const int stage = K2P_A_BYTES + (ctas == 2 ? 1 : 2) * btile * 128;
  // test indices per tile: among the heights k2p_tile_m_ok admits, the
  // largest whose tile count fills whole waves of SMs (pairs of SMs) best
  const int units = ctas == 2 ? sm_count / 2 : sm_count;
  double best = -1.0;
  int bm = 8;
  for (int m = 32; m >= 8; --m) {
    if (!k2p_tile_m_ok(batch, m)) continue;
    const int64_t tiles = (n + m - 1) / m * (p.pbs / ctas) * p.col_tiles;
    const int64_t waves = (tiles + units - 1) / units;
    const double eff = (double)tiles / (double)(waves * units);
    if (eff > best + 1e-9) {
      best = eff;
      bm = m;
    }
  }
  if (m_force > 0 && k2p_tile_m_ok(batch, m_force)) bm = m_force;
  p.m = bm;
  p.ranges = (int)((n + bm - 1) / bm);
  p.tiles = p.ranges * p.pbs * p.col_tiles;
  p.wrows = bm + 127;
  int st = k2p_stages_for(bm, p.wpitch, stage);
  if (st < 2) st = 2;
  p.stages = st;
  p.smem = 1024 + (size_t)st * stage + k2p_window_bytes(p.wrows, p.wpitch) + 4 * 128 * 4 + (size_t)(2 * st + 5) * 8 + 16;
  int cols = 64;  // two accumulators of 2 btile columns (hi | lo); chunks of 32 stay inside
  while (cols < 4 * btile) cols <<= 1;
  p.tmem_cols = cols;
  if (ctas == 2) {
    const int pairs = p.tiles / 2;
    p.grid = 2 * (pairs < units ? pairs : units);
  } else {
    p.grid = p.tiles < sm_count ? p.tiles : sm_count;
  }
  return p;
}

// uf | uh | ul | direct partials | windows
size_t k2p_scratch_bytes(const K2PPlan& p) {
  const size_t st = (size_t)p.bp * p.np;
  return st * (4 + 2 + 2) + 4 * ((size_t)p.pbs * p.n * p.bp + (size_t)p.tiles * p.wrows * p.btile);
}

// Over both kernels (the tuning may pick either).
size_t k2p_scratch_need(int64_t n, int64_t lp, int max_batch, int sm_count) {
  size_t need = 0;
  for (int b = 16; b - 16 < max_batch; b += 16)
    for (int ctas = 1; ctas <= 2; ++ctas)
      need = std::max(need, k2p_scratch_bytes(k2p_plan(n, lp, b < max_batch ? b : max_batch, sm_count, 0, ctas)));
  return need;
}

// Clusters of two that fit on the current device at once with this shared
// memory; 0 if none.  Every plan's shared memory allows one CTA per SM, so
// the count is the same for all of them and is kept per device (atomically:
// ROMs on different threads may launch concurrently).
static int k2p_pair_clusters(size_t smem) {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  const int c = cached[dev].load(std::memory_order_relaxed);
  if (c > 0) return c;
  if (cudaFuncSetAttribute(k2p_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(K2P_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, (void*)k2p_pair_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (nc > 0) cached[dev].store(nc, std::memory_order_relaxed);
  return nc;
}

bool k2p_pairs_supported() { return k2p_pair_clusters(K2P_SMEM_MAX) > 0; }

cudaError_t k2p_launch(const K2PPlan& p, const CUtensorMap* tmap, const K2Args& a, cudaStream_t s) {
  K2PDev d{};
  d.n = p.n;
  d.np = p.np;
  d.lp = p.lp;
  d.bp = p.bp;
  d.btile = p.btile;
  d.col_tiles = p.col_tiles;
  d.pblks = p.pblks;
  d.pbs = p.pbs;
  d.m = p.m;
  d.ranges = p.ranges;
  d.tiles = p.tiles;
  d.stages = p.stages;
  d.tmem_cols = p.tmem_cols;
  d.wrows = p.wrows;
  d.wpitch = p.wpitch;
  d.err = a.err;
  const size_t st = (size_t)p.bp * p.np;
  float* uf = reinterpret_cast<float*>(a.scratch);
  __nv_bfloat16* uh = reinterpret_cast<__nv_bfloat16*>(uf + st);
  __nv_bfloat16* ul = uh + st;
  d.uf = uf;
  d.cdp = reinterpret_cast<float*>(ul + st);
  d.ep = d.cdp + (size_t)p.pbs * p.n * p.bp;
  CUtensorMap mh, ml;
  if (!k2p_make_tmap_u(&mh, uh, p.np, p.bp, p.btile) || !k2p_make_tmap_u(&ml, ul, p.np, p.bp, p.btile))
    return cudaErrorInvalidValue;
  const int64_t prep = p.bp * p.np;
  k2p_prep_kernel<<<(unsigned)((prep + 255) / 256), 256, 0, s>>>(d, uf, uh, ul, a.u, a.u_stride, a.hist, a.taken,
                                                                 a.hist_stride, a.active, a.batch);
  cudaError_t e;
  if (p.ctas == 2) {
    e = cudaFuncSetAttribute(k2p_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    // persistent pairs: no more clusters than fit at once
    const int fit = k2p_pair_clusters(p.smem);
    if (fit < 1) return cudaErrorInvalidConfiguration;
    const int grid = p.grid / 2 < fit ? p.grid : 2 * fit;
    if (a.ev0) prof_record(a.ev0, s);
    k2p_pair_kernel<<<(unsigned)grid, K2P_THREADS, p.smem, s>>>(*tmap, mh, ml, d);
  } else {
    e = cudaFuncSetAttribute(k2p_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    if (a.ev0) prof_record(a.ev0, s);
    k2p_tc_kernel<<<(unsigned)p.grid, K2P_THREADS, p.smem, s>>>(*tmap, mh, ml, d);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.ev1) prof_record(a.ev1, s);
  const int64_t red = (int64_t)a.batch * p.n;
  k2p_finish_kernel<<<(unsigned)((red + 255) / 256), 256, 0, s>>>(d, a.c, a.c_stride, a.hist, a.taken,
                                                                  a.hist_stride, a.active, a.batch);
  return cudaGetLastError();
}

}  // namespace grom
