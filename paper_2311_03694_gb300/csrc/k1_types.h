// Launch plan and arguments of the streaming contraction kernels (K1 dense,
// K1P skew-packed).  Kept apart from the library's host-side objects.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace grom {

// ----------------------------------------------------------- K1 streaming
constexpr int K1_CONSUMERS = 256;                 // consumer threads (8 warps)
constexpr int K1_THREADS = K1_CONSUMERS + 32;     // + one producer warp
constexpr int K1_STAGES = 6;
constexpr int K1_STAGE_BYTES = 32768;
constexpr int K1_MAX_ROW_BYTES = K1_STAGE_BYTES;
// Rows of a chunk one consumer thread holds in registers: 8 16-byte vectors
// over its QM positions and the storage's planes (F32X2: hi and lo).  The
// plan caps the rows per chunk at this many per thread row step.
__host__ __device__ constexpr int k1_rmax(int qm, int planes) { return 8 / (qm * planes); }

struct K1Plan {
  int64_t n, np;
  // middle index of the contraction: m rows per test index.  m = n for the
  // G-ROM (the advecting index, weighted by u itself); m = rank for the
  // SVD-ROM (weighted by a separate vector, K1Args::mid); mp = padded m
  int64_t m, mp;
  int has_mid;         // 1: the middle weights come from K1Args::mid
  int64_t row_bytes;   // stored elements per row (np, or lp when packed) * element bytes
  int64_t rpc;         // rows per chunk (all in one test index i)
  int64_t cpi;         // chunks per test index
  int64_t T;           // total chunks = n * cpi
  int grid;            // persistent CTAs
  int maxseg;          // max test-index segments per CTA
  int qm;              // vector positions per consumer thread per row (1,2,4,8)
  int nb_max;          // trajectories per pass
  size_t smem;         // dynamic shared memory
  // skew-packed layout (GROM_LAYOUT_SKEW_PACKED); zero for the dense layout
  int packed;
  int rg;              // row groups per chunk that share a position (1, 2 or 4)
  int64_t h;           // stored distances d = 1..h, h = n / 2
  int64_t lp;          // stored elements per row: round_up(max(h, 1), 64)
  int64_t lw;          // transposed-term window per CTA: maxseg - 1 + lp
};
// Rows between a consumer thread's consecutive rows of a chunk: the row
// groups of the packed layout, else the rows that share the consumer threads
// (the kernels derive the same value; kept out of K1Plan, whose size is part
// of every streaming kernel's parameters).
int64_t k1_row_step(const K1Plan& p, int storage);
// Scratch of the packed kernel: D u_i per (CTA, test-index segment, trajectory,
// position) and the per-CTA transposed-term windows.
size_t k1p_dg_bytes(const K1Plan& p, int storage);
size_t k1p_tg_bytes(const K1Plan& p);

struct K1Args {
  const uint8_t* tensor;  // stored tensor (storage layout)
  const double* u;        // batch x n (FP64), first trajectory of this pass
  int64_t u_stride;       // doubles between trajectories
  double* part;           // scratch: grid x maxseg x NB partials
  double* c;              // batch x n output
  int64_t c_stride;
  int nb;                 // active trajectories in this pass (<= NB)
  int* err;               // device error flags
  // Optional per-trajectory ring addressing for the stepper: when `taken` is
  // non-null, the u of trajectory b is hist + b*hist_stride + (taken[b]%3)*n
  // and c is written to hist + b*hist_stride + (3 + taken[b]%3)*n.
  double* hist;
  const int64_t* taken;
  int64_t hist_stride;
  const int32_t* active;  // nullable: trajectories with active[b]==0 are skipped
  cudaEvent_t ev0, ev1;   // nullable: recorded around the streaming kernel
  int skip_finalize;      // 1: the caller runs a fused finalize (see k_step.cu)
  void* dg;               // packed layout: k1p_dg_bytes of scratch
  double* tg;             // packed layout: k1p_tg_bytes of scratch
  // middle weights when the plan has has_mid (batch x mid_stride FP64): the
  // weight of middle row r for trajectory b is mid[b * mid_stride + r]
  const double* mid;
  int64_t mid_stride;
};

}  // namespace grom
