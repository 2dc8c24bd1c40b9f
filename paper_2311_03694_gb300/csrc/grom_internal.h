// Internal definitions of the GB300 Galerkin ROM library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/grom.h"

namespace grom {

// ----------------------------------------------------------------- errors
void set_error(const std::string& msg);
grom_status fail(grom_status code, const std::string& msg);
grom_status cuda_fail(cudaError_t e, const char* what);

#define GROM_CUDA_TRY(expr)                                       \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::grom::cuda_fail(_e, #expr);   \
  } while (0)

// Records a kernel-timing event.  Under stream capture the record becomes an
// event node of the graph (cudaEventRecordExternal), so graph replays time
// their kernels too.
inline cudaError_t prof_record(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaGetLastError();
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// Device-side error flags (bit mask in a device int).
constexpr int DEV_ERR_TIMEOUT = 1;
constexpr int DEV_ERR_NONFINITE = 2;

// ------------------------------------------------------------- layout
// The stored tensor pads the advected index k to np = round_up(n, 64) with
// zeros, so every stored row starts on a 128-byte boundary for every
// storage type and the streaming kernels never see a ragged row.
inline int64_t padded_n(int64_t n) { return (n + 63) / 64 * 64; }

inline int storage_elem_bytes(int storage) {
  switch (storage) {
    case GROM_F64: return 8;
    case GROM_F32X2: return 8;
    case GROM_F32: return 4;
    case GROM_BF16: return 2;
  }
  return 0;
}

}  // namespace grom

#include "k1_types.h"

namespace grom {

// NVTX range over a library call, shown by Nsight tools on the host timeline
// next to the kernels it launches; a no-op when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// m = 0: the G-ROM (middle extent n, weights u); m > 0: middle extent m with
// separate weights (the SVD-ROM)
K1Plan k1_plan(int64_t n, int storage, int sm_count, int packed = 0, int64_t m = 0);
cudaError_t k1_launch(const K1Plan& plan, int storage, const K1Args& a, int batch, cudaStream_t s);

// ------------------------------------------------- K2 (tensor cores, BF16)
struct K2Plan {
  int64_t n, np;
  int btile;       // trajectories per column tile (multiple of 16, <= 256)
  int col_tiles;   // column tiles
  int i_tiles;     // 128-row tiles of the test index
  int splits;      // split of the K range (advecting index j) across CTAs
  int stages_a;    // pipeline depth of the C tiles
  int stages_b;    // pipeline depth of the KR tiles (hi and lo)
  int tmem_cols;   // allocated tensor-memory columns
  int64_t bp;      // padded batch
  size_t smem;
};
struct K2Args {
  const double* u;
  int64_t u_stride;
  double* c;
  int64_t c_stride;
  double* hist;
  const int64_t* taken;
  int64_t hist_stride;
  const int32_t* active;
  int batch;
  void* scratch;  // k2_scratch_bytes(plan)
  int* err;
  cudaEvent_t ev0, ev1;
  // MTTKRP: factor matrices P (middle index) and Q (inner index), row-major
  // n x f_stride FP64 on the device; column b < batch is rank component b.
  // Null for the contraction with the states.
  const double* fp;
  const double* fq;
  int64_t f_stride;
  int tiled;  // 1: the tensor map covers the tile-major copy (k2_build_tiles)
};
// cuTensorMapEncodeTiled through the runtime's driver entry point (null when
// the CUDA driver does not provide it); looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn();
// splits_force > 0 replaces the rule's split of the advecting index (capped at n).
K2Plan k2_plan(int64_t n, int batch, int sm_count, int splits_force = 0);
size_t k2_scratch_bytes(const K2Plan& p);
bool k2_make_tmap(CUtensorMap* m, const void* tensor, int64_t n, int64_t np);
// Tile-major BF16 copy of the stored tensor for K2 (every 256 x 64 tile of
// C_(1) contiguous) and its tensor map.
size_t k2_tiles_bytes(int64_t n);
cudaError_t k2_build_tiles(const void* rows, int64_t n, void* tiles, cudaStream_t s);
bool k2_make_tmap_tiled(CUtensorMap* m, const void* tiles, int64_t n);
cudaError_t k2_launch(const K2Plan& p, const CUtensorMap* tmap, const K2Args& a, cudaStream_t s);

// ------------------- K2P (tensor cores, BF16, skew-packed layout, factored)
struct K2PPlan {
  int64_t n, np, lp;
  int btile;       // trajectories per column tile (multiple of 16, <= 128)
  int col_tiles;   // column tiles
  int pblks;       // 128-position blocks of a stored row
  int ctas;        // 1: one CTA per tile; 2: SM pairs (cta_group::2), one pair per two blocks
  int pbs;         // blocks in the tile numbering: pblks, rounded up to even for pairs
  int m;           // test indices per CTA tile
  int ranges;      // ceil(n / m)
  int tiles;       // CTA tiles: ranges * pbs * col_tiles
  int stages;      // pipeline depth (C tile + U hi/lo tiles)
  int tmem_cols;   // two accumulators of btile columns
  int wrows;       // rows of the mirrored-entry window (m + 127)
  int wpitch;      // its pitch in floats (btile + 1)
  int grid;        // persistent CTAs (pairs: even, at most the pairs that fit at once)
  int64_t bp;      // padded batch
  size_t smem;
};
// m_force replaces the rule's tile height when k2p_tile_m_ok admits it;
// ctas_force (1 or 2) the rule's kernel, 2 only where k2p_pair_ok.
K2PPlan k2p_plan(int64_t n, int64_t lp, int batch, int sm_count, int m_force = 0, int ctas_force = 0);
bool k2p_tile_m_ok(int batch, int m);
bool k2p_pair_ok(int64_t lp);
// Whether clusters of two K2P pair CTAs (at the largest shared memory a plan
// uses) fit on the current device at all.
bool k2p_pairs_supported();
// The CTA tile of CTA `rank` (0 leader, 1 peer) of pair tile t2: column tile
// ct, position block pb (2q + rank), test indices [i0, i1), and the CTA
// tile's index in the scratch (windows, the finish kernel's numbering).
__host__ __device__ inline void k2p_pair_coords(int t2, int rank, int col_tiles, int pbs, int m, int64_t n, int& ct,
                                                int& pb, int64_t& i0, int64_t& i1, int& tile) {
  ct = t2 % col_tiles;
  const int rest = t2 / col_tiles;
  const int halves = pbs >> 1;
  pb = 2 * (rest % halves) + rank;
  const int r = rest / halves;
  i0 = (int64_t)r * m;
  i1 = i0 + m < n ? i0 + m : n;
  tile = (r * pbs + pb) * col_tiles + ct;
}
// Scratch of the largest plan over every batch a ROM with max_batch accepts.
size_t k2_scratch_need(int64_t n, int max_batch, int sm_count);
size_t k2p_scratch_need(int64_t n, int64_t lp, int max_batch, int sm_count);
size_t k2p_scratch_bytes(const K2PPlan& p);
bool k2p_make_tmap(CUtensorMap* m, const void* packed, int64_t n, int64_t lp);
// Same arguments as K2 (fp/fq and tiled unused).
cudaError_t k2p_launch(const K2PPlan& p, const CUtensorMap* tmap, const K2Args& a, cudaStream_t s);

// ------------------------------------------------------------- K3 (CP)
constexpr int K3_THREADS = 256;
struct K3Plan {
  int64_t n, r, rb, nblk;  // rank, columns per block, blocks
  int nb_max;
  size_t smem;
};
struct K3Args {
  const uint8_t* fa;  // panel layout [nblk][n][rb] per factor
  const uint8_t* fb;
  const uint8_t* fc;
  int form;           // GROM_FORM_CP or GROM_FORM_CP_SKEW
  const double* u;
  int64_t u_stride;
  double* part;       // nblk x NB x n partial outputs
  double* c;
  int64_t c_stride;
  int nb;
  double* hist;
  const int64_t* taken;
  int64_t hist_stride;
  const int32_t* active;
};
K3Plan k3_plan(int64_t n, int64_t r, int storage, int sm_count);
cudaError_t k3_launch(const K3Plan& plan, int storage, const K3Args& a, int batch, cudaStream_t s);
struct StepArgs;
// CP evaluation with the diagonal step fused into the expansion kernel.
cudaError_t k3_launch_step(const K3Plan& p, int storage, const K3Args& a0, int batch, const StepArgs* st,
                           int step_index, cudaStream_t s);
int k3_expand_blocks(int64_t n);
// Batched CP form as register-tiled GEMMs (batches of 16 or more).
size_t k3g_scratch_bytes(int64_t n, int64_t rp, int max_batch, int storage, int sm_count);
cudaError_t k3g_launch(const K3Plan& p, int storage, const K3Args& a, int batch, int max_batch, void* scratch,
                       int sm_count, cudaStream_t s);
constexpr int K3G_MIN_BATCH = 16;
// AUTO steps FP64 CP batches (16 trajectories and more) on the tensor cores
// (K3O) from this much work per step (N R B) on, else with K3D (measured on
// GB300: N = R = 1024 at 16 trajectories 0.063 against 0.085 ms, at 1024
// 0.535 against 1.93 ms; 64 trajectories of N = 512, R = 256 0.035 against
// 0.034 ms, of N = R = 256 0.031 against 0.023 ms)
constexpr int64_t K3O_MIN_WORK = (int64_t)1 << 24;
// Batched CP form of FP64 ROMs at FP64 tolerance in double-single FP32
// arithmetic (K3D, same batch sizes as K3g): hi/lo copies of the factors
// made at create, then per step a state split and two GEMMs.
size_t k3d_factor_bytes(int64_t n, int64_t rp);
size_t k3d_scratch_bytes(int64_t n, int64_t rp, int max_batch, int sm_count);
cudaError_t k3d_build_factors(const uint8_t* op, size_t panel_bytes, int64_t n, int64_t rp, void* out,
                              cudaStream_t s);
cudaError_t k3d_launch(const K3Plan& p, const K3Args& a, const void* factors, int batch, int max_batch,
                       void* scratch, int sm_count, cudaStream_t s);
struct StepArgs;
// K3D evaluation of step step_index followed by the diagonal step, which sums
// the expansion's splits and writes the next state's hi/lo planes; the state
// planes are prepared from the ring only when prep is set (the first step of
// a call).  ev0/ev1 (optional) bracket the evaluation.
cudaError_t k3d_launch_step(const K3Plan& p, const K3Args& a, const void* factors, int batch, void* scratch,
                            int sm_count, bool prep, const StepArgs& st, int step_index, cudaEvent_t ev0,
                            cudaEvent_t ev1, cudaStream_t s);
// K3O: the batched CP form of FP64 ROMs on the BF16 tensor cores, every
// operand split into 7- or 6-bit integer digit slices (Sec. 3.1, eq. tc_ap).
bool k3o_supported(int64_t n, int64_t r, int form);
size_t k3o_factor_bytes(int64_t n, int64_t rp, int64_t r, int form);
size_t k3o_scratch_bytes(int64_t n, int64_t rp, int64_t r, int form, int max_batch);
cudaError_t k3o_build_factors(const uint8_t* op, size_t panel_bytes, int64_t n, int64_t rp, int64_t r, int form,
                              void* out, cudaStream_t s);
cudaError_t k3o_launch(int64_t n, int64_t rp, int64_t r, const K3Args& a, const void* factors, int batch,
                       void* scratch, int* err, int sm_count, cudaStream_t s);
// The same evaluation for stepping (a.hist/a.taken set): the expansion's
// combine and the diagonal BDF3/EXT3 step (the blocks of k_step_diag_mc)
// run as one kernel; the same bits as k3o_launch followed by the step.
cudaError_t k3o_launch_step(int64_t n, int64_t rp, int64_t r, const K3Args& a, const void* factors, int batch,
                            void* scratch, int* err, int sm_count, const StepArgs& st, int step_index,
                            cudaStream_t s);
cudaError_t k3o_gemm_launch(const void* A, int64_t M, int64_t mslice, const void* B, int64_t ncols,
                            int64_t nslice, int64_t K, int slices, float* out, int* err, int sm_count,
                            cudaStream_t s);
// Batched CP form on the tensor cores (BF16 factors): projections and
// expansion as two tcgen05 GEMMs over copies of the factors laid out for them.
struct K3TPlan {
  int64_t n, np, r, rp;  // rank padded to 64
  int nseg, nz;          // projection segments (2 general, 3 skew), expansion blocks (1, 2)
  int64_t m1, k1, m2, k2;
  int btile, ctiles;     // trajectories per column tile (<= 64 skew, <= 128 general), column tiles
  int64_t bp;
  int jtiles;            // 128-wide rank tiles of the projection kernel
  int s1, s2;            // K splits of the two GEMMs
  int s1_max, s2_max;    // their largest admissible values
  int stages_p, tmem_p;  // projection kernel: pipeline stages, tensor-memory columns
  size_t smem_p;
  int stages, tmem_cols; // expansion kernel
  size_t smem;
};
constexpr int K3T_MIN_BATCH = 16;
constexpr int K3T_MAX_CTILES = 1024;  // column tiles (batch / btile) the counter region covers
// The expansion's trajectory-major split partials, summed by the step kernel
// (which also writes the next state's hi/lo rows for the projections).
// K3T: s2 x bp x n FP32 partials, BF16 rows [b][i] of pitch np; K3D:
// s2 x (hi, lo) x bp x n double-single partials (bp = the batch), FP32
// planes [i][b] of pitch np.
struct K3TStepFuse {
  const float* d2;
  int s2;
  int64_t bp, np;
  void* xh;         // bp x np (hi), then xl (lo)
  void* xl;
};
// s1_force, s2_force in [1, s1_max] / [1, s2_max] replace the rule's splits.
K3TPlan k3t_plan(int64_t n, int64_t r, int form, int batch, int sm_count, int s1_force = 0, int s2_force = 0);
size_t k3t_scratch_bytes(const K3TPlan& p);
size_t k3t_scratch_need(int64_t n, int64_t r, int form, int max_batch, int sm_count);
size_t k3t_factor_bytes(int64_t n, int64_t r, int form);
cudaError_t k3t_build_factors(const void* fa, const void* fb, const void* fc, int64_t n, int64_t rb, int64_t r,
                              int form, void* ft, void* ae, cudaStream_t s);
size_t k3t_counter_bytes(const K3TPlan& p);
bool k3t_make_tmaps(CUtensorMap* m_ft, CUtensorMap* m_ae, const void* ft, const void* ae, int64_t n, int64_t r,
                    int form);
cudaError_t k3t_launch(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a, int batch,
                       void* scratch, int* err, cudaStream_t s);
// One diagonal BDF step of the batch with the K3T evaluation: the state prep
// (when `prep`; the step kernel keeps the BF16 state rows current after
// that), the projection and expansion kernels (between ev0 and ev1 when
// set), then the step kernel summing the expansion's splits.
cudaError_t k3t_launch_step(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a,
                            int batch, void* scratch, int* err, bool prep, const StepArgs& st, int step_index,
                            cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t s);
// Persistent batched stepper: nsteps diagonal steps of the batch in one
// cooperative launch of one CTA per SM (projection, expansion and step
// phases between grid barriers; the same tiles and arithmetic as the
// per-step kernels).  Returns an error without launching when the plan or
// the device does not allow it; the caller then takes the per-step path.
size_t k3tp_smem(const K3TPlan& p);
constexpr int64_t K3TP_MAX_ELEMENTS = 1 << 18;  // batch x n up to which grom_step takes the persistent stepper
cudaError_t k3tp_launch(const K3TPlan& p, const CUtensorMap* m_ft, const CUtensorMap* m_ae, const K3Args& a,
                        int batch, void* scratch, int* err, const StepArgs& st, int nsteps, int sm_count,
                        cudaStream_t s);
// Persistent cooperative CPD-ROM stepper for a few trajectories.
size_t k3p_scratch_bytes(int64_t n, int64_t rp, int storage, int sm_count);
int k3p_max_batch(int storage);
bool k3p_fits(int64_t n, int64_t rp, int storage, int batch, int sm_count);
cudaError_t k3p_launch(const uint8_t* fa, const uint8_t* fb, const uint8_t* fc, int form, int64_t n, int64_t rp,
                       int storage, int batch, int nsteps, const StepArgs& st, void* scratch, int sm_count,
                       cudaStream_t s);

// --------------------------------------------------------------- stepper
struct StepArgs {
  int64_t n;
  int batch;
  int order;
  double dt, nu;
  double inv_dt;         // 1 / dt, rounded once on the host (FP64 division is slow on the device)
  double bdt[3][3];      // beta_{q+1} / dt of BDF order k (rows k = 1..3), from the host
  double* hist;          // batch x 6 x n ring (u slots 0..2, n slots 3..5)
  int64_t hist_stride;   // 6 * n
  int64_t* taken;        // batch
  const int32_t* active; // nullable
  // diagonal path
  const double* hdiag[3];   // 1 / (beta0_k/dt b_i + nu a_i), k = 1..3
  const double* mass_diag;  // nullable (identity)
  const double* lin_diag;   // nullable
  const double* forcing;    // nullable
  // dense path
  const double* hinv[3];    // n x n inverses of H_k (nullable when diagonal)
  const double* mass;       // dense B (nullable)
  const double* linear;     // dense L (nullable)
  double* work;             // batch x 4 x n scratch for the dense path
  // outputs
  double* energy;           // nullable, (step) x batch
  double* invariant;        // nullable
  int* err;                 // device error flags
  int* first_bad;           // first non-finite trajectory (atomicMin)
  // multi-CTA diagonal step: per-CTA partial sums and arrival counters
  double* red;              // batch x nblk x 2
  unsigned int* cnt;        // batch (zero between launches)
  int nblk;                 // CTAs per trajectory
  int ept;                  // elements per thread of the multi-CTA diagonal step
  // serving: per-trajectory remaining steps; a trajectory whose count
  // reaches zero is deactivated (active[b] = 0) by the step that ends it
  int32_t* steps_left;      // nullable
  int32_t* active_rw;       // writable view of `active` (same array)
};
// Ends the step of trajectory b: advance its count, retire it when its
// serving budget runs out.
__device__ __forceinline__ void step_done(const StepArgs& a, int b, int64_t l) {
  a.taken[b] = l + 1;
  if (a.steps_left) {
    const int32_t left = a.steps_left[b] - 1;
    a.steps_left[b] = left;
    if (left <= 0) a.active_rw[b] = 0;
  }
}
// The common case of the diagonal step: identity mass, no linear or forcing
// term and no energy or invariant asked for (the PLAIN kernel variants).
inline bool step_plain(const StepArgs& a) {
  return !a.mass_diag && !a.lin_diag && !a.forcing && !a.energy && !a.invariant;
}
constexpr int STEP_MC_THREADS = 128;
inline int step_mc_blocks(int64_t n) { return (int)((n + STEP_MC_THREADS - 1) / STEP_MC_THREADS); }
// fused finalize + step of the skew-packed streaming kernel: 32 test indices per block
constexpr int STEP_PK_THREADS = 1024;
constexpr int STEP_PK_MAX_GRID = 1024;  // streaming CTAs whose window starts fit the block's table
inline int step_pk_blocks(int64_t n) { return (int)((n + 31) / 32); }
// Diagonal step over several CTAs per trajectory.  With k1 != nullptr the
// K1 partial sums of trajectories b0 .. b0+nb-1 are finalised in the same
// kernel (the advection term is written to the history ring first).
cudaError_t step_diag_mc_launch(const StepArgs& a, int step_index, const K1Plan* k1, const K1Args* k1a, int b0, int nb,
                                int nbk, cudaStream_t s);
// The same step for the whole batch with n^l summed from K3T's expansion
// partials (written to the history ring) and the new state also written as
// BF16 hi/lo rows for the next projections.
cudaError_t step_diag_mc_k3t_launch(const StepArgs& a, int step_index, const K3TStepFuse& f, cudaStream_t s);
cudaError_t step_diag_mc_k3d_launch(const StepArgs& a, int step_index, const K3TStepFuse& f, cudaStream_t s);
cudaError_t step_diag_packed_launch(const StepArgs& a, int step_index, const K1Plan& pl, const K1Args& k1a, int b0,
                                    int nb, int nbk, cudaStream_t s);
// Persistent skew-packed stepper (k1p_persist.cuh): nsteps diagonal steps of
// up to 4 trajectories in one cooperative launch.  scratch: k1pp_scratch_bytes,
// zeroed once at creation.  Returns an error without launching when the plan
// or the device does not allow it (the caller then takes the regular path).
size_t k1pp_scratch_bytes(const K1Plan& p);
cudaError_t k1pp_launch(const K1Plan& plan, int storage, const K1Args& a, const StepArgs& st, int batch, int nsteps,
                        void* scratch, cudaStream_t s);
cudaError_t k1_launch_fused_step(const K1Plan& plan, int storage, const K1Args& a, const StepArgs& st, int batch,
                                 int step_index, cudaStream_t s);
cudaError_t selftest_wait_launch(int* err, uint64_t limit_ns, cudaStream_t s);
cudaError_t slot_admit_launch(double* hist, int64_t* taken, int32_t* steps_left, int32_t* active, int64_t n,
                              int count, const int32_t* slots, const int32_t* horizons, const double* u0s,
                              cudaStream_t s);
// Copies u (batch x n, device) into / out of the newest-state slot of the ring.
cudaError_t state_io_launch(double* hist, const int64_t* taken, int64_t n, int batch, double* u, bool inject,
                            cudaStream_t s);

// ------------------------------------------------------------ conversion
cudaError_t convert_rows_launch(const double* src, int64_t rows, int64_t n, int64_t np,
                                int storage, uint8_t* dst, cudaStream_t s);
// Dense FP64 rows (i, j) of n values, m rows per test index, for i from i0
// -> skew-packed stored rows (position p holds the value at k = (i + 1 + p) mod n).
cudaError_t convert_rows_packed_launch(const double* src, int64_t rows, int64_t n, int64_t m, int64_t i0, int64_t lp,
                                       int storage, uint8_t* dst, cudaStream_t s);
// Adds the skew probes of FP64 rows (i, j) (m rows per test index, i from
// i0) into acc[0..2] (probe 1, probe 2, sum of squares).
cudaError_t skew_probe_launch(const double* src, int64_t rows, int64_t n, int64_t m, int64_t i0, double* acc,
                              cudaStream_t s);
// Augmented tensor slab (cnt test indices of (n+1) x (n+1) values, index 0
// the zeroth mode) -> the core rows (cnt x n x n) and, for those test
// indices, L_ik = Cbar[i][0][k+1] + Cbar[i][k+1][0] and f_i = Cbar[i][0][0].
cudaError_t aug_split_launch(const double* src, int64_t cnt, int64_t n, double* core, double* L, double* f,
                             cudaStream_t s);
// SVD-ROM middle weights beta[b][r] = sigma_r sum_j U_jr u_bj (k_svd.cu).
cudaError_t svd_project_launch(const double* ut, const double* sigma, int64_t n, int64_t rank, int batch,
                               const double* u, int64_t u_stride, const double* hist, const int64_t* taken,
                               int64_t hist_stride, const int32_t* active, double* beta, cudaStream_t s);
cudaError_t convert_panels_launch(const double* src, int64_t n, int64_t r, int64_t rb,
                                  int storage, uint8_t* dst, cudaStream_t s);

}  // namespace grom

// ------------------------------------------------------------ ROM objects
struct grom_rom {
  int n = 0, form = 0, rank = 0, storage = 0, order = 3, max_batch = 1, layout = 0;
  int64_t np = 0;
  double nu = 0, dt = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  uint8_t* op = nullptr;  // stored tensor, or three CP factor panel sets
  size_t op_bytes = 0;
  size_t panel_bytes = 0;
  int64_t rows_uploaded = 0;
  uint8_t* row_seen = nullptr;  // host bitmap of uploaded rows (deferred tensor)
  bool diagonal = true;
  double* hdiag = nullptr;      // 3 x n
  double* hinv = nullptr;       // 3 x n x n (dense path)
  double* mass = nullptr;       // n x n
  double* mass_diag = nullptr;  // n
  double* linear = nullptr;     // n x n
  double* lin_diag = nullptr;   // n
  double* forcing = nullptr;    // n
  double* part = nullptr;       // streaming / CP partials
  size_t part_bytes = 0;
  int* err = nullptr;           // device flags [0] = mask, [1] = first bad
  void* k1pp_scratch = nullptr; // packed layout: persistent stepper barrier and partials
  void* k1p_dg = nullptr;       // packed layout: segment values D u_i
  double* k1p_tg = nullptr;     // packed layout: transposed-term windows
  double* probe = nullptr;      // packed layout: skew probe accumulators (3)
  double* svd_ut = nullptr;     // SVD form: U^T (rank x n)
  double* svd_sigma = nullptr;  // SVD form: singular values (rank)
  double* svd_beta = nullptr;   // SVD form: middle weights (max_batch x rank)
  grom::K1Plan k1{};
  grom::K3Plan k3{};
  size_t total_bytes = 0;
  int traj_count = 0;
  int kernel_choice = 0;             // GROM_KERNEL_* override
  int version = 0;                   // bumped when cached launch graphs become stale
  bool k2_ok = false;                // tensor map built (BF16 full form; K2P's map for the packed layout)
  bool k2p_pairs = false;            // clusters of two fit on this device: K2P may run on SM pairs
  CUtensorMap k2_tmap;               // TMA descriptor of the stored tensor
  void* k2_tiles = nullptr;          // tile-major copy for K2 (nullable)
  bool no_tile_copy = false;         // grom_desc.no_tile_copy
  CUtensorMap k2_tmap_tiled;         // its TMA descriptor
  void* k2_scratch = nullptr;        // K2 state copy + split-K partials
  void* k3g_scratch = nullptr;       // batched CP: Hadamard products H1, H2
  void* k3d_factors = nullptr;       // batched FP64 CP in double-single arithmetic: hi/lo factor planes
  void* k3d_scratch = nullptr;       // its states, products and split partials
  void* k3o_factors = nullptr;       // batched FP64 CP on sliced BF16 tensor cores: factor digits and scales
  void* k3o_scratch = nullptr;       // its state and H digits and slice products
  void* k3t_factors = nullptr;       // batched CP on tensor cores: FT | AE (BF16)
  void* k3t_scratch = nullptr;
  CUtensorMap k3t_tmap_ft, k3t_tmap_ae;
  void* k3p_scratch = nullptr;       // persistent CP stepper: partials, h, barrier
  size_t k2_scratch_bytes = 0;
  size_t k3t_scratch_bytes = 0;
  std::vector<grom_tuning> tuning;   // per batch bucket ceil(batch / 16); kernel 0: untuned
  bool prof = false;                 // kernel timing enabled
  std::vector<cudaEvent_t> prof_ev;  // start/stop pairs
  size_t prof_used = 0;              // pairs recorded since enable
};

struct grom_traj {
  grom_rom* rom = nullptr;
  int batch = 0;
  double* hist = nullptr;   // batch x 6 x n
  int64_t* taken = nullptr; // batch
  double* work = nullptr;   // dense-path scratch batch x 4 x n
  int* err = nullptr;       // [0] mask, [1] first bad trajectory
  double* io = nullptr;     // batch x n staging for grom_step_host
  double* red = nullptr;    // multi-CTA step partials
  unsigned int* cnt = nullptr;
  cudaGraphExec_t graph = nullptr;  // captured block of steps (no per-step outputs)
  cudaGraph_t graph_tmpl = nullptr; // its template (kept for event-node updates)
  int graph_steps = 0;
  int graph_version = -1;
  // kernel-timing event nodes of a graph captured with profiling on: node and
  // its index in the graph's event sequence (pair k: 2k start, 2k + 1 stop)
  std::vector<cudaGraphNode_t> prof_nodes;
  std::vector<int> prof_index;
  int prof_pairs = 0;
  // grom_step_host as one captured graph (state in, steps, state out) for a
  // given pair of buffers and step count
  cudaGraphExec_t io_graph = nullptr;
  const void* io_in = nullptr;
  void* io_out = nullptr;
  int io_steps = 0;
  int io_version = -1;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int32_t* active = nullptr;      // serving slots: 1 = occupied (nullable: all active)
  int32_t* steps_left = nullptr;  // serving slots: remaining steps
};
