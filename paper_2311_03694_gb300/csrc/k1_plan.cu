// K1 launch planning: chunking, persistent grid, trajectories per pass.
#include "k1_stream.cuh"
#include "k1p_persist.cuh"

namespace grom {

cudaError_t k1_dispatch_f64(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1_dispatch_f32x2(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1_dispatch_f32(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1_dispatch_bf16(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1p_dispatch_f64(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1p_dispatch_f32x2(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1p_dispatch_f32(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1p_dispatch_bf16(int qm, int nb, const K1Plan&, const K1Args&, int, cudaStream_t);
cudaError_t k1pp_dispatch_f64(int, int, const K1Plan&, const K1Args&, const StepArgs&, const K1PPArgs&, cudaStream_t);
cudaError_t k1pp_dispatch_f32x2(int, int, const K1Plan&, const K1Args&, const StepArgs&, const K1PPArgs&, cudaStream_t);
cudaError_t k1pp_dispatch_f32(int, int, const K1Plan&, const K1Args&, const StepArgs&, const K1PPArgs&, cudaStream_t);
cudaError_t k1pp_dispatch_bf16(int, int, const K1Plan&, const K1Args&, const StepArgs&, const K1PPArgs&, cudaStream_t);

static int pow2_ceil(int64_t x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

static int acc_regs(int storage) {
  switch (storage) {
    case GROM_F64: return 4;    // 2 elements x 2 words
    case GROM_F32X2: return 16;  // 4 elements x (S, s), plus hi and lo vectors held per chunk
    case GROM_F32: return 4;
    case GROM_BF16: return 8;
  }
  return 64;
}

static int epv(int storage) {
  switch (storage) {
    case GROM_F64: return 2;
    case GROM_F32X2: return 4;
    case GROM_F32: return 4;
    case GROM_BF16: return 8;
  }
  return 1;
}

// Shared-memory bytes per trajectory of a pass: u (np values) and, with
// separate middle weights, those (mp values), in the storage's arithmetic
// type (F32X2: hi and lo floats).
static int64_t k1_traj_smem(const K1Plan& p, int storage) {
  const int64_t ub = (storage == GROM_F64 || storage == GROM_F32X2) ? 8 : 4;
  return (p.np + (p.has_mid ? p.mp : 0)) * ub;
}

static constexpr int64_t K1_SMEM_BASE = 1024 + K1_STAGES * K1_STAGE_BYTES + 2 * K1_STAGES * 8 + 16;

K1Plan k1_plan(int64_t n, int storage, int sm_count, int packed, int64_t m) {
  K1Plan p{};
  p.n = n;
  p.np = padded_n(n);
  p.has_mid = m > 0 ? 1 : 0;
  p.m = m > 0 ? m : n;
  p.mp = padded_n(p.m);
  p.packed = packed;
  p.h = n / 2;
  p.lp = packed ? padded_n(p.h > 0 ? p.h : 1) : p.np;
  p.row_bytes = p.lp * storage_elem_bytes(storage);
  // vector positions per row and the consumer mapping (see k1_stream.cuh and
  // k1_packed.cuh)
  const int64_t P = p.lp / epv(storage);
  int64_t rpr;
  if (packed) {
    // up to four row groups per position, kept inside one warp
    int64_t R = 1;
    while (R < 4 && 2 * R * P <= K1_CONSUMERS) R *= 2;
    p.rg = (int)R;
    const int64_t W = K1_CONSUMERS / R;
    p.qm = pow2_ceil((P + W - 1) / W);
    rpr = R;
  } else {
    p.rg = 1;
    p.qm = pow2_ceil((P + K1_CONSUMERS - 1) / K1_CONSUMERS);
    rpr = P >= K1_CONSUMERS ? 1 : K1_CONSUMERS / P;
  }
  const int64_t rmax = k1_rmax(p.qm, storage == GROM_F32X2 ? 2 : 1);  // rows a consumer thread holds per chunk
  p.rpc = K1_STAGE_BYTES / p.row_bytes;
  if (p.rpc > rmax * rpr) p.rpc = rmax * rpr;
  if (p.rpc < 1) p.rpc = 1;
  if (p.rpc > p.m) p.rpc = p.m;
  p.cpi = (p.m + p.rpc - 1) / p.rpc;
  p.T = n * p.cpi;
  int64_t grid = sm_count;  // one persistent CTA per SM (the stage ring fills most of shared memory)
  if (grid > p.T) grid = p.T;
  if (grid < 1) grid = 1;
  p.grid = (int)grid;
  const int64_t per = (p.T + grid - 1) / grid;
  p.maxseg = (int)((per + p.cpi - 1) / p.cpi + 1);
  const int64_t per_traj = k1_traj_smem(p, storage);
  const int64_t budget = 227 * 1024 - K1_SMEM_BASE;
  int nb = 8;
  while (nb > 1 && (acc_regs(storage) * p.qm * nb > 64 || nb * per_traj > budget)) nb >>= 1;
  p.nb_max = nb;
  p.smem = (size_t)(K1_SMEM_BASE + nb * per_traj);
  p.lw = p.maxseg - 1 + p.lp;
  return p;
}

int64_t k1_row_step(const K1Plan& p, int storage) {
  if (p.packed) return p.rg;
  const int64_t P = p.lp / epv(storage);
  return P >= K1_CONSUMERS ? 1 : K1_CONSUMERS / P;
}

size_t k1p_dg_bytes(const K1Plan& p, int storage) {
  const size_t rs = (storage == GROM_F64 || storage == GROM_F32X2) ? 8 : 4;
  return (size_t)p.grid * p.maxseg * p.nb_max * p.lp * rs;
}

size_t k1p_tg_bytes(const K1Plan& p) { return (size_t)p.grid * p.nb_max * p.lw * sizeof(double); }

static cudaError_t k1_dispatch(const K1Plan& pl, int storage, int nb, const K1Args& a, int b0, cudaStream_t s) {
  if (pl.packed) {
    switch (storage) {
      case GROM_F64: return k1p_dispatch_f64(pl.qm, nb, pl, a, b0, s);
      case GROM_F32X2: return k1p_dispatch_f32x2(pl.qm, nb, pl, a, b0, s);
      case GROM_F32: return k1p_dispatch_f32(pl.qm, nb, pl, a, b0, s);
      case GROM_BF16: return k1p_dispatch_bf16(pl.qm, nb, pl, a, b0, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (storage) {
    case GROM_F64: return k1_dispatch_f64(pl.qm, nb, pl, a, b0, s);
    case GROM_F32X2: return k1_dispatch_f32x2(pl.qm, nb, pl, a, b0, s);
    case GROM_F32: return k1_dispatch_f32(pl.qm, nb, pl, a, b0, s);
    case GROM_BF16: return k1_dispatch_bf16(pl.qm, nb, pl, a, b0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t k1_launch(const K1Plan& plan, int storage, const K1Args& a0, int batch, cudaStream_t s) {
  for (int b0 = 0; b0 < batch; b0 += plan.nb_max) {
    K1Args a = a0;
    const int rem = batch - b0;
    a.nb = rem < plan.nb_max ? rem : plan.nb_max;
    const int nb = pow2_ceil(a.nb);
    K1Plan pl = plan;
    // shared memory for the template width actually launched
    pl.smem = (size_t)(K1_SMEM_BASE + nb * k1_traj_smem(pl, storage));
    cudaError_t e = k1_dispatch(pl, storage, nb, a, b0, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace grom

namespace grom {

cudaError_t k1_launch_fused_step(const K1Plan& plan, int storage, const K1Args& a0, const StepArgs& st, int batch,
                                 int step_index, cudaStream_t s) {
  for (int b0 = 0; b0 < batch; b0 += plan.nb_max) {
    K1Args a = a0;
    const int rem = batch - b0;
    a.nb = rem < plan.nb_max ? rem : plan.nb_max;
    // the finalize (dense or packed) is fused into the step kernel
    a.skip_finalize = 1;
    const int nb = pow2_ceil(a.nb);
    K1Plan pl = plan;
    pl.smem = (size_t)(K1_SMEM_BASE + nb * k1_traj_smem(pl, storage));
    cudaError_t e = k1_dispatch(pl, storage, nb, a, b0, s);
    if (e != cudaSuccess) return e;
    e = plan.packed ? step_diag_packed_launch(st, step_index, pl, a, b0, a.nb, nb, s)
                    : step_diag_mc_launch(st, step_index, &pl, &a, b0, a.nb, nb, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace grom

namespace grom {

size_t k1pp_scratch_bytes(const K1Plan& p) { return 256 + (size_t)p.grid * 4 * 2 * sizeof(double); }

cudaError_t k1pp_launch(const K1Plan& plan, int storage, const K1Args& a0, const StepArgs& st, int batch, int nsteps,
                        void* scratch, cudaStream_t s) {
  if (!plan.packed || plan.has_mid || batch < 1 || batch > 4 || batch > plan.nb_max || nsteps < 1)
    return cudaErrorInvalidValue;
  K1Args a = a0;
  a.nb = batch;
  a.skip_finalize = 1;
  const int nb = pow2_ceil(batch);
  K1Plan pl = plan;
  pl.smem = (size_t)(K1_SMEM_BASE + nb * k1_traj_smem(pl, storage));
  K1PPArgs pp{};
  pp.bar = reinterpret_cast<unsigned int*>(scratch);
  pp.red = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(scratch) + 256);
  pp.nsteps = nsteps;
  switch (storage) {
    case GROM_F64: return k1pp_dispatch_f64(pl.qm, nb, pl, a, st, pp, s);
    case GROM_F32X2: return k1pp_dispatch_f32x2(pl.qm, nb, pl, a, st, pp, s);
    case GROM_F32: return k1pp_dispatch_f32(pl.qm, nb, pl, a, st, pp, s);
    case GROM_BF16: return k1pp_dispatch_bf16(pl.qm, nb, pl, a, st, pp, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace grom
