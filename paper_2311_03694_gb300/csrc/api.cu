// C ABI of the Galerkin ROM library: object lifetime, uploads, dispatch.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "grom_internal.h"

namespace grom {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

grom_status fail(grom_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

grom_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GROM_ERR_OOM : GROM_ERR_CUDA;
}

size_t k3_scratch_bytes(const K3Plan& p, int storage);
cudaError_t step_launch_indexed(const StepArgs& a, bool diagonal, int step_index, cudaStream_t s);

static const double kBeta0[3] = {1.0, 1.5, 11.0 / 6.0};

// Host FP64 Cholesky of an SPD matrix and explicit inverse (dense path only).
static bool spd_inverse(int64_t n, std::vector<double>& H, std::vector<double>& Hinv) {
  std::vector<double> L((size_t)(n * n), 0.0);
  for (int64_t j = 0; j < n; ++j) {
    double d = H[j * n + j];
    for (int64_t m = 0; m < j; ++m) d -= L[j * n + m] * L[j * n + m];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = H[i * n + j];
      for (int64_t m = 0; m < j; ++m) s -= L[i * n + m] * L[j * n + m];
      L[i * n + j] = s / ljj;
    }
  }
  Hinv.assign((size_t)(n * n), 0.0);
  std::vector<double> x((size_t)n);
  for (int64_t c = 0; c < n; ++c) {  // solve L L^T x = e_c
    for (int64_t i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int64_t m = 0; m < i; ++m) s -= L[i * n + m] * x[m];
      x[i] = s / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = x[i];
      for (int64_t m = i + 1; m < n; ++m) s -= L[m * n + i] * x[m];
      x[i] = s / L[i * n + i];
    }
    for (int64_t i = 0; i < n; ++i) Hinv[i * n + c] = x[i];
  }
  return true;
}

static grom_status fetch(std::vector<double>& dst, const double* src, size_t count) {
  dst.resize(count);
  GROM_CUDA_TRY(cudaMemcpy(dst.data(), src, count * sizeof(double), cudaMemcpyDefault));
  return GROM_OK;
}

template <typename T>
static grom_status dmalloc(T** p, size_t bytes, size_t* total) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? GROM_ERR_OOM : GROM_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  if (total) *total += bytes;
  return GROM_OK;
}

static grom_status upload(double** dst, const double* src, size_t count, size_t* total, cudaStream_t s) {
  grom_status st = dmalloc(dst, count * sizeof(double), total);
  if (st) return st;
  GROM_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(double), cudaMemcpyDefault, s));
  return GROM_OK;
}

// Streams FP64 rows (rows of `width` doubles) through a staging buffer and
// converts them into the storage layout.
static grom_status upload_rows(grom_rom* r, const double* src, int64_t rows, int64_t width, int64_t pitch,
                               uint8_t* dst, int64_t dst_row_bytes) {
  const int64_t stage_rows_max = std::max<int64_t>(1, (int64_t)(256ll << 20) / (width * 8));
  double* stage = nullptr;
  const int64_t srows = std::min(rows, stage_rows_max);
  grom_status st = dmalloc(&stage, (size_t)(srows * width * 8), nullptr);
  if (st) return st;
  for (int64_t r0 = 0; r0 < rows; r0 += srows) {
    const int64_t cnt = std::min(srows, rows - r0);
    cudaError_t e = cudaMemcpyAsync(stage, src + r0 * width, (size_t)(cnt * width * 8), cudaMemcpyDefault, r->stream);
    if (e == cudaSuccess) e = convert_rows_launch(stage, cnt, width, pitch, r->storage, dst + r0 * dst_row_bytes, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) {
      cudaFree(stage);
      return cuda_fail(e, "tensor upload");
    }
  }
  cudaFree(stage);
  return GROM_OK;
}

// Streams dense FP64 tensor rows (i, j) for test indices [i0, i1) through a
// staging buffer into the skew-packed layout, adding their skew probes.
static grom_status upload_rows_packed(grom_rom* r, const double* src, int64_t i0, int64_t i1) {
  const int64_t n = r->n, m = r->k1.m;
  const int64_t per_i = m * n;  // doubles per test index
  const int64_t si = std::max<int64_t>(1, (int64_t)(256ll << 20) / (per_i * 8));
  double* stage = nullptr;
  grom_status st = dmalloc(&stage, (size_t)(std::min(si, i1 - i0) * per_i * 8), nullptr);
  if (st) return st;
  for (int64_t a = i0; a < i1; a += si) {
    const int64_t cnt = std::min(si, i1 - a);
    cudaError_t e = cudaMemcpyAsync(stage, src + (a - i0) * per_i, (size_t)(cnt * per_i * 8), cudaMemcpyDefault, r->stream);
    if (e == cudaSuccess) e = skew_probe_launch(stage, cnt * m, n, m, a, r->probe, r->stream);
    if (e == cudaSuccess)
      e = convert_rows_packed_launch(stage, cnt * m, n, m, a, r->k1.lp, r->storage, r->op + a * m * r->k1.row_bytes,
                                     r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) {
      cudaFree(stage);
      return cuda_fail(e, "tensor upload");
    }
  }
  cudaFree(stage);
  return GROM_OK;
}

// Augmented FULL tensor (n x (n+1) x (n+1), index 0 the zeroth mode): the
// core rows are converted like a plain tensor (dense or skew-packed), and the
// zeroth-mode terms L = C1 + C2 and f = c0 come back on the host.
static grom_status check_skew_probe(grom_rom* r);
static grom_status upload_augmented_full(grom_rom* r, const double* src, std::vector<double>& L, std::vector<double>& f) {
  const int64_t n = r->n, n1 = n + 1;
  const int64_t per_src = n1 * n1, per_core = n * n;  // doubles per test index
  const int64_t si = std::min<int64_t>(n, std::max<int64_t>(1, (int64_t)(256ll << 20) / (per_src * 8)));
  const bool packed = r->layout == GROM_LAYOUT_SKEW_PACKED;
  double *stage = nullptr, *core = nullptr, *dl = nullptr, *df = nullptr;
  grom_status st = dmalloc(&stage, (size_t)(si * per_src * 8), nullptr);
  if (!st) st = dmalloc(&core, (size_t)(si * per_core * 8), nullptr);
  if (!st) st = dmalloc(&dl, (size_t)(n * n * 8), nullptr);
  if (!st) st = dmalloc(&df, (size_t)(n * 8), nullptr);
  cudaError_t e = cudaSuccess;
  for (int64_t a = 0; !st && e == cudaSuccess && a < n; a += si) {
    const int64_t cnt = std::min(si, n - a);
    e = cudaMemcpyAsync(stage, src + a * per_src, (size_t)(cnt * per_src * 8), cudaMemcpyDefault, r->stream);
    if (e == cudaSuccess) e = aug_split_launch(stage, cnt, n, core, dl + a * n, df + a, r->stream);
    if (e == cudaSuccess && packed) {
      e = skew_probe_launch(core, cnt * n, n, n, a, r->probe, r->stream);
      if (e == cudaSuccess)
        e = convert_rows_packed_launch(core, cnt * n, n, n, a, r->k1.lp, r->storage, r->op + a * n * r->k1.row_bytes,
                                       r->stream);
    } else if (e == cudaSuccess) {
      e = convert_rows_launch(core, cnt * n, n, r->np, r->storage, r->op + a * n * r->k1.row_bytes, r->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  }
  if (!st && e == cudaSuccess) {
    L.resize((size_t)(n * n));
    f.resize((size_t)n);
    e = cudaMemcpy(L.data(), dl, (size_t)(n * n * 8), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(f.data(), df, (size_t)(n * 8), cudaMemcpyDeviceToHost);
  }
  for (double* p : {stage, core, dl, df})
    if (p) cudaFree(p);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "augmented tensor upload");
  return packed ? check_skew_probe(r) : GROM_OK;
}

// After the last row: the probes of a skew tensor vanish up to rounding.
static grom_status check_skew_probe(grom_rom* r) {
  double acc[3];
  GROM_CUDA_TRY(cudaMemcpy(acc, r->probe, sizeof(acc), cudaMemcpyDeviceToHost));
  const double fro = std::sqrt(acc[2]);
  if (!(std::fabs(acc[0]) <= 1e-9 * fro) || !(std::fabs(acc[1]) <= 1e-9 * fro))
    return fail(GROM_ERR_INVALID_ARG,
                "skew-packed layout: the tensor is not skew in its test and advected index (C_ijk = -C_kji)");
  return GROM_OK;
}

// Tile-major copy of a dense BF16 tensor for the tensor-core kernel (built
// once, outside any stream capture).
static grom_status build_k2_tiles(grom_rom* r) {
  if (r->k2_tiles || !r->k2_ok || r->no_tile_copy || r->form != GROM_FORM_FULL || r->layout != GROM_LAYOUT_DENSE ||
      r->rows_uploaded != r->n)
    return GROM_OK;
  // the copy only speeds K2 up: without room for it K2 reads the row-major tensor
  grom_status st = dmalloc(&r->k2_tiles, k2_tiles_bytes(r->n), &r->total_bytes);
  if (st) return st == GROM_ERR_OOM ? GROM_OK : st;
  cudaError_t e = k2_build_tiles(r->op, r->n, r->k2_tiles, r->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess || !k2_make_tmap_tiled(&r->k2_tmap_tiled, r->k2_tiles, r->n)) {
    cudaGetLastError();
    cudaFree(r->k2_tiles);
    r->total_bytes -= k2_tiles_bytes(r->n);
    r->k2_tiles = nullptr;
    return e != cudaSuccess ? cuda_fail(e, "tile-major copy") : GROM_OK;
  }
  ++r->version;  // captured graphs hold the other tensor map
  return GROM_OK;
}

static void rom_free(grom_rom* r) {
  if (!r) return;
  void* ptrs[] = {r->op,     r->hdiag,   r->hinv, r->mass, r->mass_diag, r->linear,
                  r->lin_diag, r->forcing, r->part, r->err,  r->k2_scratch, r->k3g_scratch, r->k3p_scratch,
                  r->k3t_factors, r->k3t_scratch, r->k3d_factors, r->k3d_scratch, r->k3o_factors, r->k3o_scratch,
                  r->k1p_dg, r->k1p_tg, r->probe, r->svd_ut, r->svd_sigma, r->svd_beta, r->k1pp_scratch,
                  r->k2_tiles};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : r->prof_ev) cudaEventDestroy(e);
  delete[] r->row_seen;
  delete r;
}

static bool full_ready(const grom_rom* r) { return r->form != GROM_FORM_FULL || r->rows_uploaded == r->n; }

// Next start/stop event pair for kernel timing (nullptr when disabled).
static bool prof_pair(grom_rom* r, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  if (!r->prof) return true;
  if (2 * r->prof_used + 2 > r->prof_ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return false;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return false;
    }
    r->prof_ev.push_back(a);
    r->prof_ev.push_back(b);
  }
  *e0 = r->prof_ev[2 * r->prof_used];
  *e1 = r->prof_ev[2 * r->prof_used + 1];
  ++r->prof_used;
  return true;
}

// ------------------------------------------------------------ autotuning
// The installed entry serving a batch (its bucket ceil(batch / 16)), if any.
static const grom_tuning* tuned(const grom_rom* r, int batch) {
  const size_t b = (size_t)((batch + 15) / 16) - 1;
  return b < r->tuning.size() && r->tuning[b].kernel != GROM_KERNEL_AUTO ? &r->tuning[b] : nullptr;
}

// AUTO's choice of the tensor-core kernel: the tuned entry's, else the rule
// (full form: batches above 8; CP forms: K3T_MIN_BATCH and more).  The
// persistent steppers ask for the rule alone (use_tuning false).
static bool tensor_choice(const grom_rom* r, int batch, bool use_tuning) {
  if (r->kernel_choice == GROM_KERNEL_TENSOR) return true;
  if (r->kernel_choice == GROM_KERNEL_STREAM) return false;
  if (use_tuning)
    if (const grom_tuning* t = tuned(r, batch)) return t->kernel == GROM_KERNEL_TENSOR;
  return r->form == GROM_FORM_FULL ? batch > 8 : batch >= K3T_MIN_BATCH;
}

static bool use_k2(const grom_rom* r, int batch, bool use_tuning = true) {
  if (r->form != GROM_FORM_FULL || r->storage != GROM_BF16 || !r->k2_ok || r->layout != GROM_LAYOUT_DENSE) return false;
  return tensor_choice(r, batch, use_tuning);
}

// K2P: the factored tensor-core kernel of the skew-packed layout
static bool use_k2p(const grom_rom* r, int batch, bool use_tuning = true) {
  if (r->form != GROM_FORM_FULL || r->storage != GROM_BF16 || !r->k2_ok || r->layout != GROM_LAYOUT_SKEW_PACKED)
    return false;
  return tensor_choice(r, batch, use_tuning);
}

static bool is_cp(const grom_rom* r) { return r->form == GROM_FORM_CP || r->form == GROM_FORM_CP_SKEW; }

static bool use_k3g(const grom_rom* r, int batch) {
  return is_cp(r) && batch >= K3G_MIN_BATCH && r->k3g_scratch;
}

// K3D: FP64 CP batches at FP64 tolerance in double-single FP32 arithmetic;
// GROM_KERNEL_STREAM keeps the FP64 GEMMs of K3g
static bool use_k3d(const grom_rom* r, int batch) {
  return is_cp(r) && r->k3d_factors && batch >= K3G_MIN_BATCH && r->kernel_choice != GROM_KERNEL_STREAM;
}

// K3O: FP64 CP batches on the tensor cores (digit slices): GROM_KERNEL_TENSOR,
// else from K3O_MIN_WORK (N R B) on, where it steps faster than K3D
static bool use_k3o(const grom_rom* r, int batch) {
  if (!is_cp(r) || !r->k3o_factors || batch < K3G_MIN_BATCH) return false;
  if (r->kernel_choice == GROM_KERNEL_TENSOR) return true;
  return r->kernel_choice == GROM_KERNEL_AUTO && (int64_t)r->n * r->rank * batch >= K3O_MIN_WORK;
}

// K3T: the batched CP form on the tensor cores (BF16 factors)
static bool use_k3t(const grom_rom* r, int batch, bool use_tuning = true) {
  if (!is_cp(r) || !r->k3t_factors) return false;
  return tensor_choice(r, batch, use_tuning);
}

// The plans with the tuned entry's shape for the batch's bucket.
static K2Plan k2_plan_of(const grom_rom* r, int batch) {
  const grom_tuning* t = tuned(r, batch);
  return k2_plan(r->n, batch, r->sm_count, t ? t->split_a : 0);
}
static K2PPlan k2p_plan_of(const grom_rom* r, int batch) {
  const grom_tuning* t = tuned(r, batch);
  // single CTAs where no cluster of two fits (the rule and a tuning entry alike)
  const int ctas = !r->k2p_pairs ? 1 : t ? t->split_b : 0;
  return k2p_plan(r->n, r->k1.lp, batch, r->sm_count, t ? t->tile_m : 0, ctas);
}
static K3TPlan k3t_plan_of(const grom_rom* r, int batch) {
  const grom_tuning* t = tuned(r, batch);
  return k3t_plan(r->n, r->rank, r->form, batch, r->sm_count, t ? t->split_a : 0, t ? t->split_b : 0);
}

// What the tune space depends on: a ROM's parameters and the scratch it holds.
struct TuneShape {
  int form = 0, storage = 0, layout = 0, max_batch = 1, sm_count = 1;
  int64_t n = 0, rank = 0, lp = 0;
  bool tensor = false;  // a tensor-core kernel exists
  size_t k2_scratch = 0, k3t_scratch = 0;
};

static TuneShape shape_of(const grom_rom* r) {
  TuneShape s;
  s.form = r->form;
  s.storage = r->storage;
  s.layout = r->layout;
  s.max_batch = r->max_batch;
  s.sm_count = r->sm_count;
  s.n = r->n;
  s.rank = r->rank;
  s.lp = r->k1.lp;
  s.tensor = (r->form == GROM_FORM_FULL && r->storage == GROM_BF16 && r->k2_ok) || (is_cp(r) && r->k3t_factors);
  s.k2_scratch = r->k2_scratch_bytes;
  s.k3t_scratch = r->k3t_scratch_bytes;
  return s;
}

static bool shape_is_cp(const TuneShape& s) { return s.form == GROM_FORM_CP || s.form == GROM_FORM_CP_SKEW; }

// Whether an entry is one of the tune space's (timing fields ignored).
static bool tuning_ok(const TuneShape& s, const grom_tuning& t) {
  if (t.batch < 1 || t.batch > s.max_batch) return false;
  if (t.kernel == GROM_KERNEL_STREAM) return t.tile_m == 0 && t.split_a == 0 && t.split_b == 0;
  if (t.kernel != GROM_KERNEL_TENSOR || !s.tensor) return false;
  if (s.form == GROM_FORM_FULL && s.layout == GROM_LAYOUT_DENSE) {
    if (t.tile_m != 0 || t.split_b != 0 || t.split_a < 0 || t.split_a > s.n) return false;
    return k2_scratch_bytes(k2_plan(s.n, t.batch, s.sm_count, t.split_a)) <= s.k2_scratch;
  }
  if (s.form == GROM_FORM_FULL) {
    if (t.split_a != 0 || t.split_b < 0 || t.split_b > 2 || (t.split_b == 2 && !k2p_pair_ok(s.lp))) return false;
    if (t.tile_m != 0 && !k2p_tile_m_ok(t.batch, t.tile_m)) return false;
    return k2p_scratch_bytes(k2p_plan(s.n, s.lp, t.batch, s.sm_count, t.tile_m, t.split_b)) <= s.k2_scratch;
  }
  const K3TPlan p = k3t_plan(s.n, s.rank, s.form, t.batch, s.sm_count, t.split_a, t.split_b);
  if (t.tile_m != 0 || t.split_a < 0 || t.split_a > p.s1_max || t.split_b < 0 || t.split_b > p.s2_max) return false;
  return k3t_scratch_bytes(p) <= s.k3t_scratch;
}

// Split counts to try around the rule's: halvings and doublings of it, and
// every power of two, within [1, hi].
static std::vector<int> split_candidates(int rule, int hi) {
  std::vector<int> v;
  for (int x = rule; x >= 1; x /= 2) v.push_back(x);
  for (int x = 2 * rule; x <= hi && x <= 4 * rule; x *= 2) v.push_back(x);
  for (int x = 1; x <= hi; x *= 2) v.push_back(x);
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  std::vector<int> out;
  for (int x : v)
    if (x >= 1 && x <= hi) out.push_back(x);
  return out;
}

// The rules' configuration first, then the alternatives: the other kernel
// family, and every admissible tile shape of the tensor-core kernel that
// differs from the rule's.
static void tune_space(const TuneShape& s, int batch, std::vector<grom_tuning>& out) {
  out.clear();
  grom_tuning base{};
  base.batch = batch;
  const bool rule_tensor = s.tensor && (s.form == GROM_FORM_FULL ? batch > 8 : batch >= K3T_MIN_BATCH);
  grom_tuning e = base;
  e.kernel = rule_tensor ? GROM_KERNEL_TENSOR : GROM_KERNEL_STREAM;
  out.push_back(e);
  if (!s.tensor) return;
  e = base;
  e.kernel = rule_tensor ? GROM_KERNEL_STREAM : GROM_KERNEL_TENSOR;
  out.push_back(e);  // the other family with its rule shape
  auto add = [&](grom_tuning c) {
    c.batch = batch;
    c.kernel = GROM_KERNEL_TENSOR;
    if (tuning_ok(s, c)) out.push_back(c);
  };
  if (s.form == GROM_FORM_FULL && s.layout == GROM_LAYOUT_DENSE) {
    const int rule = k2_plan(s.n, batch, s.sm_count).splits;
    for (int x : split_candidates(rule, (int)std::min<int64_t>(s.n, 4 * (int64_t)s.sm_count)))
      if (x != rule) {
        grom_tuning c{};
        c.split_a = x;
        add(c);
      }
  } else if (s.form == GROM_FORM_FULL) {
    const K2PPlan rp = k2p_plan(s.n, s.lp, batch, s.sm_count);
    for (int m = 8; m <= 32; ++m)
      if (m != rp.m) {
        grom_tuning c{};
        c.tile_m = m;
        add(c);
      }
    if (k2p_pair_ok(s.lp)) {  // the other kernel (single CTAs or SM pairs) with its rule height
      grom_tuning c{};
      c.split_b = rp.ctas == 2 ? 1 : 2;
      add(c);
    }
  } else if (shape_is_cp(s)) {
    const K3TPlan p = k3t_plan(s.n, s.rank, s.form, batch, s.sm_count);
    for (int a : split_candidates(p.s1, p.s1_max))
      for (int b : split_candidates(p.s2, p.s2_max))
        if (a != p.s1 || b != p.s2) {
          grom_tuning c{};
          c.split_a = a;
          c.split_b = b;
          add(c);
        }
  }
}

static K1Args k1_args(grom_rom* r) {
  K1Args a{};
  a.tensor = r->op;
  a.part = r->part;
  a.err = r->err;
  a.dg = r->k1p_dg;
  a.tg = r->k1p_tg;
  if (r->form == GROM_FORM_SVD) {
    a.mid = r->svd_beta;
    a.mid_stride = r->rank;
  }
  return a;
}

// SVD form: the middle weights beta = sigma o (U^T u) of every trajectory,
// from u (stride u_stride) or from the newest history slot.
static cudaError_t svd_beta(grom_rom* r, int batch, const double* u, int64_t u_stride, const double* hist,
                            const int64_t* taken, const int32_t* active, cudaStream_t s) {
  return svd_project_launch(r->svd_ut, r->svd_sigma, r->n, r->rank, batch, u, u_stride, hist, taken, 6 * (int64_t)r->n,
                            active, r->svd_beta, s);
}

static K3Args k3_args(grom_rom* r) {
  K3Args a{};
  a.fa = r->op;
  a.fb = r->op + r->panel_bytes;
  a.fc = r->op + 2 * r->panel_bytes;
  a.form = r->form;
  a.part = r->part;
  return a;
}

}  // namespace grom

using namespace grom;

extern "C" {

const char* grom_last_error(void) { return g_last_error.c_str(); }

int32_t grom_max_n(int32_t form, int32_t storage) {
  if (storage_elem_bytes(storage) == 0) return 0;
  if (form == GROM_FORM_FULL || form == GROM_FORM_SVD) {
    // a stored row (np elements) must fit one streaming stage
    int64_t n = K1_MAX_ROW_BYTES / storage_elem_bytes(storage);
    return (int32_t)std::min<int64_t>(n, 8192);
  }
  return 1 << 16;
}

grom_status grom_create(const grom_desc* d, void* stream, grom_rom** out) {
  TraceRange trace("grom_create");
  if (!d || !out) return fail(GROM_ERR_INVALID_ARG, "grom_create: null argument");
  *out = nullptr;
  if (d->reserved) return fail(GROM_ERR_INVALID_ARG, "grom_create: reserved fields must be zero");
  if (d->no_tile_copy != 0 && d->no_tile_copy != 1)
    return fail(GROM_ERR_INVALID_ARG, "grom_create: no_tile_copy must be 0 or 1");
  if (d->augmented != 0 && d->augmented != 1) return fail(GROM_ERR_INVALID_ARG, "grom_create: augmented must be 0 or 1");
  if (d->augmented && !((d->form == GROM_FORM_FULL && d->tensor) || d->form == GROM_FORM_CP))
    return fail(GROM_ERR_INVALID_ARG, "grom_create: augmented needs the full form with its tensor, or the general CP form");
  if (d->layout != GROM_LAYOUT_DENSE && d->layout != GROM_LAYOUT_SKEW_PACKED)
    return fail(GROM_ERR_INVALID_ARG, "grom_create: unknown layout");
  if (d->layout != GROM_LAYOUT_DENSE && d->form != GROM_FORM_FULL && d->form != GROM_FORM_SVD)
    return fail(GROM_ERR_INVALID_ARG, "grom_create: the skew-packed layout is for the full and SVD forms");
  if (d->n < 1) return fail(GROM_ERR_INVALID_ARG, "grom_create: n must be >= 1");
  if (d->form < GROM_FORM_FULL || d->form > GROM_FORM_SVD) return fail(GROM_ERR_INVALID_ARG, "grom_create: bad form");
  if (storage_elem_bytes(d->storage) == 0) return fail(GROM_ERR_INVALID_ARG, "grom_create: bad storage type");
  if (d->order < 1 || d->order > 3) return fail(GROM_ERR_INVALID_ARG, "grom_create: order must be 1, 2 or 3");
  if (!(d->dt > 0.0) || !(d->nu >= 0.0) || !std::isfinite(d->dt) || !std::isfinite(d->nu))
    return fail(GROM_ERR_INVALID_ARG, "grom_create: need dt > 0 and nu >= 0");
  if ((d->stiffness == nullptr) == (d->stiffness_diag == nullptr))
    return fail(GROM_ERR_INVALID_ARG, "grom_create: give exactly one of stiffness, stiffness_diag");
  if (d->mass && d->mass_diag) return fail(GROM_ERR_INVALID_ARG, "grom_create: give at most one of mass, mass_diag");
  if (d->linear && d->linear_diag) return fail(GROM_ERR_INVALID_ARG, "grom_create: give at most one of linear, linear_diag");
  if (d->max_batch < 0) return fail(GROM_ERR_INVALID_ARG, "grom_create: max_batch must be >= 0");
  if (d->n > grom_max_n(d->form, d->storage))
    return fail(GROM_ERR_UNSUPPORTED, "grom_create: n exceeds grom_max_n for this form and storage");
  if (d->form == GROM_FORM_FULL) {
    if (!d->tensor && !d->defer_tensor) return fail(GROM_ERR_INVALID_ARG, "grom_create: tensor is NULL");
    if (d->tensor && d->defer_tensor) return fail(GROM_ERR_INVALID_ARG, "grom_create: tensor given with defer_tensor");
  } else if (d->form == GROM_FORM_SVD) {
    if (d->rank < 1) return fail(GROM_ERR_INVALID_ARG, "grom_create: SVD rank must be >= 1");
    if (!d->fa || !d->fb || !d->fc) return fail(GROM_ERR_INVALID_ARG, "grom_create: SVD factors are NULL");
    if (d->defer_tensor) return fail(GROM_ERR_INVALID_ARG, "grom_create: defer_tensor is for the full form");
  } else {
    if (d->rank < 1) return fail(GROM_ERR_INVALID_ARG, "grom_create: CP rank must be >= 1");
    if (!d->fa || !d->fb || !d->fc) return fail(GROM_ERR_INVALID_ARG, "grom_create: CP factors are NULL");
    if (d->storage == GROM_F32X2) return fail(GROM_ERR_UNSUPPORTED, "grom_create: F32X2 storage is for the full form");
    if (d->defer_tensor) return fail(GROM_ERR_INVALID_ARG, "grom_create: defer_tensor is for the full form");
  }

  grom_rom* r = new (std::nothrow) grom_rom();
  if (!r) return fail(GROM_ERR_OOM, "grom_create: host allocation");
  r->n = d->n;
  r->form = d->form;
  r->rank = d->rank;
  r->storage = d->storage;
  r->order = d->order;
  r->nu = d->nu;
  r->dt = d->dt;
  r->max_batch = d->max_batch > 0 ? d->max_batch : 1;
  r->layout = d->layout;
  r->no_tile_copy = d->no_tile_copy != 0;
  r->stream = static_cast<cudaStream_t>(stream);
  const int64_t n = r->n;
  grom_status st = GROM_OK;
  std::vector<double> Laug, faug;  // zeroth-mode terms of an augmented operator
  auto bail = [&](grom_status s) {
    cudaStreamSynchronize(r->stream);
    rom_free(r);
    return s;
  };
  if (cudaGetDevice(&r->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, r->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(GROM_ERR_CUDA, "grom_create: no usable CUDA device"));
  }

  // ---------------------------------------------------- advection operator
  if (r->form == GROM_FORM_FULL) {
    r->np = padded_n(n);
    const bool packed = r->layout == GROM_LAYOUT_SKEW_PACKED;
    r->k1 = k1_plan(n, r->storage, r->sm_count, packed ? 1 : 0);
    const size_t row_bytes = (size_t)r->k1.row_bytes;
    r->op_bytes = (size_t)n * (size_t)n * row_bytes;
    if ((st = dmalloc(&r->op, r->op_bytes, &r->total_bytes))) return bail(st);
    r->part_bytes = (size_t)r->k1.grid * r->k1.maxseg * (K1_CONSUMERS / 32) * r->k1.nb_max * sizeof(double);
    if ((st = dmalloc(&r->part, r->part_bytes, &r->total_bytes))) return bail(st);
    if (packed) {
      if ((st = dmalloc(&r->k1p_dg, k1p_dg_bytes(r->k1, r->storage), &r->total_bytes))) return bail(st);
      if ((st = dmalloc(&r->k1p_tg, k1p_tg_bytes(r->k1), &r->total_bytes))) return bail(st);
      if ((st = dmalloc(&r->probe, 3 * sizeof(double), &r->total_bytes))) return bail(st);
      if ((st = dmalloc(&r->k1pp_scratch, k1pp_scratch_bytes(r->k1), &r->total_bytes))) return bail(st);
      if (cudaMemsetAsync(r->probe, 0, 3 * sizeof(double), r->stream) != cudaSuccess ||
          cudaMemsetAsync(r->k1pp_scratch, 0, k1pp_scratch_bytes(r->k1), r->stream) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "grom_create"));
    }
    if (r->storage == GROM_BF16 && packed) {
      r->k2_ok = k2p_make_tmap(&r->k2_tmap, r->op, n, r->k1.lp);
      r->k2p_pairs = r->k2_ok && k2p_pairs_supported();
      if (r->k2_ok) {
        // scratch for the largest plan over the batch sizes this ROM accepts
        const size_t need = k2p_scratch_need(n, r->k1.lp, r->max_batch, r->sm_count);
        r->k2_scratch_bytes = need;
        if ((st = dmalloc(&r->k2_scratch, need, &r->total_bytes))) return bail(st);
      }
    }
    if (r->storage == GROM_BF16 && !packed) {
      r->k2_ok = k2_make_tmap(&r->k2_tmap, r->op, n, r->np);
      if (r->k2_ok) {
        // scratch for the largest plan over the batch sizes this ROM accepts
        const size_t need = k2_scratch_need(n, r->max_batch, r->sm_count);
        r->k2_scratch_bytes = need;
        if ((st = dmalloc(&r->k2_scratch, need, &r->total_bytes))) return bail(st);
      }
    }
    if (d->tensor && d->augmented) {
      if ((st = upload_augmented_full(r, d->tensor, Laug, faug))) return bail(st);
      r->rows_uploaded = n;
      if (r->max_batch > 8 && (st = build_k2_tiles(r))) return bail(st);
    } else if (d->tensor) {
      if (packed) {
        if ((st = upload_rows_packed(r, d->tensor, 0, n))) return bail(st);
        if ((st = check_skew_probe(r))) return bail(st);
      } else if ((st = upload_rows(r, d->tensor, n * n, n, r->np, r->op, (int64_t)row_bytes))) {
        return bail(st);
      }
      r->rows_uploaded = n;
      if (r->max_batch > 8 && (st = build_k2_tiles(r))) return bail(st);
    } else {
      r->row_seen = new (std::nothrow) uint8_t[(size_t)n]();
      if (!r->row_seen) return bail(fail(GROM_ERR_OOM, "grom_create: host allocation"));
    }
  } else if (r->form == GROM_FORM_SVD) {
    // V slices V[i][r][k] as n * rank streamed rows; U^T and sigma in FP64
    const bool packed = r->layout == GROM_LAYOUT_SKEW_PACKED;
    const int64_t R = r->rank;
    r->np = padded_n(n);
    r->k1 = k1_plan(n, r->storage, r->sm_count, packed ? 1 : 0, R);
    const size_t row_bytes = (size_t)r->k1.row_bytes;
    r->op_bytes = (size_t)n * (size_t)R * row_bytes;
    if ((st = dmalloc(&r->op, r->op_bytes, &r->total_bytes))) return bail(st);
    r->part_bytes = (size_t)r->k1.grid * r->k1.maxseg * (K1_CONSUMERS / 32) * r->k1.nb_max * sizeof(double);
    if ((st = dmalloc(&r->part, r->part_bytes, &r->total_bytes))) return bail(st);
    if (packed) {
      if ((st = dmalloc(&r->k1p_dg, k1p_dg_bytes(r->k1, r->storage), &r->total_bytes))) return bail(st);
      if ((st = dmalloc(&r->k1p_tg, k1p_tg_bytes(r->k1), &r->total_bytes))) return bail(st);
      if ((st = dmalloc(&r->probe, 3 * sizeof(double), &r->total_bytes))) return bail(st);
      if (cudaMemsetAsync(r->probe, 0, 3 * sizeof(double), r->stream) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "grom_create"));
      if ((st = upload_rows_packed(r, d->fc, 0, n))) return bail(st);
      if ((st = check_skew_probe(r))) return bail(st);
    } else if ((st = upload_rows(r, d->fc, n * R, n, r->np, r->op, (int64_t)row_bytes))) {
      return bail(st);
    }
    std::vector<double> U, sig, ut((size_t)(R * n));
    if ((st = fetch(U, d->fa, (size_t)(n * R)))) return bail(st);
    if ((st = fetch(sig, d->fb, (size_t)R))) return bail(st);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t q = 0; q < R; ++q) ut[q * n + j] = U[j * R + q];
    if ((st = upload(&r->svd_ut, ut.data(), ut.size(), &r->total_bytes, r->stream))) return bail(st);
    if ((st = upload(&r->svd_sigma, sig.data(), sig.size(), &r->total_bytes, r->stream))) return bail(st);
    if ((st = dmalloc(&r->svd_beta, (size_t)r->max_batch * R * sizeof(double), &r->total_bytes))) return bail(st);
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "grom_create"));
    r->rows_uploaded = n;
  } else {
    r->k3 = k3_plan(n, r->rank, r->storage, r->sm_count);
    const int64_t rp = r->k3.rb;
    r->panel_bytes = (size_t)n * rp * storage_elem_bytes(r->storage);
    r->panel_bytes = (r->panel_bytes + 255) / 256 * 256;
    r->op_bytes = 3 * r->panel_bytes;
    if ((st = dmalloc(&r->op, r->op_bytes, &r->total_bytes))) return bail(st);
    // augmented factors: rows 1..n of fb and fc are the core factors
    const int64_t off = d->augmented ? r->rank : 0;
    const double* f[3] = {d->fa, d->fb + off, d->fc + off};
    for (int q = 0; q < 3; ++q)
      if ((st = upload_rows(r, f[q], n, r->rank, rp, r->op + q * r->panel_bytes, rp * storage_elem_bytes(r->storage))))
        return bail(st);
    r->part_bytes = k3_scratch_bytes(r->k3, r->storage);
    if ((st = dmalloc(&r->part, r->part_bytes, &r->total_bytes))) return bail(st);
    if (r->max_batch >= K3G_MIN_BATCH &&
        (st = dmalloc(&r->k3g_scratch, k3g_scratch_bytes(n, rp, r->max_batch, r->storage, r->sm_count),
                      &r->total_bytes)))
      return bail(st);
    if (r->k3g_scratch && cudaMemsetAsync(r->k3g_scratch, 0,
                                          k3g_scratch_bytes(n, rp, r->max_batch, r->storage, r->sm_count),
                                          r->stream) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "grom_create"));
    if (r->storage == GROM_F64 && r->max_batch >= K3G_MIN_BATCH) {
      // hi/lo FP32 copies of the factors for the double-single GEMMs (K3D)
      if ((st = dmalloc(&r->k3d_factors, k3d_factor_bytes(n, rp), &r->total_bytes))) return bail(st);
      const size_t kd = k3d_scratch_bytes(n, rp, r->max_batch, r->sm_count);
      if ((st = dmalloc(&r->k3d_scratch, kd, &r->total_bytes))) return bail(st);
      if (cudaMemsetAsync(r->k3d_scratch, 0, kd, r->stream) != cudaSuccess ||
          k3d_build_factors(r->op, r->panel_bytes, n, rp, r->k3d_factors, r->stream) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "grom_create: double-single factor copies"));
      if (k3o_supported(n, r->rank, r->form)) {
        // digit slices of the factors for the tensor-core path (K3O)
        if ((st = dmalloc(&r->k3o_factors, k3o_factor_bytes(n, rp, r->rank, r->form), &r->total_bytes)))
          return bail(st);
        if ((st = dmalloc(&r->k3o_scratch, k3o_scratch_bytes(n, rp, r->rank, r->form, r->max_batch),
                          &r->total_bytes)))
          return bail(st);
        if (k3o_build_factors(r->op, r->panel_bytes, n, rp, r->rank, r->form, r->k3o_factors, r->stream) !=
            cudaSuccess)
          return bail(cuda_fail(cudaGetLastError(), "grom_create: factor digit slices"));
      }
    }
    if (r->storage == GROM_BF16) {
      // the factors again, laid out for the tensor-core GEMMs (K3T), and the
      // scratch of the largest plan over the batch sizes this ROM accepts
      if ((st = dmalloc(&r->k3t_factors, k3t_factor_bytes(n, r->rank, r->form), &r->total_bytes))) return bail(st);
      uint8_t* ft = static_cast<uint8_t*>(r->k3t_factors);
      const K3TPlan p0 = k3t_plan(n, r->rank, r->form, 16, r->sm_count);
      uint8_t* ae = ft + (size_t)p0.m1 * p0.np * 2;
      if (k3t_build_factors(r->op, r->op + r->panel_bytes, r->op + 2 * r->panel_bytes, n, rp, r->rank, r->form, ft,
                            ae, r->stream) != cudaSuccess ||
          !k3t_make_tmaps(&r->k3t_tmap_ft, &r->k3t_tmap_ae, ft, ae, n, r->rank, r->form))
        return bail(cuda_fail(cudaGetLastError(), "grom_create: tensor-core factor copies"));
      r->k3t_scratch_bytes = k3t_scratch_need(n, r->rank, r->form, r->max_batch, r->sm_count);
      if ((st = dmalloc(&r->k3t_scratch, r->k3t_scratch_bytes, &r->total_bytes))) return bail(st);
      // the projection tiles' arrival counters start at zero
      if (cudaMemsetAsync(r->k3t_scratch, 0, k3t_counter_bytes(p0), r->stream) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "grom_create"));
    }
    // persistent stepper (its grid-barrier word starts at zero)
    const size_t kp = k3p_scratch_bytes(n, rp, r->storage, r->sm_count);
    if ((st = dmalloc(&r->k3p_scratch, kp, &r->total_bytes))) return bail(st);
    if (cudaMemsetAsync(r->k3p_scratch, 0, kp, r->stream) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "grom_create"));
    // the per-tile arrival counters of the projection kernel start at zero
    if (cudaMemsetAsync(r->part, 0, r->part_bytes, r->stream) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "grom_create"));
  }

  if (d->augmented && r->form == GROM_FORM_CP) {
    // zeroth-mode terms of the CP model: X_i0k = sum_m A_im b0_m C_km,
    // X_ij0 = sum_m A_im B_jm c0_m, X_i00 = sum_m A_im b0_m c0_m
    const int64_t R = r->rank;
    std::vector<double> Af, Bf, Cf;
    if ((st = fetch(Af, d->fa, (size_t)(n * R)))) return bail(st);
    if ((st = fetch(Bf, d->fb, (size_t)((n + 1) * R)))) return bail(st);
    if ((st = fetch(Cf, d->fc, (size_t)((n + 1) * R)))) return bail(st);
    Laug.assign((size_t)(n * n), 0.0);
    faug.assign((size_t)n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
      const double* Ai = Af.data() + i * R;
      for (int64_t m = 0; m < R; ++m) faug[i] += Ai[m] * Bf[m] * Cf[m];
      for (int64_t k = 0; k < n; ++k) {
        const double* Bk = Bf.data() + (k + 1) * R;
        const double* Ck = Cf.data() + (k + 1) * R;
        double s = 0.0;
        for (int64_t m = 0; m < R; ++m) s += Ai[m] * (Bf[m] * Ck[m] + Cf[m] * Bk[m]);
        Laug[i * n + k] = s;
      }
    }
  }

  // ------------------------------------------------------ linear operators
  std::vector<double> A, Bm, mdiag, adiag;
  const bool a_dense = d->stiffness != nullptr;
  const bool b_dense = d->mass != nullptr;
  if (a_dense) {
    if ((st = fetch(A, d->stiffness, (size_t)(n * n)))) return bail(st);
  } else if ((st = fetch(adiag, d->stiffness_diag, (size_t)n))) {
    return bail(st);
  }
  if (b_dense) {
    if ((st = fetch(Bm, d->mass, (size_t)(n * n)))) return bail(st);
  } else if (d->mass_diag) {
    if ((st = fetch(mdiag, d->mass_diag, (size_t)n))) return bail(st);
  } else {
    mdiag.assign((size_t)n, 1.0);
  }
  const bool aug = d->augmented != 0;
  r->diagonal = !a_dense && !b_dense && !d->linear && !aug;
  const bool h_diag = !a_dense && !b_dense;
  if (h_diag) {
    std::vector<double> hd((size_t)(3 * n));
    for (int k = 0; k < 3; ++k)
      for (int64_t i = 0; i < n; ++i) {
        const double h = kBeta0[k] / r->dt * mdiag[i] + r->nu * adiag[i];
        if (!(h > 0.0) || !std::isfinite(h)) return bail(fail(GROM_ERR_INVALID_ARG, "grom_create: H_k is not positive"));
        hd[k * n + i] = 1.0 / h;
      }
    if ((st = upload(&r->hdiag, hd.data(), hd.size(), &r->total_bytes, r->stream))) return bail(st);
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "upload"));
  } else {
    std::vector<double> H((size_t)(n * n)), Hinv, all((size_t)(3 * n * n));
    for (int k = 0; k < r->order; ++k) {
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
          const double b = b_dense ? Bm[i * n + j] : (i == j ? mdiag[i] : 0.0);
          const double a = a_dense ? A[i * n + j] : (i == j ? adiag[i] : 0.0);
          H[i * n + j] = kBeta0[k] / r->dt * b + r->nu * a;
        }
      if (!spd_inverse(n, H, Hinv)) return bail(fail(GROM_ERR_INVALID_ARG, "grom_create: H_k is not SPD"));
      std::memcpy(all.data() + k * n * n, Hinv.data(), (size_t)(n * n) * sizeof(double));
    }
    if ((st = upload(&r->hinv, all.data(), all.size(), &r->total_bytes, r->stream))) return bail(st);
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "upload"));
  }
  if (b_dense) {
    if ((st = upload(&r->mass, Bm.data(), Bm.size(), &r->total_bytes, r->stream))) return bail(st);
  } else if (d->mass_diag) {
    if ((st = upload(&r->mass_diag, mdiag.data(), mdiag.size(), &r->total_bytes, r->stream))) return bail(st);
  }
  if (aug) {
    // the caller's L and f plus the zeroth-mode terms, as a dense L
    std::vector<double> Lh, fh, tmp;
    if (d->linear) {
      if ((st = fetch(Lh, d->linear, (size_t)(n * n)))) return bail(st);
    } else {
      Lh.assign((size_t)(n * n), 0.0);
      if (d->linear_diag) {
        if ((st = fetch(tmp, d->linear_diag, (size_t)n))) return bail(st);
        for (int64_t i = 0; i < n; ++i) Lh[i * n + i] = tmp[i];
      }
    }
    if (d->forcing) {
      if ((st = fetch(fh, d->forcing, (size_t)n))) return bail(st);
    } else {
      fh.assign((size_t)n, 0.0);
    }
    for (size_t q = 0; q < Lh.size(); ++q) Lh[q] += Laug[q];
    for (size_t q = 0; q < fh.size(); ++q) fh[q] += faug[q];
    if ((st = upload(&r->linear, Lh.data(), Lh.size(), &r->total_bytes, r->stream))) return bail(st);
    if ((st = upload(&r->forcing, fh.data(), fh.size(), &r->total_bytes, r->stream))) return bail(st);
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "upload"));
  } else {
    if (d->linear && (st = upload(&r->linear, d->linear, (size_t)(n * n), &r->total_bytes, r->stream))) return bail(st);
    if (d->linear_diag && (st = upload(&r->lin_diag, d->linear_diag, (size_t)n, &r->total_bytes, r->stream)))
      return bail(st);
    if (d->forcing && (st = upload(&r->forcing, d->forcing, (size_t)n, &r->total_bytes, r->stream))) return bail(st);
  }
  if ((st = dmalloc(&r->err, 2 * sizeof(int), &r->total_bytes))) return bail(st);
  if (cudaMemsetAsync(r->err, 0, 2 * sizeof(int), r->stream) != cudaSuccess ||
      cudaStreamSynchronize(r->stream) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "grom_create"));
  *out = r;
  return GROM_OK;
}

grom_status grom_upload_tensor_slab(grom_rom* r, int32_t i0, int32_t i1, const double* rows) {
  if (!r || !rows) return fail(GROM_ERR_INVALID_ARG, "grom_upload_tensor_slab: null argument");
  if (r->form != GROM_FORM_FULL || !r->row_seen)
    return fail(GROM_ERR_INVALID_ARG, "grom_upload_tensor_slab: ROM was not created with defer_tensor");
  if (i0 < 0 || i1 > r->n || i0 >= i1) return fail(GROM_ERR_INVALID_ARG, "grom_upload_tensor_slab: bad row range");
  const int64_t n = r->n;
  const bool packed = r->layout == GROM_LAYOUT_SKEW_PACKED;
  if (packed) {
    // the probe adds every row once
    for (int64_t i = i0; i < i1; ++i)
      if (r->row_seen[i]) return fail(GROM_ERR_INVALID_ARG, "grom_upload_tensor_slab: rows already uploaded (packed layout)");
  }
  grom_status st = packed ? upload_rows_packed(r, rows, i0, i1)
                          : upload_rows(r, rows, (int64_t)(i1 - i0) * n, n, r->np,
                                        r->op + (size_t)i0 * n * (size_t)r->k1.row_bytes, r->k1.row_bytes);
  if (st) return st;
  for (int64_t i = i0; i < i1; ++i)
    if (!r->row_seen[i]) {
      r->row_seen[i] = 1;
      ++r->rows_uploaded;
    }
  if (packed && r->rows_uploaded == n && (st = check_skew_probe(r))) {
    r->rows_uploaded = n - 1;  // the ROM stays unusable
    return st;
  }
  if (r->rows_uploaded == n && r->max_batch > 8 && (st = build_k2_tiles(r))) return st;
  return GROM_OK;
}

grom_status grom_destroy(grom_rom* r) {
  if (!r) return GROM_OK;
  if (r->traj_count > 0) return fail(GROM_ERR_INVALID_ARG, "grom_destroy: trajectories still exist");
  cudaStreamSynchronize(r->stream);
  rom_free(r);
  return GROM_OK;
}

grom_status grom_sync(grom_rom* r) {
  if (!r) return fail(GROM_ERR_INVALID_ARG, "grom_sync: null rom");
  GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
  int flags[2] = {0, 0};
  GROM_CUDA_TRY(cudaMemcpy(flags, r->err, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags[0] & DEV_ERR_TIMEOUT) {
    // reported once; the ROM stays usable
    GROM_CUDA_TRY(cudaMemset(r->err, 0, sizeof(int)));
    return fail(GROM_ERR_TIMEOUT, "a device-side wait timed out");
  }
  return GROM_OK;
}

grom_status grom_selftest_timeout(grom_rom* r, int64_t limit_ns) {
  if (!r || limit_ns < 0) return fail(GROM_ERR_INVALID_ARG, "grom_selftest_timeout: bad argument");
  GROM_CUDA_TRY(selftest_wait_launch(r->err, (uint64_t)limit_ns, r->stream));
  return GROM_OK;
}

int64_t grom_rom_bytes(const grom_rom* r) { return r ? (int64_t)r->total_bytes : 0; }

grom_status grom_nonlinear(grom_rom* r, int32_t batch, const double* u, double* c) {
  TraceRange trace("grom_nonlinear");
  if (!r || !u || !c) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear: null argument");
  if (batch < 1 || batch > r->max_batch) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear: batch out of range");
  if (!full_ready(r)) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear: tensor rows missing");
  cudaError_t e;
  if (use_k2(r, batch)) {
    K2Args a{};
    a.u = u;
    a.u_stride = r->n;
    a.c = c;
    a.c_stride = r->n;
    a.batch = batch;
    a.scratch = r->k2_scratch;
    a.err = r->err;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return fail(GROM_ERR_CUDA, "event creation failed");
    a.tiled = r->k2_tiles != nullptr;
    e = k2_launch(k2_plan_of(r, batch), a.tiled ? &r->k2_tmap_tiled : &r->k2_tmap, a, r->stream);
  } else if (use_k2p(r, batch)) {
    K2Args a{};
    a.u = u;
    a.u_stride = r->n;
    a.c = c;
    a.c_stride = r->n;
    a.batch = batch;
    a.scratch = r->k2_scratch;
    a.err = r->err;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return fail(GROM_ERR_CUDA, "event creation failed");
    e = k2p_launch(k2p_plan_of(r, batch), &r->k2_tmap, a, r->stream);
  } else if (!is_cp(r)) {
    K1Args a = k1_args(r);
    a.u = u;
    a.u_stride = r->n;
    a.c = c;
    a.c_stride = r->n;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return fail(GROM_ERR_CUDA, "event creation failed");
    e = r->form == GROM_FORM_SVD ? svd_beta(r, batch, u, r->n, nullptr, nullptr, nullptr, r->stream) : cudaSuccess;
    if (e == cudaSuccess) e = k1_launch(r->k1, r->storage, a, batch, r->stream);
  } else {
    K3Args a = k3_args(r);
    a.u = u;
    a.u_stride = r->n;
    a.c = c;
    a.c_stride = r->n;
    cudaEvent_t e0, e1;
    if (!prof_pair(r, &e0, &e1)) return fail(GROM_ERR_CUDA, "event creation failed");
    if (e0) prof_record(e0, r->stream);
    e = use_k3t(r, batch) ? k3t_launch(k3t_plan_of(r, batch), &r->k3t_tmap_ft,
                                       &r->k3t_tmap_ae, a, batch, r->k3t_scratch, r->err, r->stream)
        : use_k3o(r, batch) ? k3o_launch(r->n, r->k3.rb, r->rank, a, r->k3o_factors, batch, r->k3o_scratch, r->err,
                                         r->sm_count, r->stream)
        : use_k3d(r, batch) ? k3d_launch(r->k3, a, r->k3d_factors, batch, r->max_batch, r->k3d_scratch, r->sm_count,
                                         r->stream)
        : use_k3g(r, batch) ? k3g_launch(r->k3, r->storage, a, batch, r->max_batch, r->k3g_scratch, r->sm_count, r->stream)
                            : k3_launch(r->k3, r->storage, a, batch, r->stream);
    if (e1) prof_record(e1, r->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "grom_nonlinear launch");
  return GROM_OK;
}

grom_status grom_traj_create(grom_rom* r, int32_t batch, const double* u0, grom_traj** out) {
  TraceRange trace("grom_traj_create");
  if (!r || !u0 || !out) return fail(GROM_ERR_INVALID_ARG, "grom_traj_create: null argument");
  *out = nullptr;
  if (batch < 1 || batch > r->max_batch) return fail(GROM_ERR_INVALID_ARG, "grom_traj_create: batch out of range");
  grom_traj* t = new (std::nothrow) grom_traj();
  if (!t) return fail(GROM_ERR_OOM, "grom_traj_create: host allocation");
  t->rom = r;
  t->batch = batch;
  const int64_t n = r->n;
  auto bail = [&](grom_status s) {
    cudaStreamSynchronize(r->stream);
    if (t->hist) cudaFree(t->hist);
    if (t->taken) cudaFree(t->taken);
    if (t->work) cudaFree(t->work);
    if (t->err) cudaFree(t->err);
    if (t->io) cudaFree(t->io);
    if (t->red) cudaFree(t->red);
    if (t->cnt) cudaFree(t->cnt);
    delete t;
    return s;
  };
  grom_status st;
  if ((st = dmalloc(&t->hist, (size_t)batch * 6 * n * sizeof(double), nullptr))) return bail(st);
  if ((st = dmalloc(&t->taken, (size_t)batch * sizeof(int64_t), nullptr))) return bail(st);
  if ((st = dmalloc(&t->err, 2 * sizeof(int), nullptr))) return bail(st);
  if ((st = dmalloc(&t->io, (size_t)batch * n * sizeof(double), nullptr))) return bail(st);
  if (r->diagonal) {
    const int nblk = std::max(std::max(step_mc_blocks(n), k3_expand_blocks(n)), step_pk_blocks(n));
    if ((st = dmalloc(&t->red, (size_t)batch * nblk * 2 * sizeof(double), nullptr))) return bail(st);
    if ((st = dmalloc(&t->cnt, (size_t)batch * sizeof(unsigned int), nullptr))) return bail(st);
    if (cudaMemsetAsync(t->cnt, 0, (size_t)batch * sizeof(unsigned int), r->stream) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "grom_traj_create"));
  }
  if (!r->diagonal && (st = dmalloc(&t->work, (size_t)batch * 4 * n * sizeof(double), nullptr))) return bail(st);
  const int init[2] = {0, INT_MAX};
  if (cudaMemsetAsync(t->hist, 0, (size_t)batch * 6 * n * sizeof(double), r->stream) != cudaSuccess ||
      cudaMemsetAsync(t->taken, 0, (size_t)batch * sizeof(int64_t), r->stream) != cudaSuccess ||
      cudaMemcpyAsync(t->err, init, sizeof(init), cudaMemcpyHostToDevice, r->stream) != cudaSuccess ||
      cudaMemcpy2DAsync(t->hist, (size_t)6 * n * sizeof(double), u0, (size_t)n * sizeof(double),
                        (size_t)n * sizeof(double), (size_t)batch, cudaMemcpyDefault, r->stream) != cudaSuccess ||
      cudaStreamSynchronize(r->stream) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "grom_traj_create"));
  ++r->traj_count;
  *out = t;
  return GROM_OK;
}

grom_status grom_traj_destroy(grom_traj* t) {
  if (!t) return GROM_OK;
  cudaStreamSynchronize(t->rom->stream);
  cudaFree(t->hist);
  cudaFree(t->taken);
  if (t->work) cudaFree(t->work);
  cudaFree(t->err);
  cudaFree(t->io);
  if (t->red) cudaFree(t->red);
  if (t->cnt) cudaFree(t->cnt);
  if (t->graph) cudaGraphExecDestroy(t->graph);
  if (t->graph_tmpl) cudaGraphDestroy(t->graph_tmpl);
  if (t->io_graph) cudaGraphExecDestroy(t->io_graph);
  if (t->gstream) cudaStreamDestroy(t->gstream);
  if (t->ev_in) cudaEventDestroy(t->ev_in);
  if (t->ev_out) cudaEventDestroy(t->ev_out);
  if (t->active) cudaFree(t->active);
  if (t->steps_left) cudaFree(t->steps_left);
  --t->rom->traj_count;
  delete t;
  return GROM_OK;
}

static cudaError_t traj_nonlinear(grom_traj* t, cudaStream_t strm) {
  grom_rom* r = t->rom;
  if (use_k2(r, t->batch)) {
    K2Args a{};
    a.hist = t->hist;
    a.taken = t->taken;
    a.hist_stride = 6 * (int64_t)r->n;
    a.active = t->active;
    a.batch = t->batch;
    a.scratch = r->k2_scratch;
    a.err = r->err;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return cudaErrorMemoryAllocation;
    a.tiled = r->k2_tiles != nullptr;
    return k2_launch(k2_plan_of(r, t->batch), a.tiled ? &r->k2_tmap_tiled : &r->k2_tmap, a, strm);
  }
  if (use_k2p(r, t->batch)) {
    K2Args a{};
    a.hist = t->hist;
    a.taken = t->taken;
    a.hist_stride = 6 * (int64_t)r->n;
    a.active = t->active;
    a.batch = t->batch;
    a.scratch = r->k2_scratch;
    a.err = r->err;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return cudaErrorMemoryAllocation;
    return k2p_launch(k2p_plan_of(r, t->batch), &r->k2_tmap, a, strm);
  }
  if (!is_cp(r)) {
    K1Args a = k1_args(r);
    a.hist = t->hist;
    a.taken = t->taken;
    a.hist_stride = 6 * (int64_t)r->n;
    a.active = t->active;
    if (!prof_pair(r, &a.ev0, &a.ev1)) return cudaErrorMemoryAllocation;
    if (r->form == GROM_FORM_SVD) {
      const cudaError_t e = svd_beta(r, t->batch, nullptr, 0, t->hist, t->taken, t->active, strm);
      if (e != cudaSuccess) return e;
    }
    return k1_launch(r->k1, r->storage, a, t->batch, strm);
  }
  K3Args a = k3_args(r);
  a.hist = t->hist;
  a.taken = t->taken;
  a.hist_stride = 6 * (int64_t)r->n;
  a.active = t->active;
  cudaEvent_t e0, e1;
  if (!prof_pair(r, &e0, &e1)) return cudaErrorMemoryAllocation;
  if (e0) prof_record(e0, strm);
  cudaError_t e = use_k3t(r, t->batch)
                      ? k3t_launch(k3t_plan_of(r, t->batch), &r->k3t_tmap_ft,
                                   &r->k3t_tmap_ae, a, t->batch, r->k3t_scratch, r->err, strm)
                  : use_k3o(r, t->batch)
                      ? k3o_launch(r->n, r->k3.rb, r->rank, a, r->k3o_factors, t->batch, r->k3o_scratch, r->err,
                                   r->sm_count, strm)
                  : use_k3d(r, t->batch)
                      ? k3d_launch(r->k3, a, r->k3d_factors, t->batch, r->max_batch, r->k3d_scratch, r->sm_count, strm)
                  : use_k3g(r, t->batch)
                      ? k3g_launch(r->k3, r->storage, a, t->batch, r->max_batch, r->k3g_scratch, r->sm_count, strm)
                      : k3_launch(r->k3, r->storage, a, t->batch, strm);
  if (e1 && e == cudaSuccess) e = prof_record(e1, strm);
  return e;
}

static StepArgs step_args(grom_traj* t, double* energy, double* invariant) {
  grom_rom* r = t->rom;
  StepArgs a{};
  a.n = r->n;
  a.batch = t->batch;
  a.order = r->order;
  a.dt = r->dt;
  a.inv_dt = 1.0 / r->dt;
  // beta_1 .. beta_k of BDFk over dt (the same products the device forms)
  static const double kBetaQ[3][3] = {{-1.0, 0.0, 0.0}, {-2.0, 0.5, 0.0}, {-3.0, 1.5, -1.0 / 3.0}};
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q) a.bdt[k][q] = kBetaQ[k][q] * a.inv_dt;
  a.nu = r->nu;
  a.hist = t->hist;
  a.hist_stride = 6 * (int64_t)r->n;
  a.taken = t->taken;
  for (int k = 0; k < 3; ++k) {
    a.hdiag[k] = r->hdiag ? r->hdiag + k * r->n : nullptr;
    a.hinv[k] = r->hinv ? r->hinv + (size_t)std::min(k, r->order - 1) * r->n * r->n : nullptr;
  }
  a.mass_diag = r->mass_diag;
  a.lin_diag = r->lin_diag;
  a.forcing = r->forcing;
  a.mass = r->mass;
  a.linear = r->linear;
  a.work = t->work;
  a.energy = energy;
  a.invariant = invariant;
  a.err = t->err;
  a.first_bad = t->err + 1;
  a.red = t->red;
  a.cnt = t->cnt;
  // large batches with the energy or invariant asked for: four elements per
  // thread, so the per-block FP64 reduction is paid once per four elements;
  // otherwise one (more, shorter blocks)
  a.ept = t->batch >= 64 && (energy || invariant) ? 4 : 1;
  a.nblk = (int)((r->n + (int64_t)STEP_MC_THREADS * a.ept - 1) / ((int64_t)STEP_MC_THREADS * a.ept));
  a.active = t->active;
  a.active_rw = t->active;
  a.steps_left = t->steps_left;
  return a;
}

// Enqueues `count` steps (per-step outputs at step_index offset) on strm.
static cudaError_t launch_steps(grom_traj* t, int count, double* energy, double* invariant, cudaStream_t strm) {
  grom_rom* r = t->rom;
  StepArgs a = step_args(t, energy, invariant);
  const bool fused_k1 = r->diagonal && !is_cp(r) && !use_k2(r, t->batch) && !use_k2p(r, t->batch);
  const bool fused_k3 = r->diagonal && is_cp(r) && !use_k3g(r, t->batch) && !use_k3t(r, t->batch);
  const bool fused_k3t = r->diagonal && use_k3t(r, t->batch);
  const bool fused_k3d = r->diagonal && use_k3d(r, t->batch) && !use_k3o(r, t->batch);
  const bool fused_k3o = r->diagonal && !use_k3t(r, t->batch) && use_k3o(r, t->batch);
  for (int s = 0; s < count; ++s) {
    cudaError_t e;
    if (fused_k3o) {
      // the expansion's combine and the step in one kernel
      K3Args k = k3_args(r);
      k.hist = t->hist;
      k.taken = t->taken;
      k.hist_stride = 6 * (int64_t)r->n;
      k.active = t->active;
      cudaEvent_t e0, e1;
      if (!prof_pair(r, &e0, &e1)) return cudaErrorMemoryAllocation;
      if (e0) prof_record(e0, strm);
      e = k3o_launch_step(r->n, r->k3.rb, r->rank, k, r->k3o_factors, t->batch, r->k3o_scratch, r->err,
                          r->sm_count, a, s, strm);
      if (e1 && e == cudaSuccess) e = prof_record(e1, strm);
    } else if (fused_k3d) {
      // as K3T: the state planes once per call, then the ones the step kernel writes
      K3Args k = k3_args(r);
      k.hist = t->hist;
      k.taken = t->taken;
      k.hist_stride = 6 * (int64_t)r->n;
      k.active = t->active;
      cudaEvent_t e0, e1;
      if (!prof_pair(r, &e0, &e1)) return cudaErrorMemoryAllocation;
      e = k3d_launch_step(r->k3, k, r->k3d_factors, t->batch, r->k3d_scratch, r->sm_count, s == 0, a, s, e0, e1,
                          strm);
    } else if (fused_k3t) {
      // the state prep once per call; later steps reuse the rows the step kernel writes
      K3Args k = k3_args(r);
      k.hist = t->hist;
      k.taken = t->taken;
      k.hist_stride = 6 * (int64_t)r->n;
      k.active = t->active;
      cudaEvent_t e0, e1;
      if (!prof_pair(r, &e0, &e1)) return cudaErrorMemoryAllocation;
      e = k3t_launch_step(k3t_plan_of(r, t->batch), &r->k3t_tmap_ft, &r->k3t_tmap_ae, k, t->batch, r->k3t_scratch,
                          r->err, s == 0, a, s, e0, e1, strm);
    } else if (fused_k3) {
      K3Args k = k3_args(r);
      k.hist = t->hist;
      k.taken = t->taken;
      k.hist_stride = 6 * (int64_t)r->n;
      k.active = t->active;
      StepArgs st3 = a;
      st3.nblk = k3_expand_blocks(r->n);
      cudaEvent_t e0, e1;
      if (!prof_pair(r, &e0, &e1)) return cudaErrorMemoryAllocation;
      if (e0) prof_record(e0, strm);
      e = k3_launch_step(r->k3, r->storage, k, t->batch, &st3, s, strm);
      if (e1 && e == cudaSuccess) e = prof_record(e1, strm);
    } else if (fused_k1) {
      K1Args k = k1_args(r);
      k.hist = t->hist;
      k.taken = t->taken;
      k.hist_stride = 6 * (int64_t)r->n;
      k.active = t->active;
      if (!prof_pair(r, &k.ev0, &k.ev1)) return cudaErrorMemoryAllocation;
      e = r->form == GROM_FORM_SVD ? svd_beta(r, t->batch, nullptr, 0, t->hist, t->taken, t->active, strm) : cudaSuccess;
      if (e == cudaSuccess) e = k1_launch_fused_step(r->k1, r->storage, k, a, t->batch, s, strm);
    } else {
      e = traj_nonlinear(t, strm);
      if (e == cudaSuccess) e = step_launch_indexed(a, r->diagonal, s, strm);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// grom_step runs a call of nsteps on the persistent stepper (so a captured
// call must too, for the same bits): the skew-packed full form with a few
// trajectories, unless the caller asked for the per-step kernels
// (GROM_KERNEL_STREAM).  One launch per call of any length: the finalize of
// the transposed term runs between grid barriers instead of in a second
// launch.
static bool persistent_ok(const grom_traj* t, int nsteps) {
  const grom_rom* r = t->rom;
  return r->form == GROM_FORM_FULL && r->layout == GROM_LAYOUT_SKEW_PACKED && r->diagonal && r->k1pp_scratch &&
         !t->active && t->batch <= 4 && t->batch <= r->k1.nb_max && nsteps >= 1 &&
         r->kernel_choice != GROM_KERNEL_STREAM && !use_k2p(r, t->batch, false);
}

grom_status grom_step(grom_traj* t, int32_t nsteps, double* energy, double* invariant) {
  TraceRange trace("grom_step");
  if (!t) return fail(GROM_ERR_INVALID_ARG, "grom_step: null trajectory");
  if (nsteps < 0) return fail(GROM_ERR_INVALID_ARG, "grom_step: nsteps < 0");
  grom_rom* r = t->rom;
  if (!full_ready(r)) return fail(GROM_ERR_INVALID_ARG, "grom_step: tensor rows missing");
  // CP forms with a few trajectories: all steps in one persistent launch
  if (r->diagonal && is_cp(r) && r->k3p_scratch && !t->active && !r->prof &&
      t->batch <= k3p_max_batch(r->storage) && nsteps >= 4 && !use_k3t(r, t->batch, false) &&
      k3p_fits(r->n, r->k3.rb, r->storage, t->batch, r->sm_count)) {
    StepArgs a = step_args(t, energy, invariant);
    cudaError_t e = k3p_launch(r->op, r->op + r->panel_bytes, r->op + 2 * r->panel_bytes, r->form, r->n, r->k3.rb,
                               r->storage, t->batch, nsteps, a, r->k3p_scratch, r->sm_count, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grom_step persistent launch");
    return GROM_OK;
  }
  // full G-ROM with the skew-packed tensor and a few trajectories: all steps
  // in one persistent launch (falls back to the graphs below when the launch
  // cannot be placed)
  if (persistent_ok(t, nsteps)) {
    StepArgs a = step_args(t, energy, invariant);
    K1Args k = k1_args(r);
    k.hist = t->hist;
    k.taken = t->taken;
    k.hist_stride = 6 * (int64_t)r->n;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!prof_pair(r, &e0, &e1)) return fail(GROM_ERR_CUDA, "event creation failed");
    k.ev0 = e0;
    k.ev1 = e1;
    const cudaError_t e = k1pp_launch(r->k1, r->storage, k, a, t->batch, nsteps, r->k1pp_scratch, r->stream);
    if (e == cudaSuccess) return GROM_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorInvalidValue)
      return cuda_fail(e, "grom_step persistent launch");
    cudaGetLastError();
    if (e0) --r->prof_used;  // the timing pair was not recorded
  }
  // batched CP forms on the tensor cores (K3T, diagonal operators): every
  // step of a call of two or more steps in one persistent cooperative
  // launch, serving pools included, up to 2^18 state elements per batch
  // (1024 trajectories of N = 1024 step faster through the per-step kernels,
  // whose step kernel hides its latency with many more warps per SM);
  // single-step calls, timed calls and launches that cannot be placed take
  // the per-step kernels below
  if (r->diagonal && is_cp(r) && r->k3t_factors && use_k3t(r, t->batch) && nsteps >= 2 && !r->prof &&
      (int64_t)t->batch * r->n <= K3TP_MAX_ELEMENTS) {
    StepArgs a = step_args(t, energy, invariant);
    K3Args k = k3_args(r);
    k.hist = t->hist;
    k.taken = t->taken;
    k.hist_stride = 6 * (int64_t)r->n;
    k.active = t->active;
    const cudaError_t e = k3tp_launch(k3t_plan_of(r, t->batch), &r->k3t_tmap_ft, &r->k3t_tmap_ae, k, t->batch,
                                      r->k3t_scratch, r->err, a, nsteps, r->sm_count, r->stream);
    if (e == cudaSuccess) return GROM_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorInvalidValue)
      return cuda_fail(e, "grom_step persistent launch");
    cudaGetLastError();
  }
  constexpr int G = 8;  // steps per captured graph
  int done = 0;
  if (!energy && !invariant && nsteps >= G) {
    // A graph of G steps, captured on a private stream (the ROM's stream may
    // be the legacy default stream, which cannot be captured) and replayed on
    // the ROM's stream.
    if (t->graph && t->graph_version != r->version) {
      cudaGraphExecDestroy(t->graph);
      cudaGraphDestroy(t->graph_tmpl);
      t->graph = nullptr;
      t->graph_tmpl = nullptr;
      t->prof_nodes.clear();
      t->prof_index.clear();
      t->prof_pairs = 0;
    }
    if (!t->graph) {
      if (!t->gstream) {
        GROM_CUDA_TRY(cudaStreamCreateWithFlags(&t->gstream, cudaStreamNonBlocking));
        GROM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_in, cudaEventDisableTiming));
        GROM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_out, cudaEventDisableTiming));
      }
      cudaGraph_t g = nullptr;
      const size_t used0 = r->prof_used;
      GROM_CUDA_TRY(cudaStreamBeginCapture(t->gstream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = launch_steps(t, G, nullptr, nullptr, t->gstream);
      cudaError_t e2 = cudaStreamEndCapture(t->gstream, &g);
      // the timing pairs taken during capture are placeholders: each replay
      // points the event nodes at fresh pairs
      const size_t used1 = r->prof_used;
      r->prof_used = used0;
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : e2, "grom_step graph capture");
      }
      if (r->prof) {
        size_t count = 0;
        e = cudaGraphGetNodes(g, nullptr, &count);
        std::vector<cudaGraphNode_t> nodes(count);
        if (e == cudaSuccess && count) e = cudaGraphGetNodes(g, nodes.data(), &count);
        for (size_t q = 0; e == cudaSuccess && q < count; ++q) {
          cudaGraphNodeType ty;
          if ((e = cudaGraphNodeGetType(nodes[q], &ty)) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
          cudaEvent_t ev;
          if ((e = cudaGraphEventRecordNodeGetEvent(nodes[q], &ev)) != cudaSuccess) break;
          for (size_t p = 2 * used0; p < 2 * used1; ++p)
            if (r->prof_ev[p] == ev) {
              t->prof_nodes.push_back(nodes[q]);
              t->prof_index.push_back((int)(p - 2 * used0));
            }
        }
        t->prof_pairs = (int)(used1 - used0);
        if (e != cudaSuccess) {
          cudaGraphDestroy(g);
          return cuda_fail(e, "grom_step graph timing nodes");
        }
      }
      e = cudaGraphInstantiate(&t->graph, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        t->prof_nodes.clear();
        t->prof_index.clear();
        return cuda_fail(e, "grom_step graph instantiate");
      }
      t->graph_tmpl = g;
      t->graph_steps = G;
      t->graph_version = r->version;
    }
    for (; done + G <= nsteps; done += G) {
      if (r->prof) {
        // fresh timing pairs for this replay, in the graph's event order
        std::vector<cudaEvent_t> evs((size_t)2 * t->prof_pairs);
        for (int k = 0; k < t->prof_pairs; ++k)
          if (!prof_pair(r, &evs[2 * k], &evs[2 * k + 1])) return fail(GROM_ERR_CUDA, "event creation failed");
        for (size_t q = 0; q < t->prof_nodes.size(); ++q)
          GROM_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(t->graph, t->prof_nodes[q], evs[t->prof_index[q]]));
      }
      GROM_CUDA_TRY(cudaGraphLaunch(t->graph, r->stream));
    }
  }
  cudaError_t e = launch_steps(t, nsteps - done, energy, invariant, r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "grom_step launch");
  return GROM_OK;
}

static bool pinned_or_device(const void* p, bool* host) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *host = at.type == cudaMemoryTypeHost;
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeDevice;
}

// The address the device uses for p (pinned host memory is mapped into the
// device's address space), or null.
static double* device_alias(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice) return const_cast<double*>(static_cast<const double*>(p));
  if (at.type == cudaMemoryTypeHost) return static_cast<double*>(at.devicePointer);
  return nullptr;
}

grom_status grom_step_host(grom_traj* t, int32_t nsteps, const double* u_in, double* u_out) {
  TraceRange trace("grom_step_host");
  if (!t) return fail(GROM_ERR_INVALID_ARG, "grom_step_host: null trajectory");
  grom_rom* r = t->rom;
  const int64_t n = r->n;
  const size_t bytes = (size_t)t->batch * n * sizeof(double);
  if (nsteps < 0) return fail(GROM_ERR_INVALID_ARG, "grom_step_host: nsteps must be >= 0");
  if (!full_ready(r)) return fail(GROM_ERR_INVALID_ARG, "grom_step_host: tensor rows missing");
  bool in_host = false, out_host = false;
  // Short calls with pinned (or device) buffers: the copy in, the steps and
  // the copy out replay as one captured graph, one launch per call.  (Longer
  // CP calls keep the persistent stepper of grom_step.)
  if (u_in && u_out && nsteps >= 1 && nsteps <= 8 && !r->prof && !t->active &&
      (!is_cp(r) || nsteps < 4) && pinned_or_device(u_in, &in_host) &&
      pinned_or_device(u_out, &out_host)) {
    if (t->io_graph && (t->io_in != u_in || t->io_out != u_out || t->io_steps != nsteps || t->io_version != r->version)) {
      cudaGraphExecDestroy(t->io_graph);
      t->io_graph = nullptr;
    }
    if (!t->io_graph) {
      if (!t->gstream) {
        GROM_CUDA_TRY(cudaStreamCreateWithFlags(&t->gstream, cudaStreamNonBlocking));
        GROM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_in, cudaEventDisableTiming));
        GROM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_out, cudaEventDisableTiming));
      }
      // The state moves straight between the caller's buffers and the
      // history ring (pinned host memory through its device mapping, no
      // copy nodes); the steps are the persistent stepper where it applies
      // (one cooperative launch), else the per-step kernels.
      double* din = device_alias(u_in);
      double* dout = device_alias(u_out);
      cudaError_t e = cudaSuccess, e2 = cudaSuccess;
      for (int attempt = 0; attempt < 2; ++attempt) {
        const bool persist = attempt == 0 && persistent_ok(t, nsteps);
        if (attempt == 1 && !persistent_ok(t, nsteps)) break;  // the first attempt was already the plain one
        cudaGraph_t g = nullptr;
        GROM_CUDA_TRY(cudaStreamBeginCapture(t->gstream, cudaStreamCaptureModeThreadLocal));
        e = cudaSuccess;
        if (din) {
          e = state_io_launch(t->hist, t->taken, n, t->batch, din, true, t->gstream);
        } else {
          e = cudaMemcpyAsync(t->io, u_in, bytes, cudaMemcpyDefault, t->gstream);
          if (e == cudaSuccess) e = state_io_launch(t->hist, t->taken, n, t->batch, t->io, true, t->gstream);
        }
        if (e == cudaSuccess) {
          if (persist) {
            StepArgs a = step_args(t, nullptr, nullptr);
            K1Args k = k1_args(r);
            k.hist = t->hist;
            k.taken = t->taken;
            k.hist_stride = 6 * (int64_t)r->n;
            e = k1pp_launch(r->k1, r->storage, k, a, t->batch, nsteps, r->k1pp_scratch, t->gstream);
          } else {
            e = launch_steps(t, nsteps, nullptr, nullptr, t->gstream);
          }
        }
        if (e == cudaSuccess) {
          if (dout) {
            e = state_io_launch(t->hist, t->taken, n, t->batch, dout, false, t->gstream);
          } else {
            e = state_io_launch(t->hist, t->taken, n, t->batch, t->io, false, t->gstream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(u_out, t->io, bytes, cudaMemcpyDefault, t->gstream);
          }
        }
        e2 = cudaStreamEndCapture(t->gstream, &g);
        if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&t->io_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess && e2 == cudaSuccess) break;
        cudaGetLastError();
        t->io_graph = nullptr;
        if (!persist) break;  // the persistent launch could not be captured: retry with the per-step kernels
      }
      if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        t->io_graph = nullptr;
        return cuda_fail(e != cudaSuccess ? e : e2, "grom_step_host graph");
      }
      t->io_in = u_in;
      t->io_out = u_out;
      t->io_steps = nsteps;
      t->io_version = r->version;
    }
    GROM_CUDA_TRY(cudaGraphLaunch(t->io_graph, r->stream));
    if (out_host) GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
    return GROM_OK;
  }
  if (u_in) {
    GROM_CUDA_TRY(cudaMemcpyAsync(t->io, u_in, bytes, cudaMemcpyDefault, r->stream));
    GROM_CUDA_TRY(state_io_launch(t->hist, t->taken, n, t->batch, t->io, true, r->stream));
  }
  grom_status st = grom_step(t, nsteps, nullptr, nullptr);
  if (st) return st;
  if (u_out) {
    GROM_CUDA_TRY(state_io_launch(t->hist, t->taken, n, t->batch, t->io, false, r->stream));
    GROM_CUDA_TRY(cudaMemcpyAsync(u_out, t->io, bytes, cudaMemcpyDefault, r->stream));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, u_out) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
    }
  }
  return GROM_OK;
}

grom_status grom_set_kernel(grom_rom* r, int32_t kernel) {
  if (!r) return fail(GROM_ERR_INVALID_ARG, "grom_set_kernel: null rom");
  if (kernel < GROM_KERNEL_AUTO || kernel > GROM_KERNEL_TENSOR)
    return fail(GROM_ERR_INVALID_ARG, "grom_set_kernel: unknown kernel");
  if (kernel == GROM_KERNEL_TENSOR && !(r->form == GROM_FORM_FULL && r->storage == GROM_BF16 && r->k2_ok) &&
      !(is_cp(r) && (r->k3t_factors || r->k3o_factors)))
    return fail(GROM_ERR_UNSUPPORTED,
                "grom_set_kernel: the tensor-core kernels need BF16 storage (full or CP form) or an FP64 CP ROM of "
                "16 or more trajectories");
  if (kernel == GROM_KERNEL_TENSOR) {
    grom_status st = build_k2_tiles(r);
    if (st) return st;
  }
  r->kernel_choice = kernel;
  ++r->version;
  return GROM_OK;
}

int32_t grom_tune_space(int32_t form, int32_t storage, int32_t layout, int32_t n, int32_t rank, int32_t max_batch,
                        int32_t batch, int32_t sm_count, grom_tuning* out, int32_t cap) {
  const bool cp = form == GROM_FORM_CP || form == GROM_FORM_CP_SKEW;
  if (n < 1 || max_batch < 1 || batch < 1 || batch > max_batch || sm_count < 1 || cap < 0 || (cap > 0 && !out) ||
      storage_elem_bytes(storage) == 0 || form < GROM_FORM_FULL || form > GROM_FORM_SVD ||
      (layout != GROM_LAYOUT_DENSE && layout != GROM_LAYOUT_SKEW_PACKED) || ((cp || form == GROM_FORM_SVD) && rank < 1))
    return -1;
  TuneShape s;
  s.form = form;
  s.storage = storage;
  s.layout = layout;
  s.max_batch = max_batch;
  s.sm_count = sm_count;
  s.n = n;
  s.rank = rank;
  if (form == GROM_FORM_FULL && storage == GROM_BF16) {
    const bool packed = layout == GROM_LAYOUT_SKEW_PACKED;
    s.tensor = true;
    s.lp = k1_plan(n, storage, sm_count, packed ? 1 : 0).lp;
    s.k2_scratch = packed ? k2p_scratch_need(n, s.lp, max_batch, sm_count) : k2_scratch_need(n, max_batch, sm_count);
  } else if (cp && storage == GROM_BF16) {
    s.tensor = true;
    s.k3t_scratch = k3t_scratch_need(n, rank, form, max_batch, sm_count);
  }
  std::vector<grom_tuning> v;
  tune_space(s, batch, v);
  for (size_t i = 0; i < v.size() && (int64_t)i < cap; ++i) out[i] = v[i];
  return (int32_t)v.size();
}

grom_status grom_autotune(grom_rom* r, int32_t batch, int32_t reps, grom_tuning* out) {
  TraceRange trace("grom_autotune");
  if (!r) return fail(GROM_ERR_INVALID_ARG, "grom_autotune: null rom");
  if (batch < 1 || batch > r->max_batch) return fail(GROM_ERR_INVALID_ARG, "grom_autotune: batch out of range");
  if (reps < 0 || reps > 10000) return fail(GROM_ERR_INVALID_ARG, "grom_autotune: reps out of range");
  if (!full_ready(r)) return fail(GROM_ERR_INVALID_ARG, "grom_autotune: tensor rows missing");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  GROM_CUDA_TRY(cudaStreamIsCapturing(r->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(GROM_ERR_INVALID_ARG, "grom_autotune: the stream is being captured");
  grom_status st = grom_sync(r);  // earlier work's errors are reported as they are
  if (st) return st;
  if (reps == 0) reps = 10;
  const TuneShape shape = shape_of(r);
  std::vector<grom_tuning> cand;
  tune_space(shape, batch, cand);
  if (shape.tensor && (st = build_k2_tiles(r))) return st;

  const int64_t n = r->n, cnt = (int64_t)batch * n;
  std::vector<double> hu((size_t)cnt);
  for (int64_t b = 0; b < batch; ++b)
    for (int64_t i = 0; i < n; ++i) hu[(size_t)(b * n + i)] = std::cos(0.37 * (double)(i + 1) + 1.3 * (double)b) / (double)(i + 1);
  const size_t bucket = (size_t)((batch + 15) / 16) - 1;
  if (r->tuning.size() <= bucket) r->tuning.resize(bucket + 1, grom_tuning{});
  const grom_tuning saved = r->tuning[bucket];
  const int saved_choice = r->kernel_choice;
  const bool saved_prof = r->prof;
  double *du = nullptr, *dc = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  auto finish = [&](grom_status code) {
    cudaStreamSynchronize(r->stream);
    r->kernel_choice = saved_choice;
    r->prof = saved_prof;
    if (code != GROM_OK) r->tuning[bucket] = saved;
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (du) cudaFree(du);
    if (dc) cudaFree(dc);
    ++r->version;  // captured graphs hold the plans
    return code;
  };
  if ((st = dmalloc(&du, (size_t)cnt * sizeof(double), nullptr)) ||
      (st = dmalloc(&dc, (size_t)cnt * sizeof(double), nullptr)))
    return finish(st);
  if (cudaMemcpy(du, hu.data(), (size_t)cnt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
    return finish(cuda_fail(cudaGetLastError(), "grom_autotune"));
  r->kernel_choice = GROM_KERNEL_AUTO;  // the entry under test picks the kernel
  r->prof = false;
  for (grom_tuning& c : cand) {
    r->tuning[bucket] = c;
    for (int w = 0; w < 2; ++w)
      if ((st = grom_nonlinear(r, batch, du, dc))) return finish(st);
    float g[3];
    for (int q = 0; q < 3; ++q) {
      if (cudaEventRecord(ev[0], r->stream) != cudaSuccess) return finish(cuda_fail(cudaGetLastError(), "grom_autotune"));
      for (int k = 0; k < reps; ++k)
        if ((st = grom_nonlinear(r, batch, du, dc))) return finish(st);
      float ms = 0.f;
      if (cudaEventRecord(ev[1], r->stream) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess)
        return finish(cuda_fail(cudaGetLastError(), "grom_autotune"));
      g[q] = ms / (float)reps;
    }
    std::sort(g, g + 3);
    c.ms = g[1];
  }
  if ((st = grom_sync(r))) return finish(st);
  size_t best = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (cand[i].ms < cand[best].ms) best = i;
  grom_tuning chosen = cand[best].ms < 0.98f * cand[0].ms ? cand[best] : cand[0];
  chosen.timed = (int32_t)cand.size();
  chosen.ms_rule = cand[0].ms;
  r->tuning[bucket] = chosen;
  if (out) *out = chosen;
  return finish(GROM_OK);
}

grom_status grom_set_tuning(grom_rom* r, const grom_tuning* t) {
  if (!r || !t) return fail(GROM_ERR_INVALID_ARG, "grom_set_tuning: null argument");
  if (t->batch < 1 || t->batch > r->max_batch) return fail(GROM_ERR_INVALID_ARG, "grom_set_tuning: batch out of range");
  const size_t bucket = (size_t)((t->batch + 15) / 16) - 1;
  if (t->kernel == GROM_KERNEL_AUTO) {
    if (bucket < r->tuning.size()) r->tuning[bucket] = grom_tuning{};
    ++r->version;
    return GROM_OK;
  }
  if (!tuning_ok(shape_of(r), *t))
    return fail(GROM_ERR_INVALID_ARG, "grom_set_tuning: the ROM's plans do not admit this configuration");
  if (t->kernel == GROM_KERNEL_TENSOR) {
    grom_status st = build_k2_tiles(r);
    if (st) return st;
  }
  if (r->tuning.size() <= bucket) r->tuning.resize(bucket + 1, grom_tuning{});
  r->tuning[bucket] = *t;
  ++r->version;
  return GROM_OK;
}

grom_status grom_get_tuning(const grom_rom* r, int32_t batch, grom_tuning* out) {
  if (!r || !out) return fail(GROM_ERR_INVALID_ARG, "grom_get_tuning: null argument");
  if (batch < 1 || batch > r->max_batch) return fail(GROM_ERR_INVALID_ARG, "grom_get_tuning: batch out of range");
  const grom_tuning* t = tuned(r, batch);
  if (t) {
    *out = *t;
  } else {
    *out = grom_tuning{};
    out->batch = batch;
  }
  return GROM_OK;
}

grom_status grom_profile_enable(grom_rom* r, int32_t enable) {
  if (!r) return fail(GROM_ERR_INVALID_ARG, "grom_profile_enable: null rom");
  GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
  if (r->prof != (enable != 0)) ++r->version;  // captured graphs carry (or lack) timing nodes
  r->prof = enable != 0;
  r->prof_used = 0;
  return GROM_OK;
}

grom_status grom_profile_read(grom_rom* r, double* total_ms, int64_t* launches) {
  if (!r || !total_ms || !launches) return fail(GROM_ERR_INVALID_ARG, "grom_profile_read: null argument");
  GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
  double sum = 0.0;
  for (size_t q = 0; q < r->prof_used; ++q) {
    float ms = 0.f;
    GROM_CUDA_TRY(cudaEventElapsedTime(&ms, r->prof_ev[2 * q], r->prof_ev[2 * q + 1]));
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)r->prof_used;
  r->prof_used = 0;
  return GROM_OK;
}

grom_status grom_traj_status(grom_traj* t, int32_t* first_bad) {
  if (!t) return fail(GROM_ERR_INVALID_ARG, "grom_traj_status: null trajectory");
  grom_status st = grom_sync(t->rom);
  if (st) return st;
  int flags[2];
  GROM_CUDA_TRY(cudaMemcpy(flags, t->err, sizeof(flags), cudaMemcpyDeviceToHost));
  if (first_bad) *first_bad = (flags[0] & DEV_ERR_NONFINITE) ? flags[1] : -1;
  if (flags[0] & DEV_ERR_NONFINITE) return fail(GROM_ERR_NONFINITE, "a trajectory state became non-finite");
  return GROM_OK;
}

grom_status grom_get_state(grom_traj* t, double* hist) {
  if (!t || !hist) return fail(GROM_ERR_INVALID_ARG, "grom_get_state: null argument");
  grom_rom* r = t->rom;
  if (!full_ready(r)) return fail(GROM_ERR_INVALID_ARG, "grom_get_state: tensor rows missing");
  const int64_t n = r->n, B = t->batch;
  // n^l of the newest state, so the export is self-consistent
  cudaError_t e = traj_nonlinear(t, r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "grom_get_state");
  grom_status st = grom_sync(r);
  if (st) return st;
  std::vector<double> ring((size_t)(B * 6 * n));
  std::vector<int64_t> taken((size_t)B);
  GROM_CUDA_TRY(cudaMemcpy(ring.data(), t->hist, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
  GROM_CUDA_TRY(cudaMemcpy(taken.data(), t->taken, taken.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
  for (int64_t b = 0; b < B; ++b) {
    const int64_t l = taken[b];
    double* dst = hist + b * (6 * n + 1);
    for (int q = 0; q < 3; ++q) {
      const int64_t m = ((l - q) % 3 + 3) % 3;
      std::memcpy(dst + q * n, ring.data() + (b * 6 + m) * n, (size_t)n * sizeof(double));
      std::memcpy(dst + (3 + q) * n, ring.data() + (b * 6 + 3 + m) * n, (size_t)n * sizeof(double));
    }
    dst[6 * n] = (double)l;
  }
  return GROM_OK;
}

grom_status grom_set_state(grom_traj* t, const double* hist) {
  if (!t || !hist) return fail(GROM_ERR_INVALID_ARG, "grom_set_state: null argument");
  grom_rom* r = t->rom;
  const int64_t n = r->n, B = t->batch;
  std::vector<double> ring((size_t)(B * 6 * n));
  std::vector<int64_t> taken((size_t)B);
  for (int64_t b = 0; b < B; ++b) {
    const double* src = hist + b * (6 * n + 1);
    const double lf = src[6 * n];
    if (!(lf >= 0.0) || lf != std::floor(lf) || lf > 9.0e15)
      return fail(GROM_ERR_INVALID_ARG, "grom_set_state: bad step count");
    const int64_t l = (int64_t)lf;
    taken[b] = l;
    for (int q = 0; q < 3; ++q) {
      const int64_t m = ((l - q) % 3 + 3) % 3;
      std::memcpy(ring.data() + (b * 6 + m) * n, src + q * n, (size_t)n * sizeof(double));
      std::memcpy(ring.data() + (b * 6 + 3 + m) * n, src + (3 + q) * n, (size_t)n * sizeof(double));
    }
  }
  GROM_CUDA_TRY(cudaStreamSynchronize(r->stream));
  GROM_CUDA_TRY(cudaMemcpy(t->hist, ring.data(), ring.size() * sizeof(double), cudaMemcpyHostToDevice));
  GROM_CUDA_TRY(cudaMemcpy(t->taken, taken.data(), taken.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  return GROM_OK;
}

}  // extern "C"
