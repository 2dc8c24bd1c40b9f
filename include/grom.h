/*
 * grom.h — C ABI of the GB300 Galerkin reduced-order-model engine.
 *
 * The library evaluates the advection term of a Galerkin ROM and steps the
 * reduced system with the semi-implicit BDFk/EXTk scheme of arXiv 2311.03694
 * ("Accelerating Galerkin Reduced-Order Models for Turbulent Flows with
 * Tensor Decomposition"), on one CUDA GPU (sm_103a).
 *
 *   model      B du/dt = -C(u)u - nu A u                       (Sec. 2.2, eq. nse_ode)
 *   full form  [C(u)u]_i = sum_jk C_ijk u_j u_k                 (Sec. 2.2, eq. Cu; cost 2N^3)
 *   CP form    [C(u)u]_i = sum_r a_ir (sum_j b_jr u_j)(sum_k c_kr u_k)   (Sec. 3.1, eq. tc_ap)
 *   skew CP    A1 = [U W], A2 = [V V], A3 = [W -U]              (Sec. 3.3, eq. skew_abc_struct)
 *   step       (beta0/dt B + nu A) u^{l+1} = -sum_i alpha_i (n^{l+1-i} + L u^{l+1-i} + f)
 *                                            - B sum_i beta_i/dt u^{l+1-i}   (Sec. 2.2, eq. nse_d1)
 *
 * Index convention: a dense tensor is row-major, entry C[(i*n + j)*n + k],
 * with i the test index, j the advecting index and k the advected index (the
 * paper writes C_ikj with j and k named the other way round).  CP factors are
 * n x rank row-major.  Vectors of a batch are batch x n row-major.
 *
 * Conventions for every call:
 *  - Every call returns a grom_status; nothing throws across the ABI.  On an
 *    error, grom_last_error() returns a message (thread-local, valid until
 *    the next call on the same thread).
 *  - Calls that take a stream enqueue work asynchronously on it; errors of
 *    the enqueued kernels surface at the next synchronising call
 *    (grom_traj_status, grom_get_state, grom_sync) as GROM_ERR_CUDA.
 *  - Pointer arguments documented as "host or device" may point to either;
 *    the library copies from them with cudaMemcpyDefault and never keeps them.
 *  - Objects are not thread-safe: serialise calls on one object.
 */
#ifndef GROM_H
#define GROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t grom_status;
#define GROM_OK 0
#define GROM_ERR_INVALID_ARG 1
#define GROM_ERR_OOM 2
#define GROM_ERR_CUDA 3
#define GROM_ERR_NONFINITE 4
#define GROM_ERR_TIMEOUT 5
#define GROM_ERR_BUDGET 6
#define GROM_ERR_UNSUPPORTED 7

/* Form of the advection operator. */
#define GROM_FORM_FULL 0    /* dense n^3 tensor (standard G-ROM, eq. Cu)          */
#define GROM_FORM_CP 1      /* general CP factors fa=A1, fb=A2, fc=A3 (eq. tc_ap)  */
#define GROM_FORM_CP_SKEW 2 /* skew CP blocks fa=U, fb=V, fc=W (eq. skew_abc_struct):
                               evaluated as c = U(p o q) - W(p o s) with p = V^T u,
                               q = W^T u, s = U^T u; paper rank 2*rank            */
#define GROM_FORM_SVD 3     /* SVD-ROM (Sec. 4.4.2): truncated SVD of the tensor's
                               matricization over the advecting index,
                               C_ijk ~ sum_r U_jr sigma_r V[i][r][k], with
                               fa = U (n x rank), fb = sigma (rank values) and
                               fc = V (n x rank x n, V[i][r][k], each slice
                               V[.][r][.] an n x n matrix over (test, advected));
                               evaluated as c_i = sum_r beta_r sum_k V[i][r][k] u_k,
                               beta = sigma o (U^T u); storage and layout apply to V
                               (the skew-packed layout needs each slice skew) */

/* Storage (and arithmetic) type of the advection operator on the device.
 * The state update, the reduced solve and the energy/invariant sums are FP64
 * in every case. */
#define GROM_F64 0   /* IEEE double; FP64 fused multiply-add                       */
#define GROM_F32X2 1 /* each double split once into hi = rn(x), lo = rn(x - hi)
                        (two floats, 8 bytes, 48 significant bits); products and
                        sums use error-free FP32 transformations on the FP32 pipe */
#define GROM_F32 2   /* rn(x) to float; FP32 accumulation                          */
#define GROM_BF16 3  /* rn(x) to bfloat16; FP32 accumulation                       */

/* Stored layout of the FULL tensor.
 *
 * GROM_LAYOUT_DENSE: all n^3 entries (rows (i, j), advected index k inner).
 *
 * GROM_LAYOUT_SKEW_PACKED: for the skew-symmetric tensors of the energy-
 * conserving G-ROM (Sec. 3.2: C_ijk = -C_kji, test and advected index
 * swapped; hence C_iji = 0), each unordered pair {i, k} is stored once.  Row
 * (i, j) keeps the entries k = (i + d) mod n for d = 1 .. floor(n/2); for even
 * n the entry at d = n/2 is kept only in rows with i < n/2 (row i >= n/2
 * stores zero there).  The other entries follow from C_ijk = -C_kji, so
 *   c_i = sum_j u_j [ sum_d C_{i,j,i+d} u_{i+d} - sum_d C_{i-d,j,i} u_{i-d} ]
 * (indices mod n) is the same contraction as the dense one.  This halves the
 * bytes and the multiply-adds of the streaming contraction.
 * The caller's tensor must be skew to rounding.  While uploading, the library
 * forms the probe sum_ijk x_i y_j x_k C_ijk for two seeded +-1 vector pairs
 * (zero for a skew tensor, about ||sym(C)||_F otherwise) and rejects the
 * tensor with GROM_ERR_INVALID_ARG if a probe exceeds 1e-9 ||C||_F.  With
 * BF16 storage, batches of the packed tensor go to the factored tensor-core
 * kernel K2P (see GROM_KERNEL_TENSOR); with the other storage types, every
 * batch goes to the streaming kernel. */
#define GROM_LAYOUT_DENSE 0
#define GROM_LAYOUT_SKEW_PACKED 1

typedef struct grom_rom grom_rom;
typedef struct grom_traj grom_traj;

typedef struct grom_desc {
  int32_t n;       /* number of modes N >= 1                                       */
  int32_t form;    /* GROM_FORM_*                                                  */
  int32_t rank;    /* CP or SVD rank (columns of each factor); ignored for FULL   */
  int32_t storage; /* GROM_F64, GROM_F32X2, GROM_F32, GROM_BF16                     */
  /* FULL: n*n*n doubles, host or device; NULL together with defer_tensor = 1
   * to upload the rows later with grom_upload_tensor_slab. */
  const double* tensor;
  /* CP forms: three n x rank factor matrices, host or device.  SVD form: see
   * GROM_FORM_SVD (U: n x rank, sigma: rank, V: n x rank x n). */
  const double* fa;
  const double* fb;
  const double* fc;
  /* Stiffness A: n*n dense (stiffness) or its diagonal (stiffness_diag, n
   * entries); exactly one must be given.  Host or device. */
  const double* stiffness;
  const double* stiffness_diag;
  /* Mass B: n*n dense, its diagonal (mass_diag), or both NULL for identity. */
  const double* mass;
  const double* mass_diag;
  /* Optional explicit linear operator L (n*n) and constant forcing f (n),
   * both extrapolated with EXTk (NULL = zero).  In the paper's notation
   * L = C1 + C2 restricted to modes 1..N and f collects -c0 and nu*a0
   * (Sec. 2.2, eq. zeroth_contribution). */
  const double* linear;
  const double* linear_diag; /* diagonal of L (n entries) instead of `linear`  */
  const double* forcing;
  double nu;     /* viscosity 1/Re (> = 0)                                          */
  double dt;     /* time step (> 0)                                                 */
  int32_t order; /* BDF/EXT order k in 1..3; steps 1 and 2 use orders 1 and 2       */
  int32_t defer_tensor; /* FULL only: 1 = rows come from grom_upload_tensor_slab  */
  int32_t max_batch;    /* largest batch passed to grom_nonlinear/grom_traj_create
                           (sizes the library's scratch); 0 means 1.  FULL, BF16,
                           dense layout, max_batch > 8: the library also keeps a
                           tile-major copy of the tensor (another n^3 * 2 bytes)
                           for the tensor-core kernel; if that allocation fails
                           the kernel reads the row-major tensor instead      */
  int32_t layout;       /* FULL and SVD: GROM_LAYOUT_DENSE (0) or GROM_LAYOUT_SKEW_PACKED */
  /* 1: the operator includes the zeroth mode phi_0 (coefficient 1 in the
   * augmented vector ubar = (1, u), eq. nse_ode; the "full" tensor of
   * Sec. 4.2).  FULL: tensor holds n x (n+1) x (n+1) doubles Cbar[i][j][k]
   * (j, k = 0 is the zeroth mode; defer_tensor not allowed).  The core
   * j, k >= 1 becomes the advection tensor, and the zeroth-mode terms join the
   * stepper (eq. nse_d1, eq. zeroth_contribution): L += C1 + C2 with
   * C1_ik = Cbar[i][0][k], C2_ij = Cbar[i][j][0], and f += c0 with
   * c0_i = Cbar[i][0][0].  CP (general form only): fb and fc have n+1 rows,
   * row 0 the zeroth mode; L += A diag(fb_0) fc'^T + A diag(fc_0) fb'^T and
   * f += A (fb_0 o fc_0), fb', fc' the rows 1..n.  grom_nonlinear then
   * evaluates the core term only; grom_step advances the full model. */
  int32_t augmented;
  /* FULL, dense layout, BF16 storage and max_batch > 8: by default the
   * library keeps a tile-major copy of the stored tensor beside it for the
   * tensor-core kernel K2 (every 256 x 64 operand tile one contiguous block;
   * round_up(n, 256) * n * round_up(n, 64) * 2 bytes).  1: keep the row layout
   * only (less memory; K2 then reads the row layout, at lower bandwidth for
   * small batches).  The skew-packed layout keeps no copy. */
  int32_t no_tile_copy;
  int32_t reserved;     /* must be zero                                           */
} grom_desc;

/* Creates a ROM on the current CUDA device.  Every input is copied; the caller
 * keeps ownership.  Operators are converted once (round to nearest even) to
 * the storage type; H_k = beta0_k/dt B + nu A is factored in FP64 and its
 * inverse cached for k = 1..order.  `stream` (cudaStream_t, may be NULL for
 * the legacy default stream) is where all later work of this ROM runs.
 * Errors: INVALID_ARG (bad sizes, pointers or combination), OOM, CUDA,
 * UNSUPPORTED (n too large for the storage type, see grom_max_n). */
grom_status grom_create(const grom_desc* desc, void* stream, grom_rom** out);

/* Copies tensor rows i0..i1-1 (rows of n*n doubles, host or device) into a ROM
 * created with defer_tensor = 1, converting them to the storage type.  All n
 * rows must be uploaded before the first evaluation. */
grom_status grom_upload_tensor_slab(grom_rom* rom, int32_t i0, int32_t i1, const double* rows);

/* Frees the ROM.  Waits for its stream; trajectories of the ROM must be
 * destroyed first. */
grom_status grom_destroy(grom_rom* rom);

/* Largest n supported for a storage type and form. */
int32_t grom_max_n(int32_t form, int32_t storage);

/* Evaluates c_b = C(u_b) u_b (positive sign) for b < batch.  u and c are
 * DEVICE pointers to batch x n FP64 arrays owned by the caller; they must not
 * overlap.  Asynchronous on the ROM's stream.  batch <= max_batch. */
grom_status grom_nonlinear(grom_rom* rom, int32_t batch, const double* u, double* c);

/* Creates `batch` trajectories of the ROM starting from u0 (batch x n FP64,
 * host or device), with no steps taken. */
grom_status grom_traj_create(grom_rom* rom, int32_t batch, const double* u0, grom_traj** out);
grom_status grom_traj_destroy(grom_traj* traj);

/* Advances every trajectory by nsteps steps of eq. nse_d1 (orders 1, 2, then
 * desc.order).  energy and invariant are nullable DEVICE pointers to
 * nsteps x batch doubles receiving, per step, E = 1/2 u^T B u of the new state
 * and u^T C(u)u of the state the step started from.  Asynchronous; a
 * non-finite state is recorded and reported by grom_traj_status. */
grom_status grom_step(grom_traj* traj, int32_t nsteps, double* energy, double* invariant);

/* Host round trip of a stepping call: if u_in is non-NULL it replaces the
 * newest state u^l of every trajectory (batch x n, host or device; the older
 * history is kept, as when an observed state is fed back in an online loop),
 * then nsteps steps are taken, then, if u_out is non-NULL, the newest state is
 * copied to it (batch x n, host or device).  Synchronous when either pointer
 * is host memory. */
grom_status grom_step_host(grom_traj* traj, int32_t nsteps, const double* u_in, double* u_out);

/* Synchronises the ROM's stream and reports GROM_ERR_NONFINITE (first bad
 * trajectory index in *first_bad, else -1) or GROM_OK. */
grom_status grom_traj_status(grom_traj* traj, int32_t* first_bad);

/* Checkpoint / resume.  hist is HOST memory of batch x (6n+1) doubles; per
 * trajectory: u^l, u^{l-1}, u^{l-2}, n^l, n^{l-1}, n^{l-2} (n each) and the
 * number of steps taken.  n^l is C(u^l)u^l of the newest state.  Get
 * synchronises; set is ordered on the ROM's stream. */
grom_status grom_get_state(grom_traj* traj, double* hist);
grom_status grom_set_state(grom_traj* traj, const double* hist);

/* Waits for all work of the ROM. */
grom_status grom_sync(grom_rom* rom);

/* Bytes of device memory held by the ROM (operators, caches and scratch). */
int64_t grom_rom_bytes(const grom_rom* rom);

/* Choice of the contraction kernel.  AUTO picks the tensor-core kernel for
 * BF16 storage and batches above 8 trajectories (full form) or of 16 and more
 * (CP forms), else the streaming (full) or SIMT (CP) kernels; an autotuning
 * entry for the batch's bucket (grom_autotune, grom_set_tuning) replaces that
 * rule.  FP64 CP ROMs step batches of 16 and more at FP64 tolerance
 * (per-evaluation error ~1e-13 against FP64) with K3D: the projections and
 * the expansion as double-single FP32 GEMMs (every operand a hi/lo FP32 pair,
 * error-free products and sums) on hi/lo copies of the factors made at
 * create; from N R B >= 2^24 on (N modes, R rank, B trajectories), and with
 * GROM_KERNEL_TENSOR, with K3O: every operand split into integer digit
 * slices (eight of 7 bits for the projections of ROMs with N <= 1024, else
 * nine of 6 bits), the slice products on the tcgen05 tensor cores (exact in
 * FP32 for dot products of up to 1024 and 4096 terms respectively, so N and
 * the expansion's 2R (skew) or R at most 4096) and the slice pairs summed in
 * double-single arithmetic. */
#define GROM_KERNEL_AUTO 0
#define GROM_KERNEL_STREAM 1 /* K1: SIMT streaming kernel, up to 8 trajectories per pass, one
                                launch per step (no persistent stepper); CP forms: the SIMT
                                kernels (K3, K3g; FP64 factors in FP64 arithmetic, no K3D)    */
#define GROM_KERNEL_TENSOR 2 /* BF16 storage (and FP64 CP forms, below).  Dense layout, K2: tcgen05 GEMM over the
                                Khatri-Rao product of the states (Sec. 2.2, eq. Cu with the
                                mode-1 matricisation).  Skew-packed layout, K2P: the factored
                                form, one tcgen05 GEMM D_i = P_i^T U^T per test index i over
                                the stored half, then c_i += D_i u_k and c_k -= D_i u_i for
                                every stored pair (i, k); half the bytes and MMA work of K2.
                                Rows of more than 128 stored positions run one 256-row MMA
                                over each pair of SMs (a cluster of two CTAs, cta_group::2).
                                CP forms, K3T: the projections [B C]^T X (skew: [V W U]^T X)
                                and the expansion A Z (skew: [U, -W] Z) of the batch as two
                                tcgen05 GEMMs (Sec. 3.1, eq. tc_ap; Sec. 3.3).  FP64 CP forms
                                (batches of 16 and more): K3O, the same two GEMMs on digit
                                slices of the factors and of the states (FP64 tolerance)     */
grom_status grom_set_kernel(grom_rom* rom, int32_t kernel);

/* ------------------------------------------------------------ autotuning
 * The launch shapes of the batched tensor-core kernels come from fixed rules
 * (their plans): K2 splits the advecting index j across CTAs, K2P covers m
 * test indices per tile, K3T splits the K range of each of its two GEMMs;
 * and AUTO picks between the tensor-core and the SIMT kernels by batch size.
 * The autotuner times the alternatives on the device and keeps the fastest
 * for the ROM, per batch bucket: batches with the same ceil(batch / 16) have
 * identical plans apart from the batch itself, so one entry serves them all.
 * Entries change only which valid configuration runs (the results differ by
 * FP32 summation order, within each kernel's bound); the persistent steppers
 * (few trajectories, whole step in one launch) ignore them, and a kernel
 * forced by grom_set_kernel overrides an entry's `kernel`. */
typedef struct grom_tuning {
  int32_t batch;   /* trajectories tuned for; the entry serves ceil(batch / 16)       */
  int32_t kernel;  /* GROM_KERNEL_STREAM or GROM_KERNEL_TENSOR (in grom_set_tuning,
                      GROM_KERNEL_AUTO removes the bucket's entry)                      */
  int32_t tile_m;  /* K2P: test indices per tile, 8..32; 0 = the plan's rule           */
  int32_t split_a; /* K2: CTAs sharing one output tile (split of j), 1..n;
                      K3T: splits of the projection GEMM; 0 = the rule                  */
  int32_t split_b; /* K3T: splits of the expansion GEMM; K2P: 1 = one CTA per tile,
                      2 = SM pairs (one 256-row MMA over two CTAs); 0 = the rule        */
  int32_t timed;   /* grom_autotune: configurations timed                              */
  float ms;        /* grom_autotune: median device ms per evaluation of this entry      */
  float ms_rule;   /* grom_autotune: the same for the rules' configuration             */
} grom_tuning;

/* The configurations grom_autotune times for `batch` trajectories of a ROM
 * with these parameters (host arithmetic only, no device needed): the rules'
 * own first, then every alternative the plans admit whose scratch fits what
 * grom_create allocates for max_batch.  Writes up to `cap` entries to `out`
 * (NULL with cap 0 to count) and returns how many there are, or -1 for
 * invalid arguments.  sm_count: the device's multiprocessor count. */
int32_t grom_tune_space(int32_t form, int32_t storage, int32_t layout, int32_t n, int32_t rank, int32_t max_batch,
                        int32_t batch, int32_t sm_count, grom_tuning* out, int32_t cap);

/* Times every configuration of grom_tune_space for `batch` trajectories on
 * the ROM's stream: synthetic states, two untimed evaluations, then three
 * groups of `reps` (0: 10) back-to-back evaluations between CUDA events; a
 * configuration's time is the median of its groups.  Installs the fastest for
 * the bucket if it beats the rules' by more than 2 %, else the rules' (so the
 * entry records the decision), and returns the installed entry in *out
 * (nullable).  Synchronises the stream; not allowed while it is being
 * captured (INVALID_ARG).  A device-side wait that timed out returns TIMEOUT
 * and leaves the bucket untuned. */
grom_status grom_autotune(grom_rom* rom, int32_t batch, int32_t reps, grom_tuning* out);

/* Installs an entry, e.g. one saved from grom_autotune in an earlier run;
 * INVALID_ARG unless it is one of grom_tune_space's for this ROM (the timing
 * fields are ignored).  kernel = GROM_KERNEL_AUTO removes the bucket's entry. */
grom_status grom_set_tuning(grom_rom* rom, const grom_tuning* entry);

/* The entry serving `batch` (kernel = GROM_KERNEL_AUTO: none, the rules apply). */
grom_status grom_get_tuning(const grom_rom* rom, int32_t batch, grom_tuning* out);

/* ------------------------------------------------------------ serving
 * A server keeps several ROMs resident and steps trajectory requests as they
 * arrive, with continuous batching: each ROM owns a pool of max_slots
 * trajectory slots stepped together by the batched kernels (inactive slots
 * are skipped); a request is admitted into a free slot of its ROM as soon as
 * one is free and its state fits the HBM budget, is stepped in scheduling
 * quanta alongside whatever else is resident, and leaves (its final state
 * copied to the host, its slot and memory released) after its horizon.  The
 * ROMs step concurrently when they were created on different streams. */
typedef struct grom_server grom_server;

typedef struct grom_request {
  int32_t model;    /* id returned by grom_server_add_rom / _add_simulated       */
  int32_t horizon;  /* steps to take, >= 1                                       */
  double arrival;   /* seconds after the start of grom_serve                     */
  const double* u0; /* n doubles, host: initial state                            */
  double* u_final;  /* n doubles, host, or NULL: final state                     */
} grom_request;

typedef struct grom_result {
  int32_t status;   /* GROM_OK, GROM_ERR_NONFINITE (final state not finite) or
                       GROM_ERR_BUDGET (the request can never fit the budget)    */
  int32_t steps;    /* steps taken                                                */
  double t_admit;   /* seconds after start: slot and memory granted               */
  double t_done;    /* seconds after start: final state on the host               */
} grom_result;

typedef struct grom_serve_stats {
  int64_t trajectory_steps; /* steps taken by all requests                       */
  int64_t quanta;           /* scheduling rounds                                 */
  double seconds;           /* duration of grom_serve                            */
  int64_t peak_bytes;       /* peak charged footprint (models + admitted states) */
  int32_t peak_active;      /* peak number of concurrently stepped trajectories  */
  int32_t reserved;
} grom_serve_stats;

/* hbm_budget_bytes caps the footprint charged for resident models and
 * admitted trajectory states; quantum_steps (a multiple of 8 is best) is the
 * number of steps each ROM advances between scheduling decisions.  With
 * simulate = 1 nothing runs on a GPU: models are added with
 * grom_server_add_simulated and a quantum costs quantum_steps * step_seconds
 * of virtual time (for testing the scheduler). */
grom_status grom_server_create(int64_t hbm_budget_bytes, int32_t quantum_steps, int32_t simulate,
                               grom_server** out);
/* Makes `rom` resident with a pool of max_slots slots (max_slots <= the ROM's
 * max_batch).  Charged: the ROM's bytes plus the pool; GROM_ERR_BUDGET if it
 * does not fit.  The ROM must outlive the server.  The pool is stepped as one
 * batch of max_slots trajectories, so a tuning entry for that batch
 * (grom_autotune(rom, max_slots, ...) before serving) applies to it. */
grom_status grom_server_add_rom(grom_server* s, grom_rom* rom, int32_t max_slots, int32_t* model);
/* Simulation mode only: a model of n modes occupying rom_bytes whose batched
 * step takes step_seconds. */
grom_status grom_server_add_simulated(grom_server* s, int32_t n, int64_t rom_bytes, int32_t max_slots,
                                      double step_seconds, int32_t* model);
/* Runs the requests to completion in real time (arrival times are honoured;
 * simulation mode uses virtual time) and fills results[count].  Each
 * admitted request is charged 8 * (7 n + 4) bytes of trajectory state.
 * stats is nullable. */
grom_status grom_serve(grom_server* s, const grom_request* reqs, int32_t count, grom_result* results,
                       grom_serve_stats* stats);
grom_status grom_server_destroy(grom_server* s);

/* Kernel timing: while enabled, the library records CUDA events on the ROM's
 * stream around every launch of its main contraction kernel (full form: the
 * streaming kernel K1/K1P, or K2/K2P for batches on the tensor cores; CP
 * forms: the projection and expansion kernels together).
 * grom_profile_read synchronises and returns the summed device time in ms and
 * the number of timed launches since the last enable. */
grom_status grom_profile_enable(grom_rom* rom, int32_t enable);
grom_status grom_profile_read(grom_rom* rom, double* total_ms, int64_t* launches);

/* Allocation-free dense contraction for callers that cannot let a library
 * allocate device memory: programs whose HBM is owned by another allocator
 * (a framework's caching allocator, a fixed start-up budget) and real-time
 * loops where an allocation could synchronise the device or stall.  The paper
 * has no counterpart; this is an integration entry point.
 *
 * Computes c = C(u)u for ONE trajectory on `stream` (asynchronously) with the
 * same streaming kernel as grom_nonlinear, without any ROM object: tensor, u
 * and c are caller-owned DEVICE pointers.  `tensor` (16-byte aligned) is in
 * the stored layout: n*n rows, row (i*n + j) holding C_ijk for k < np and
 * zeros for n <= k < np, np = n rounded up to a multiple of 64, elements of
 * the `storage` type (GROM_F64 double, GROM_F32 float, GROM_BF16 bfloat16;
 * GROM_F32X2 rows are np floats hi = rn(C) followed by np floats
 * lo = rn(C - hi)).  For n a multiple of 64 an F64/F32/BF16 tensor is plain
 * row-major n^3.
 *
 * Scratch: a fixed 1 MiB file-scope device array inside the library (held by
 * every GPU that loads the library until the process exits), enough for any
 * n <= grom_max_n on up to ~1000 SMs; a size that needs more is rejected with
 * GROM_ERR_UNSUPPORTED.  The call makes no cudaMalloc/cudaFree and calls no
 * allocating library routine.  Its first call on each device resolves the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's partial sums, so calls that overlap on
 * the GPU (other streams, other host threads) race: serialise them.
 * `stream` (cudaStream_t, NULL = the legacy default stream) must belong to
 * the current device (GROM_ERR_INVALID_ARG otherwise), since the scratch
 * address is the current device's.  The call does not synchronise: a
 * device-side wait that times out leaves c unspecified and is reported by
 * grom_nonlinear_full_noalloc_status.
 *
 * The library cannot check the extent of caller pointers: tensor must hold
 * n*n rows of the stored layout, u and c n doubles, all on the current
 * device; anything shorter makes the kernel read or write out of bounds. */
grom_status grom_nonlinear_full_noalloc(int32_t n, int32_t storage, const void* tensor, const double* u,
                                        double* c, void* stream);

/* Outcome of the last grom_nonlinear_full_noalloc call on the current device:
 * reads its device error word on `stream` (the stream of that call) and
 * synchronises the stream.  GROM_OK, or GROM_ERR_TIMEOUT when a device wait
 * of that call gave up (its c is unspecified); the next call clears the
 * word.  Allocates nothing. */
grom_status grom_nonlinear_full_noalloc_status(void* stream);

/* Self-test of failure detection: enqueues on the ROM's stream a kernel that
 * waits on a device barrier nothing ever signals, through the same bounded
 * wait the library's kernels use, with a limit of limit_ns.  The wait gives
 * up and raises the ROM's timeout flag, so the next grom_sync returns
 * GROM_ERR_TIMEOUT (once); the ROM stays usable.  Faults nothing. */
grom_status grom_selftest_timeout(grom_rom* rom, int64_t limit_ns);

/* ------------------------------------------------------------ CP fitting
 * CP decomposition of a dense tensor by alternating least squares (Sec. 2.3,
 * eq. cp_als) or by the skew-preserving ALS-skew (Sec. 3.3, eq.
 * skew_abc_struct and cp_als_quad), the offline step that produces a
 * CPD-ROM's factors.  Every least-squares subproblem is solved through its
 * normal equations, A_m = MTTKRP_m (Hadamard product of the other two Gram
 * matrices)^-1; the MTTKRP X_(m) (P kr Q) runs on the tensor cores (BF16
 * tensor, Khatri-Rao product of the FP32 factors split into BF16 hi/lo
 * parts, FP32 accumulation, split sums in FP64); the Gram matrices and the
 * rank x rank SPD solves (blocked Cholesky, then two triangular solves per
 * row) are FP64 on the device, where the factors stay for the whole fit. */
typedef struct grom_als grom_als;
#define GROM_ALS_PLAIN 0
#define GROM_ALS_SKEW 1

/* Fitting context for the n x n x n FP64 tensor (host or device, row-major
 * [(i*n + j)*n + k], copied; the caller keeps ownership): three BF16 copies,
 * one per matricization (3 n^2 round_up(n, 64) * 2 bytes of device memory),
 * and ||X||_F^2 of that BF16 tensor (the one the fit sees) in FP64.  Runs on `stream` (cudaStream_t, may be NULL). */
grom_status grom_als_create(int32_t n, const double* tensor, void* stream, grom_als** out);

/* `iters` iterations from the given factors, updated in place (host arrays,
 * row-major FP64):
 *   GROM_ALS_PLAIN: fa, fb, fc are n x rank (A1, A2, A3); an iteration solves
 *     the subproblems for A1, A2 and A3 in turn.
 *   GROM_ALS_SKEW: rank even; fa = A1 = [A1_1 A1_2] (n x rank), fb = B1
 *     (n x rank/2), fc unused (A2 = [B1 B1], A3 = [A1_2, -A1_1]).  An
 *     iteration solves the A2 subproblem as in ALS (its two halves, equal for
 *     a skew tensor, are averaged into B1), then `subiters` times solves the
 *     A1 subproblem with A2, A3 fixed and sets A1 <- lambda A1 + (1 - lambda)
 *     A1_next, A3 = [A1_2, -A1_1] (0 <= lambda < 1).
 * ridge (>= 0): every normal matrix H gets ridge * max diag(H) added to its
 * diagonal (Tikhonov; 0 = the exact normal equations of the paper).  The
 * MTTKRP's relative noise (~1e-5 to 1e-3 under heavy cancellation) is
 * amplified by the condition number of H, which ALS on tensors dominated by a
 * few components drives to 1e9 and beyond; a ridge near 1e-5 keeps such fits
 * stable.
 * residual (nullable, iters entries): ||X - [[A1, A2, A3]]||_F / ||X||_F of the
 * BF16 tensor after each iteration, from ||X||^2 - 2 <X, K> + ||K||^2 with
 * <X, K> from one extra mode-1 MTTKRP of the final factors (the FP32
 * accumulation limits it to about 1e-5 in the squared residual).  A numerically singular normal
 * matrix is solved with a ridge mu I, mu = 1e-12 max diag, growing 100x up
 * to three times.  Errors: INVALID_ARG (sizes, odd rank for SKEW, a
 * Gram product that is not positive definite), OOM, CUDA, TIMEOUT. */
grom_status grom_als_fit(grom_als* als, int32_t rank, int32_t method, int32_t iters, double lambda, int32_t subiters,
                         double ridge, double* fa, double* fb, double* fc, double* residual);
/* Time spent since the previous call: summed device time of the MTTKRP
 * launches (CUDA events around each tensor-core launch), their number, and
 * the wall time of the SPD solves, each from its first launch to its end on
 * the device (ms).  Resets the counters. */
grom_status grom_als_stats(grom_als* als, double* mttkrp_ms, int64_t* mttkrp_calls, double* solve_ms);
grom_status grom_als_destroy(grom_als* als);

/* Message of the last failed call on this thread ("" if none). */
const char* grom_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GROM_H */
