/*
 * FP64 CPU oracle for the Galerkin ROM advection term and its BDFk/EXTk
 * time-stepper (arXiv 2311.03694).  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the GPU library
 * never does.  It shares no code with the GPU library.
 *
 * Everything here is the plain definition written out with loops, in FP64,
 * in the paper's order of operations:
 *   - full contraction  c_i = sum_j sum_k C_ijk u_j u_k          (Sec. 2.2, eq. Cu / nse_ode)
 *   - CP contraction    c_i = sum_r a_ir (sum_j b_jr u_j)(sum_k c_kr u_k)   (Sec. 3.1, eq. tc_ap)
 *   - skew CP structure A1=[U W], A2=[V V], A3=[W -U]              (Sec. 3.3, eq. skew_abc_struct)
 *   - CP reconstruction X_ijk = sum_r a_ir b_jr c_kr                (Sec. 2.3, eq. cpd)
 *   - SVD-ROM contraction c_i = sum_r sigma_r (sum_j U_jr u_j)(sum_k V[i][r][k] u_k)   (Sec. 4.4.2)
 *   - the same contractions of operators that include the zeroth mode, with the
 *     augmented vector ubar = (1, u)                                 (Sec. 2.2, eq. nse_ode; Sec. 4.2)
 *   - BDFk/EXTk step (beta0/dt B + nu A) u^{l+1} = -sum_i alpha_i (n^{l+1-i} + L u^{l+1-i} + f)
 *                                                  - B sum_i beta_i/dt u^{l+1-i}   (Sec. 2.2, eq. nse_d1)
 *     solved with a dense Cholesky factorisation written here.
 *
 * Index convention: a dense tensor is row-major C[(i*n + j)*n + k] with i the
 * test index, j the advecting index and k the advected index (the paper's
 * C_ikj with its k and j renamed).  CP factors are n x r row-major.
 *
 * Parity pins: see tests/test_oracle_*.py.  The skew-symmetry invariant
 * u^T c(u) = 0, the rank-one closed form, brute force against numpy einsum,
 * CP versus its reconstructed tensor, exact exponential decay of the linear
 * system, third-order convergence of BDF3/EXT3 and agreement with an
 * independent RK4 integration pin every function below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Thread count of the contraction loops (OpenMP over the test index). */
void oracle_set_threads(int t) {
#ifdef _OPENMP
  omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Full contraction for test rows i0..i1-1; C_rows holds those rows only
 * ((i1-i0) * n * n entries); c has i1-i0 entries. */
void oracle_nonlinear_full_rows(int64_t n, int64_t i0, int64_t i1, const double* C_rows,
                                const double* u, double* c) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = i0; i < i1; ++i) {
    const double* Ci = C_rows + (i - i0) * n * n;
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k) s += Ci[j * n + k] * u[j] * u[k];
    c[i - i0] = s;
  }
}

void oracle_nonlinear_full(int64_t n, const double* C, const double* u, double* c) {
  oracle_nonlinear_full_rows(n, 0, n, C, u, c);
}

/* CP contraction (eq. tc_ap): p = B^T u, q = C^T u, c = A (p o q). */
void oracle_nonlinear_cp(int64_t n, int64_t r, const double* A, const double* B, const double* Cf,
                         const double* u, double* c) {
  double* p = (double*)calloc((size_t)r, sizeof(double));
  double* q = (double*)calloc((size_t)r, sizeof(double));
  for (int64_t m = 0; m < r; ++m) {
    double sp = 0.0, sq = 0.0;
    for (int64_t j = 0; j < n; ++j) sp += B[j * r + m] * u[j];
    for (int64_t k = 0; k < n; ++k) sq += Cf[k * r + m] * u[k];
    p[m] = sp;
    q[m] = sq;
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t m = 0; m < r; ++m) s += A[i * r + m] * p[m] * q[m];
    c[i] = s;
  }
  free(p);
  free(q);
}

/* Skew-preserving CP structure (eq. skew_abc_struct) from its blocks
 * U = A1_1, W = A1_2 and the shared middle block V = A2_1, each n x r:
 * A1 = [U W], A2 = [V V], A3 = [W -U]; outputs are n x 2r. */
void oracle_cp_skew_expand(int64_t n, int64_t r, const double* U, const double* V, const double* W,
                           double* A1, double* A2, double* A3) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t m = 0; m < r; ++m) {
      A1[i * 2 * r + m] = U[i * r + m];
      A1[i * 2 * r + r + m] = W[i * r + m];
      A2[i * 2 * r + m] = V[i * r + m];
      A2[i * 2 * r + r + m] = V[i * r + m];
      A3[i * 2 * r + m] = W[i * r + m];
      A3[i * 2 * r + r + m] = -U[i * r + m];
    }
}

/* CP contraction of the skew structure, evaluated through the expanded
 * rank-2r factors exactly as eq. tc_ap prescribes. */
void oracle_nonlinear_cp_skew(int64_t n, int64_t r, const double* U, const double* V,
                              const double* W, const double* u, double* c) {
  size_t sz = (size_t)n * 2 * r;
  double* A1 = (double*)malloc(sz * sizeof(double));
  double* A2 = (double*)malloc(sz * sizeof(double));
  double* A3 = (double*)malloc(sz * sizeof(double));
  oracle_cp_skew_expand(n, r, U, V, W, A1, A2, A3);
  oracle_nonlinear_cp(n, 2 * r, A1, A2, A3, u, c);
  free(A1);
  free(A2);
  free(A3);
}

/* Kruskal operator (eq. cpd): X_ijk = sum_m a_im b_jm c_km. */
void oracle_cp_reconstruct(int64_t n, int64_t r, const double* A, const double* B, const double* Cf,
                           double* X) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int64_t m = 0; m < r; ++m) s += A[i * r + m] * B[j * r + m] * Cf[k * r + m];
        X[(i * n + j) * n + k] = s;
      }
}

/* SVD-ROM (Sec. 4.4.2).  The tensor's matricization over the advecting index
 * j (rows j, columns the pairs (i, k)) is approximated by its truncated SVD
 * U_R Sigma_R V_R^T; with V_R's column r read as the n x n matrix V[i][r][k],
 *   C_ijk ~ sum_r U_jr sigma_r V[i][r][k],
 * and the advection term of that tensor is
 *   c_i = sum_r sigma_r (sum_j U_jr u_j) (sum_k V[i][r][k] u_k).
 * U is n x r row-major, sigma has r entries, V is n x r x n row-major. */
void oracle_nonlinear_svd(int64_t n, int64_t r, const double* U, const double* sigma, const double* V,
                          const double* u, double* c) {
  double* a = (double*)malloc((size_t)r * sizeof(double));
  for (int64_t m = 0; m < r; ++m) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += U[j * r + m] * u[j];
    a[m] = sigma[m] * s;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ci = 0.0;
    for (int64_t m = 0; m < r; ++m) {
      double s = 0.0;
      for (int64_t k = 0; k < n; ++k) s += V[(i * r + m) * n + k] * u[k];
      ci += a[m] * s;
    }
    c[i] = ci;
  }
  free(a);
}

/* Full tensor including the zeroth mode (Sec. 4.2): Cbar is n x (n+1) x (n+1)
 * (test index 1..n, advecting and advected index 0..n, index 0 the zeroth
 * mode) and c_i = sum_{j,k=0..n} Cbar_ijk ubar_j ubar_k with ubar = (1, u). */
void oracle_nonlinear_full_augmented(int64_t n, const double* Cbar, const double* u, double* c) {
  const int64_t n1 = n + 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n1; ++j) {
      const double uj = j == 0 ? 1.0 : u[j - 1];
      for (int64_t k = 0; k < n1; ++k) {
        const double uk = k == 0 ? 1.0 : u[k - 1];
        s += Cbar[(i * n1 + j) * n1 + k] * uj * uk;
      }
    }
    c[i] = s;
  }
}

/* CP form of a tensor including the zeroth mode: A is n x r, Bbar and Cbar
 * are (n+1) x r (row 0 the zeroth mode), c_i = sum_m A_im (sum_j Bbar_jm
 * ubar_j)(sum_k Cbar_km ubar_k). */
void oracle_nonlinear_cp_augmented(int64_t n, int64_t r, const double* A, const double* Bbar, const double* Cbar,
                                   const double* u, double* c) {
  double* p = (double*)malloc((size_t)r * sizeof(double));
  double* q = (double*)malloc((size_t)r * sizeof(double));
  for (int64_t m = 0; m < r; ++m) {
    double sp = Bbar[m], sq = Cbar[m];
    for (int64_t j = 0; j < n; ++j) {
      sp += Bbar[(j + 1) * r + m] * u[j];
      sq += Cbar[(j + 1) * r + m] * u[j];
    }
    p[m] = sp;
    q[m] = sq;
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t m = 0; m < r; ++m) s += A[i * r + m] * p[m] * q[m];
    c[i] = s;
  }
  free(p);
  free(q);
}

/* ---------------------------------------------------------------- stepper */

/* BDFk/EXTk coefficients for k = 1, 2, 3 (standard values; the paper states
 * the scheme but prints no coefficients).  beta[0] multiplies u^{l+1}. */
static const double BDF_BETA[3][4] = {
    {1.0, -1.0, 0.0, 0.0},
    {1.5, -2.0, 0.5, 0.0},
    {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0},
};
static const double EXT_ALPHA[3][3] = {
    {1.0, 0.0, 0.0},
    {2.0, -1.0, 0.0},
    {3.0, -3.0, 1.0},
};

void oracle_bdf_ext_coefficients(int k, double* beta4, double* alpha3) {
  for (int i = 0; i < 4; ++i) beta4[i] = BDF_BETA[k - 1][i];
  for (int i = 0; i < 3; ++i) alpha3[i] = EXT_ALPHA[k - 1][i];
}

/* Dense Cholesky H = L L^T (lower, row-major).  Returns 0 on success, -1 if
 * H is not positive definite. */
int oracle_cholesky(int64_t n, const double* H, double* L) {
  memset(L, 0, (size_t)(n * n) * sizeof(double));
  for (int64_t j = 0; j < n; ++j) {
    double d = H[j * n + j];
    for (int64_t m = 0; m < j; ++m) d -= L[j * n + m] * L[j * n + m];
    if (!(d > 0.0)) return -1;
    double ljj = sqrt(d);
    L[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = H[i * n + j];
      for (int64_t m = 0; m < j; ++m) s -= L[i * n + m] * L[j * n + m];
      L[i * n + j] = s / ljj;
    }
  }
  return 0;
}

/* Solve L L^T x = b by forward and back substitution. */
void oracle_cholesky_solve(int64_t n, const double* L, const double* b, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t m = 0; m < i; ++m) s -= L[i * n + m] * x[m];
    x[i] = s / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t m = i + 1; m < n; ++m) s -= L[m * n + i] * x[m];
    x[i] = s / L[i * n + i];
  }
}

/* The reduced model stepped by the oracle.  form: 0 = dense tensor C,
 * 1 = general CP factors (fa, fb, fc; n x rank), 2 = skew CP blocks
 * (fa = U, fb = V, fc = W; n x rank), 3 = SVD factors (fa = U, n x rank;
 * fb = sigma, rank; fc = V, n x rank x n), 4 = tensor including the zeroth
 * mode (C is n x (n+1) x (n+1)), 5 = CP factors including the zeroth mode
 * (fa n x rank, fb and fc (n+1) x rank).  A is n x n (dense), B is n x n or
 * NULL for the identity, L is n x n or NULL, f has n entries or is NULL. */
typedef struct {
  int64_t n;
  int form;
  int64_t rank;
  const double* C;
  const double* fa;
  const double* fb;
  const double* fc;
  const double* A;
  const double* B;
  const double* L;
  const double* f;
  double nu;
  double dt;
  int order;
} oracle_rom;

static void rom_nonlinear(const oracle_rom* m, const double* u, double* c) {
  if (m->form == 0)
    oracle_nonlinear_full(m->n, m->C, u, c);
  else if (m->form == 1)
    oracle_nonlinear_cp(m->n, m->rank, m->fa, m->fb, m->fc, u, c);
  else if (m->form == 2)
    oracle_nonlinear_cp_skew(m->n, m->rank, m->fa, m->fb, m->fc, u, c);
  else if (m->form == 3)
    oracle_nonlinear_svd(m->n, m->rank, m->fa, m->fb, m->fc, u, c);
  else if (m->form == 4)
    oracle_nonlinear_full_augmented(m->n, m->C, u, c);
  else
    oracle_nonlinear_cp_augmented(m->n, m->rank, m->fa, m->fb, m->fc, u, c);
}

static void matvec(int64_t n, const double* M, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += M[i * n + j] * x[j];
    y[i] = s;
  }
}

/*
 * Advance one trajectory by nsteps steps of eq. nse_d1.
 *
 * hist (in/out) holds 6n+1 doubles: u^l, u^{l-1}, u^{l-2}, n^l, n^{l-1},
 * n^{l-2} and the number of steps already taken (as a double).  n^l is the
 * advection term C(u^l)u^l of the newest state (recomputed here).  Step l
 * (0-based count of steps taken) uses order min(l+1, m->order): BDF1/EXT1,
 * then BDF2/EXT2, then BDFk/EXTk.  The right-hand side at time t^l is
 *   rhs = -sum_{i=1..k} alpha_i (n^{l+1-i} + L u^{l+1-i} + f) - B sum_{i=1..k} beta_i/dt u^{l+1-i}
 * and u^{l+1} solves (beta_0/dt B + nu A) u^{l+1} = rhs.
 *
 * energy (nullable, nsteps entries): E = 1/2 u^T B u of each new state.
 * invariant (nullable): u^T C(u) u of the state the step started from.
 * Returns 0, or -1 if a Cholesky factorisation fails.
 */
int oracle_rom_step(const oracle_rom* m, double* hist, int64_t nsteps, double* energy,
                    double* invariant) {
  int64_t n = m->n;
  double* u[3] = {hist, hist + n, hist + 2 * n};
  double* nl[3] = {hist + 3 * n, hist + 4 * n, hist + 5 * n};
  double* H = (double*)malloc((size_t)(n * n) * sizeof(double));
  double* Lc[3];
  int have[3] = {0, 0, 0};
  double* rhs = (double*)malloc((size_t)n * sizeof(double));
  double* tmp = (double*)malloc((size_t)n * sizeof(double));
  double* unew = (double*)malloc((size_t)n * sizeof(double));
  int rc = 0;
  for (int q = 0; q < 3; ++q) Lc[q] = (double*)malloc((size_t)(n * n) * sizeof(double));

  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t taken = (int64_t)hist[6 * n];
    int k = (int)(taken + 1 < m->order ? taken + 1 : m->order);
    double beta[4], alpha[3];
    oracle_bdf_ext_coefficients(k, beta, alpha);
    if (!have[k - 1]) {
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
          double b = m->B ? m->B[i * n + j] : (i == j ? 1.0 : 0.0);
          H[i * n + j] = beta[0] / m->dt * b + m->nu * m->A[i * n + j];
        }
      if (oracle_cholesky(n, H, Lc[k - 1]) != 0) { rc = -1; break; }
      have[k - 1] = 1;
    }
    /* advection term of the newest state */
    rom_nonlinear(m, u[0], nl[0]);
    if (invariant) {
      double t = 0.0;
      for (int64_t i = 0; i < n; ++i) t += u[0][i] * nl[0][i];
      invariant[s] = t;
    }
    /* rhs = -sum alpha_i (n + L u + f) */
    for (int64_t i = 0; i < n; ++i) rhs[i] = 0.0;
    for (int q = 0; q < k; ++q) {
      for (int64_t i = 0; i < n; ++i) rhs[i] -= alpha[q] * nl[q][i];
      if (m->L) {
        matvec(n, m->L, u[q], tmp);
        for (int64_t i = 0; i < n; ++i) rhs[i] -= alpha[q] * tmp[i];
      }
      if (m->f)
        for (int64_t i = 0; i < n; ++i) rhs[i] -= alpha[q] * m->f[i];
    }
    /* rhs -= B sum beta_i/dt u^{l+1-i} */
    for (int64_t i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int q = 0; q < k; ++q) acc += beta[q + 1] / m->dt * u[q][i];
      tmp[i] = acc;
    }
    if (m->B) {
      matvec(n, m->B, tmp, unew);
      for (int64_t i = 0; i < n; ++i) rhs[i] -= unew[i];
    } else {
      for (int64_t i = 0; i < n; ++i) rhs[i] -= tmp[i];
    }
    oracle_cholesky_solve(n, Lc[k - 1], rhs, unew);
    /* rotate the history */
    memcpy(u[2], u[1], (size_t)n * sizeof(double));
    memcpy(u[1], u[0], (size_t)n * sizeof(double));
    memcpy(u[0], unew, (size_t)n * sizeof(double));
    memcpy(nl[2], nl[1], (size_t)n * sizeof(double));
    memcpy(nl[1], nl[0], (size_t)n * sizeof(double));
    hist[6 * n] = (double)(taken + 1);
    if (energy) {
      double e = 0.0;
      if (m->B) {
        matvec(n, m->B, u[0], tmp);
        for (int64_t i = 0; i < n; ++i) e += u[0][i] * tmp[i];
      } else {
        for (int64_t i = 0; i < n; ++i) e += u[0][i] * u[0][i];
      }
      energy[s] = 0.5 * e;
    }
  }
  /* leave n^l consistent with the newest state */
  if (rc == 0) rom_nonlinear(m, u[0], nl[0]);
  for (int q = 0; q < 3; ++q) free(Lc[q]);
  free(H);
  free(rhs);
  free(tmp);
  free(unew);
  return rc;
}

/* Compression ratios and cost reduction of the CP model (Sec. 4, eq.
 * compress_ratio and the cost ratio below eq. tc_ap). */
double oracle_cr_als(int64_t n, int64_t r) { return (double)n * (double)n / (3.0 * (double)r); }
double oracle_cr_als_skew(int64_t n, int64_t r) { return 2.0 * (double)n * (double)n / (3.0 * (double)r); }
double oracle_cost_reduction(int64_t n, int64_t r) { return (double)n * (double)n / (3.0 * (double)r); }
/* Whole-solve speedup when a fraction `frac` of the time is the contraction
 * and its cost falls by `reduction`, the rest unchanged (Amdahl's law; the
 * "theoretical speedup" of Sec. 4.1.2-4.1.4). */
double oracle_amdahl_speedup(double frac, double reduction) { return 1.0 / ((1.0 - frac) + frac / reduction); }
/* Compression ratio of the SVD-ROM: N^3 / (N^2 R) (Sec. 4.4.2). */
double oracle_cr_svd(int64_t n, int64_t r) { return (double)n / (double)r; }
