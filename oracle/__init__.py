"""FP64 CPU oracle for the Galerkin ROM advection term (arXiv 2311.03694).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the GPU library; the
library itself never imports, links or calls it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain loops in FP64); this module only
compiles it with gcc and marshals numpy arrays.  Functions and the paper
passage each one follows:

* ``nonlinear_full``      c_i = sum_jk C_ijk u_j u_k          Sec. 2.2, eq. Cu, eq. nse_ode
* ``nonlinear_cp``        c = A((B^T u) o (C^T u))            Sec. 3.1, eq. tc_ap
* ``cp_skew_expand``      A1=[U W], A2=[V V], A3=[W -U]       Sec. 3.3, eq. skew_abc_struct
* ``nonlinear_cp_skew``   eq. tc_ap on the expanded factors
* ``cp_reconstruct``      Kruskal operator                    Sec. 2.3, eq. cpd
* ``rom_step``            BDFk/EXTk step with cached Cholesky Sec. 2.2, eq. nse_d1
* ``cr_als``, ``cr_als_skew``, ``cost_reduction``              Sec. 4, eq. compress_ratio; Sec. 3.1
* ``amdahl_speedup``      1 / ((1 - f) + f / reduction)         Sec. 4.1.2-4.1.4 (theoretical speedup)

Index convention: C[i, j, k] with i the test index, j the advecting index
and k the advected index.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into _oracle.so (gcc -O2, OpenMP over the test index)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Rom(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("form", ctypes.c_int), ("rank", ctypes.c_int64),
        ("C", ctypes.c_void_p), ("fa", ctypes.c_void_p), ("fb", ctypes.c_void_p),
        ("fc", ctypes.c_void_p), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
        ("L", ctypes.c_void_p), ("f", ctypes.c_void_p), ("nu", ctypes.c_double),
        ("dt", ctypes.c_double), ("order", ctypes.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, vp, dbl = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
        for name, args in {
            "oracle_nonlinear_full_rows": [i64, i64, i64, vp, vp, vp],
            "oracle_nonlinear_full": [i64, vp, vp, vp],
            "oracle_nonlinear_cp": [i64, i64, vp, vp, vp, vp, vp],
            "oracle_nonlinear_cp_skew": [i64, i64, vp, vp, vp, vp, vp],
            "oracle_cp_skew_expand": [i64, i64, vp, vp, vp, vp, vp, vp],
            "oracle_cp_reconstruct": [i64, i64, vp, vp, vp, vp],
            "oracle_nonlinear_svd": [i64, i64, vp, vp, vp, vp, vp],
            "oracle_nonlinear_full_augmented": [i64, vp, vp, vp],
            "oracle_nonlinear_cp_augmented": [i64, i64, vp, vp, vp, vp, vp],
            "oracle_bdf_ext_coefficients": [ctypes.c_int, vp, vp],
            "oracle_cholesky_solve": [i64, vp, vp, vp],
            "oracle_set_threads": [ctypes.c_int],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = None
        lib.oracle_cholesky.argtypes = [i64, vp, vp]
        lib.oracle_cholesky.restype = ctypes.c_int
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = ctypes.c_int
        lib.oracle_rom_step.argtypes = [ctypes.POINTER(_Rom), vp, i64, vp, vp]
        lib.oracle_rom_step.restype = ctypes.c_int
        for name in ("oracle_cr_als", "oracle_cr_als_skew", "oracle_cost_reduction", "oracle_cr_svd"):
            fn = getattr(lib, name)
            fn.argtypes = [i64, i64]
            fn.restype = dbl
        lib.oracle_amdahl_speedup.argtypes = [dbl, dbl]
        lib.oracle_amdahl_speedup.restype = dbl
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data


def set_threads(t):
    _load().oracle_set_threads(int(t))


def get_threads():
    return _load().oracle_get_threads()


def nonlinear_full(C, u):
    C, u = _f64(C), _f64(u)
    n = u.shape[-1]
    assert C.size == n ** 3
    c = np.empty(n)
    _load().oracle_nonlinear_full(n, _p(C), _p(u), _p(c))
    return c


def nonlinear_full_rows(C_rows, i0, u):
    """c_i for the rows i0..i0+len(C_rows)-1, given only those tensor rows."""
    C_rows, u = _f64(C_rows), _f64(u)
    n = u.shape[-1]
    rows = C_rows.size // (n * n)
    c = np.empty(rows)
    _load().oracle_nonlinear_full_rows(n, i0, i0 + rows, _p(C_rows), _p(u), _p(c))
    return c


def nonlinear_cp(A, B, Cf, u):
    A, B, Cf, u = _f64(A), _f64(B), _f64(Cf), _f64(u)
    n, r = A.shape
    c = np.empty(n)
    _load().oracle_nonlinear_cp(n, r, _p(A), _p(B), _p(Cf), _p(u), _p(c))
    return c


def nonlinear_cp_skew(U, V, W, u):
    U, V, W, u = _f64(U), _f64(V), _f64(W), _f64(u)
    n, r = U.shape
    c = np.empty(n)
    _load().oracle_nonlinear_cp_skew(n, r, _p(U), _p(V), _p(W), _p(u), _p(c))
    return c


def cp_skew_expand(U, V, W):
    U, V, W = _f64(U), _f64(V), _f64(W)
    n, r = U.shape
    A1, A2, A3 = (np.empty((n, 2 * r)) for _ in range(3))
    _load().oracle_cp_skew_expand(n, r, _p(U), _p(V), _p(W), _p(A1), _p(A2), _p(A3))
    return A1, A2, A3


def cp_reconstruct(A, B, Cf):
    A, B, Cf = _f64(A), _f64(B), _f64(Cf)
    n, r = A.shape
    X = np.empty((n, n, n))
    _load().oracle_cp_reconstruct(n, r, _p(A), _p(B), _p(Cf), _p(X))
    return X


def nonlinear_svd(U, sigma, V, u):
    """SVD-ROM advection term (Sec. 4.4.2): c_i = sum_r sigma_r (U^T u)_r sum_k V[i][r][k] u_k.

    U is n x r, sigma has r entries, V is n x r x n (V[i][r][k])."""
    U, sigma, V, u = _f64(U), _f64(sigma), _f64(V), _f64(u)
    n, r = U.shape
    assert sigma.shape == (r,) and V.shape == (n, r, n)
    c = np.empty(n)
    _load().oracle_nonlinear_svd(n, r, _p(U), _p(sigma), _p(V), _p(u), _p(c))
    return c


def nonlinear_full_augmented(Cbar, u):
    """c_i = sum_{j,k=0..n} Cbar_ijk ubar_j ubar_k, ubar = (1, u); Cbar is
    n x (n+1) x (n+1) with index 0 the zeroth mode (Sec. 4.2)."""
    Cbar, u = _f64(Cbar), _f64(u)
    n = u.size
    assert Cbar.shape == (n, n + 1, n + 1)
    c = np.empty(n)
    _load().oracle_nonlinear_full_augmented(n, _p(Cbar), _p(u), _p(c))
    return c


def nonlinear_cp_augmented(A, Bbar, Cbar, u):
    """CP contraction with ubar = (1, u): A is n x r, Bbar and Cbar (n+1) x r."""
    A, Bbar, Cbar, u = _f64(A), _f64(Bbar), _f64(Cbar), _f64(u)
    n, r = A.shape
    assert Bbar.shape == (n + 1, r) and Cbar.shape == (n + 1, r)
    c = np.empty(n)
    _load().oracle_nonlinear_cp_augmented(n, r, _p(A), _p(Bbar), _p(Cbar), _p(u), _p(c))
    return c


def advecting_matricization(C):
    """The tensor unfolded over its advecting index: row j holds the n x n
    matrix (i, k) -> C_ijk, flattened row-major (Sec. 4.4.1)."""
    n = C.shape[0]
    return np.ascontiguousarray(np.transpose(_f64(C), (1, 0, 2)).reshape(n, n * n))


def svd_factors(C, r):
    """Rank-r truncated SVD of the advecting-index matricization (numpy's SVD
    as the library step), returned as (U, sigma, V) with V[i][m][k] the
    right singular vector m read as an n x n matrix over (i, k)."""
    n = C.shape[0]
    Um, s, Vt = np.linalg.svd(advecting_matricization(C), full_matrices=False)
    V = np.ascontiguousarray(Vt[:r].reshape(r, n, n).transpose(1, 0, 2))
    return np.ascontiguousarray(Um[:, :r]), np.ascontiguousarray(s[:r]), V


def svd_reconstruct(U, sigma, V):
    """C_ijk = sum_m U_jm sigma_m V[i][m][k] (plain loops over the rank)."""
    U, sigma, V = _f64(U), _f64(sigma), _f64(V)
    n, r = U.shape
    X = np.zeros((n, n, n))
    for m in range(r):
        X += sigma[m] * U[None, :, m, None] * V[:, None, m, :]
    return X


# ------------------------------------------------------------ CP fitting
def kr(P, Q):
    """Khatri-Rao product: column r is kron(P[:, r], Q[:, r]), rows (a, b)
    with the second index fastest."""
    return np.einsum("ar,br->abr", _f64(P), _f64(Q)).reshape(P.shape[0] * Q.shape[0], P.shape[1])


def mttkrp(X, factors, mode):
    """X_(mode) times the Khatri-Rao product of the other two factors (mode
    0, 1, 2 = first, second, third index), the right-hand side of the ALS
    normal equations (Sec. 2.3)."""
    A1, A2, A3 = factors
    if mode == 0:
        return _f64(X).reshape(X.shape[0], -1) @ kr(A2, A3)
    if mode == 1:
        return np.transpose(_f64(X), (1, 0, 2)).reshape(X.shape[1], -1) @ kr(A1, A3)
    return np.transpose(_f64(X), (2, 0, 1)).reshape(X.shape[2], -1) @ kr(A1, A2)


def gram_hadamard(factors, mode):
    """Hadamard product of the Gram matrices of the two factors other than mode."""
    G = np.ones((factors[0].shape[1],) * 2)
    for q, F in enumerate(factors):
        if q != mode:
            G = G * (F.T @ F)
    return G


def spd_solve(H, B):
    """H^-1 B for the symmetric positive (semi)definite H through its Cholesky
    factor; a numerically singular H is retried with H + mu I, mu = 1e-12
    max diag(H), growing 100x up to three times (the paper is silent on
    singular normal equations)."""
    mu = 0.0
    for _ in range(4):
        try:
            L = np.linalg.cholesky(H + mu * np.eye(H.shape[0]))
            return np.linalg.solve(L.T, np.linalg.solve(L, B))
        except np.linalg.LinAlgError:
            mu = 1e-12 * np.max(np.diag(H)) if mu == 0.0 else mu * 100.0
    raise np.linalg.LinAlgError("Gram matrix is not positive definite")


def als_update(X, factors, mode, ridge=0.0):
    """Exact solution of the mode's linear least-squares subproblem of eq.
    cp_als through its normal equations, A = MTTKRP (Hadamard of Grams)^-1;
    ridge > 0 adds ridge * max diag to the normal matrix (Tikhonov)."""
    M = mttkrp(X, factors, mode)
    H = gram_hadamard(factors, mode)
    H = H + ridge * np.max(np.diag(H)) * np.eye(H.shape[0])
    return spd_solve(H, M.T).T


def cp_residual(X, factors):
    """Relative residual ||X - [[A1, A2, A3]]||_F / ||X||_F (eq. cp_nls)."""
    return float(np.linalg.norm(X - np.einsum("ir,jr,kr->ijk", *factors)) / np.linalg.norm(X))


def cp_als(X, factors, iters, ridge=0.0):
    """Plain ALS (Sec. 2.3, eq. cp_als): each iteration solves the three
    subproblems in sequence.  Returns the factors and the relative residual
    after every iteration."""
    F = [_f64(f).copy() for f in factors]
    res = []
    for _ in range(iters):
        for mode in range(3):
            F[mode] = als_update(X, F, mode, ridge)
        res.append(cp_residual(X, F))
    return F, res


def skew_structure(A1, B1):
    """Skew-preserving factors (eq. skew_abc_struct) from the blocks: A1 = [A1_1 A1_2]
    (n x R), A2 = [B1 B1], A3 = [A1_2, -A1_1]."""
    h = A1.shape[1] // 2
    return [A1, np.hstack([B1, B1]), np.hstack([A1[:, h:], -A1[:, :h]])]


def cp_als_skew(X, A1, B1, iters, lam=0.5, subiters=1, ridge=0.0):
    """ALS-skew (Sec. 3.3): A2 = [B1 B1] is updated as in ALS (its two halves,
    equal for a skew X, are averaged); A1 takes `subiters` least-squares
    subiterations of eq. cp_als_quad with A3 fixed, each followed by the
    momentum update A1 <- lam A1 + (1 - lam) A1_next and A3 = [A1_2, -A1_1].
    Returns (A1, B1) and the relative residual after every iteration."""
    A1, B1 = _f64(A1).copy(), _f64(B1).copy()
    h = A1.shape[1] // 2
    res = []
    for _ in range(iters):
        F = skew_structure(A1, B1)
        A2 = als_update(X, F, 1, ridge)
        B1 = 0.5 * (A2[:, :h] + A2[:, h:])
        for _ in range(subiters):
            F = skew_structure(A1, B1)
            A1 = lam * A1 + (1.0 - lam) * als_update(X, F, 0, ridge)
        res.append(cp_residual(X, skew_structure(A1, B1)))
    return (A1, B1), res


def bdf_ext_coefficients(k):
    beta, alpha = np.empty(4), np.empty(3)
    _load().oracle_bdf_ext_coefficients(int(k), _p(beta), _p(alpha))
    return beta, alpha


def cholesky(H):
    H = _f64(H)
    n = H.shape[0]
    L = np.empty((n, n))
    if _load().oracle_cholesky(n, _p(H), _p(L)) != 0:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    return L


def cholesky_solve(L, b):
    L, b = _f64(L), _f64(b)
    x = np.empty(L.shape[0])
    _load().oracle_cholesky_solve(L.shape[0], _p(L), _p(b), _p(x))
    return x


class Rom:
    """A reduced model for the oracle stepper.

    form: "full" (C is n x n x n), "cp" (factors A, B, Cf, each n x r),
    "cp_skew" (blocks U, V, W, each n x r), "svd" (factors U (n x r),
    sigma (r), V (n x r x n)), "full_aug" (C is n x (n+1) x (n+1), index 0 the
    zeroth mode) or "cp_aug" (A n x r, B and C (n+1) x r).  A is the stiffness matrix (n x n,
    or a length-n diagonal), B the mass matrix (None = identity), L an
    optional explicit linear operator and f an optional constant forcing.
    """

    FORMS = {"full": 0, "cp": 1, "cp_skew": 2, "svd": 3, "full_aug": 4, "cp_aug": 5}

    def __init__(self, form, n, A, nu, dt, order=3, C=None, factors=None, B=None, L=None, f=None):
        self.n = int(n)
        self._keep = []
        Ad = _f64(A)
        if Ad.ndim == 1:
            Ad = np.diag(Ad)
        s = _Rom()
        s.n, s.form, s.nu, s.dt, s.order = self.n, self.FORMS[form], float(nu), float(dt), int(order)
        s.rank = 0
        s.A = self._hold(Ad)
        s.B = self._hold(None if B is None else _f64(B))
        s.L = self._hold(None if L is None else (np.diag(_f64(L)) if np.ndim(L) == 1 else _f64(L)))
        s.f = self._hold(None if f is None else _f64(f))
        s.C = self._hold(None if C is None else _f64(C))
        if factors is not None:
            fa, fb, fc = (_f64(x) for x in factors)
            s.rank = fa.shape[1]
            s.fa, s.fb, s.fc = self._hold(fa), self._hold(fb), self._hold(fc)
        self._s = s

    def _hold(self, a):
        if a is None:
            return None
        self._keep.append(a)
        return a.ctypes.data

    def initial_history(self, u0):
        h = np.zeros(6 * self.n + 1)
        h[: self.n] = u0
        return h

    def step(self, hist, nsteps, want_energy=False, want_invariant=False):
        """Advance hist (6n+1 doubles, modified in place) by nsteps steps."""
        assert hist.dtype == np.float64 and hist.size == 6 * self.n + 1 and hist.flags.c_contiguous
        e = np.empty(nsteps) if want_energy else None
        inv = np.empty(nsteps) if want_invariant else None
        rc = _load().oracle_rom_step(ctypes.byref(self._s), _p(hist), int(nsteps), _p(e), _p(inv))
        if rc != 0:
            raise np.linalg.LinAlgError("reduced operator is not positive definite")
        return e, inv


def cr_als(n, r):
    return _load().oracle_cr_als(n, r)


def cr_als_skew(n, r):
    return _load().oracle_cr_als_skew(n, r)


def cr_svd(n, r):
    return _load().oracle_cr_svd(n, r)


def cost_reduction(n, r):
    return _load().oracle_cost_reduction(n, r)


def amdahl_speedup(frac, reduction):
    return _load().oracle_amdahl_speedup(float(frac), float(reduction))
