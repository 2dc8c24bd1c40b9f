"""Seeded synthetic workloads shaped like the paper's ROM experiments.

This module is the single source of inputs for both sides of every parity
check (the FP64 CPU oracle and the GPU library) and for the benchmark.  It
contains no step of the method itself: it draws counter-based normals
(``synth.c``) and assembles the workload recipe of each configuration.

Recipes (base seed 20231106; workload c uses seed 20231106 + c):

* skew normal tensor (N=64 trajectory workload): C_ijk = S_ijk - S_kji with
  S_ijk = G_ijk / N, G standard normal on stream 1.  Exactly skew in the test
  index i and the advected index k (the partial skew-symmetry of Sec. 3.2).
* CP factors U, V, W (N x R): X_ir = z_ir * r^-1 / sqrt(R), r = 1..R, streams
  3, 4, 5.
* CP-structured tensor: C_ijk = sum_r V_jr (U_ir W_kr - W_ir U_kr) + E with
  E_ijk = s (G_ijk - G_kji), G on stream 2, and s chosen so that the expected
  Frobenius norm of E, s * sqrt(2 N^2 (N-1)), is 1e-3 times the exact
  Frobenius norm of the CP part.  The CP part is the paper's skew-preserving
  CP structure (Sec. 3.3, eq. skew_abc_struct) with A1 = U, A2 = W and the
  shared middle factor V.
* initial condition: u_i = z_i / i (i = 1..N), stream 6, index traj*N + i-1.
* operators: A = diag((i/N)^2), B = identity, nu = 1e-2, dt = 1e-3.
"""
import ctypes
import os
import subprocess

import numpy as np

BASE_SEED = 20231106
STREAM_S, STREAM_G, STREAM_U, STREAM_V, STREAM_W, STREAM_IC, STREAM_ARRIVAL = 1, 2, 3, 4, 5, 6, 7
STREAM_SVD_U, STREAM_SVD_V = 8, 9
STREAM_ZEROTH = 10

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lib = None


def build(force=False):
    """Compile synth.c into _synth.so (plain gcc, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64, i64, dbl, dp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
        lib.synth_normal.restype = dbl
        lib.synth_normal.argtypes = [u64, u64, u64]
        lib.synth_uniform.restype = dbl
        lib.synth_uniform.argtypes = [u64, u64, u64]
        lib.synth_draw_u64.restype = u64
        lib.synth_draw_u64.argtypes = [u64, u64, u64]
        lib.synth_fill_normal.restype = None
        lib.synth_fill_normal.argtypes = [u64, u64, u64, i64, dbl, dp]
        lib.synth_add_skew_normal_slab.restype = None
        lib.synth_add_skew_normal_slab.argtypes = [i64, u64, u64, dbl, i64, i64, dp]
        _lib = lib
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def seed_for(workload):
    return BASE_SEED + int(workload)


def normal(seed, stream, start, count, scale=1.0):
    out = np.empty(int(count), dtype=np.float64)
    _load().synth_fill_normal(seed, stream, int(start), int(count), float(scale), _ptr(out))
    return out


def uniform(seed, stream, ctr):
    return _load().synth_uniform(seed, stream, int(ctr))


def skew_normal_tensor(n, seed, i0=0, i1=None):
    """Rows i0..i1-1 of C_ijk = (G_ijk - G_kji)/n (shape (i1-i0, n, n))."""
    i1 = n if i1 is None else i1
    out = np.zeros((i1 - i0) * n * n, dtype=np.float64)
    _load().synth_add_skew_normal_slab(n, seed, STREAM_S, 1.0 / n, i0, i1, _ptr(out))
    return out.reshape(i1 - i0, n, n)


def cp_factors(n, rank, seed):
    """U, V, W (n x rank, row-major FP64) with column norms decaying as r^-1."""
    decay = 1.0 / (np.arange(1, rank + 1, dtype=np.float64) * np.sqrt(rank))
    out = []
    for stream in (STREAM_U, STREAM_V, STREAM_W):
        z = normal(seed, stream, 0, n * rank).reshape(n, rank)
        out.append(np.ascontiguousarray(z * decay[None, :]))
    return tuple(out)


def cp_part_frobenius(U, V, W):
    """Exact Frobenius norm of sum_r V_jr (U_ir W_kr - W_ir U_kr) from Gram matrices."""
    GU, GV, GW, GUW = U.T @ U, V.T @ V, W.T @ W, U.T @ W
    s = 2.0 * np.sum(GV * (GU * GW - GUW * GUW.T))
    return float(np.sqrt(max(s, 0.0)))


def residual_scale(n, cp_norm, rel=1e-3):
    return rel * cp_norm / np.sqrt(2.0 * n * n * (n - 1)) if n > 1 else 0.0


def cp_tensor(U, V, W, seed, resid_scale, i0=0, i1=None, block=16):
    """Rows i0..i1-1 of the CP-structured tensor plus the skew normal residual."""
    n, rank = U.shape
    i1 = n if i1 is None else i1
    out = np.empty((i1 - i0, n, n), dtype=np.float64)
    for b0 in range(i0, i1, block):
        b1 = min(i1, b0 + block)
        t1 = (U[b0:b1, None, :] * V[None, :, :]).reshape(-1, rank) @ W.T
        t2 = (W[b0:b1, None, :] * V[None, :, :]).reshape(-1, rank) @ U.T
        out[b0 - i0:b1 - i0] = (t1 - t2).reshape(b1 - b0, n, n)
    if resid_scale != 0.0:
        flat = out.reshape(-1)
        _load().synth_add_skew_normal_slab(n, seed, STREAM_G, float(resid_scale), i0, i1, _ptr(flat))
    return out


def svd_workload(n, rank, seed):
    """Seeded factors shaped like the SVD-ROM's (Sec. 4.4.2): U (n x rank,
    z / sqrt(n), stream 8), sigma_r = 1/r, and V (n x rank x n) whose slices
    V[:, r, :] = (G_r - G_r^T)/n are exactly skew (G from stream 9)."""
    U = normal(seed, STREAM_SVD_U, 0, n * rank).reshape(n, rank) / np.sqrt(n)
    sigma = 1.0 / np.arange(1, rank + 1, dtype=np.float64)
    G = normal(seed, STREAM_SVD_V, 0, n * rank * n).reshape(n, rank, n)
    V = (G - G.transpose(2, 1, 0)) / n
    return np.ascontiguousarray(U), sigma, np.ascontiguousarray(V)


def augment_tensor(C, seed):
    """Embeds a core tensor (n x n x n) into one that includes the zeroth mode
    (n x (n+1) x (n+1), index 0 = phi_0): the planes j = 0 and k = 0 get
    seeded normal entries / n (stream 10)."""
    n = C.shape[0]
    Cbar = np.zeros((n, n + 1, n + 1))
    Cbar[:, 1:, 1:] = C
    z = normal(seed, STREAM_ZEROTH, 0, n * (2 * n + 1)).reshape(n, 2 * n + 1) / n
    Cbar[:, 0, :] = z[:, : n + 1]
    Cbar[:, 1:, 0] = z[:, n + 1:]
    return Cbar


def augment_tensor_device(C, seed):
    """augment_tensor for a core tensor held on a torch device."""
    import torch

    n = C.shape[0]
    Cbar = torch.zeros((n, n + 1, n + 1), dtype=torch.float64, device=C.device)
    Cbar[:, 1:, 1:] = C
    z = torch.from_numpy(normal(seed, STREAM_ZEROTH, 0, n * (2 * n + 1)).reshape(n, 2 * n + 1) / n).to(C.device)
    Cbar[:, 0, :] = z[:, : n + 1]
    Cbar[:, 1:, 0] = z[:, n + 1:]
    return Cbar


def augment_cp(A, B, Cf, seed):
    """General CP factors including the zeroth mode: B and C get a leading
    row of seeded normal entries / sqrt(r) (stream 10)."""
    n, r = A.shape
    z = normal(seed, STREAM_ZEROTH, 0, 2 * r).reshape(2, r) / np.sqrt(r)
    return A, np.vstack([z[0], B]), np.vstack([z[1], Cf])


def initial_condition(n, seed, traj=0, count=1):
    """(count, n) initial states u_i = z_i / i for trajectories traj..traj+count-1."""
    z = normal(seed, STREAM_IC, traj * n, count * n).reshape(count, n)
    return z / np.arange(1, n + 1, dtype=np.float64)[None, :]


def diag_stiffness(n):
    i = np.arange(1, n + 1, dtype=np.float64)
    return (i / n) ** 2


def cp_workload(n, rank, workload):
    """Factors, residual scale and seed of the CP-structured workloads."""
    seed = seed_for(workload)
    U, V, W = cp_factors(n, rank, seed)
    return U, V, W, residual_scale(n, cp_part_frobenius(U, V, W)), seed


def arrivals(count, rate, seed, hmin=100, hmax=10000):
    """Poisson arrival times (s) and log-uniform integer horizons (steps)."""
    lib = _load()
    t, times, horizons, variant = 0.0, [], [], []
    for q in range(count):
        u1 = 1.0 - lib.synth_uniform(seed, STREAM_ARRIVAL, 4 * q)
        t += -np.log(u1) / rate
        times.append(t)
        u2 = lib.synth_uniform(seed, STREAM_ARRIVAL, 4 * q + 1)
        horizons.append(int(np.exp(np.log(hmin) + u2 * (np.log(hmax) - np.log(hmin)))))
        variant.append(lib.synth_draw_u64(seed, STREAM_ARRIVAL, 4 * q + 2))
    return np.array(times), np.array(horizons, dtype=np.int64), np.array(variant, dtype=np.uint64)


def cp_tensor_device(U, V, W, seed, resid_scale, device, block=64):
    """The CP-structured tensor assembled on a torch device (FP64).

    Same recipe as cp_tensor; the CP part is summed by the device's FP64
    matrix multiply, so entries agree with the host build to FP64 rounding of
    that sum.  Used for tensors too large to assemble quickly on the host.
    """
    import torch

    n, rank = U.shape
    Ud, Vd, Wd = (torch.from_numpy(np.ascontiguousarray(x)).to(device) for x in (U, V, W))
    C = torch.empty((n, n, n), dtype=torch.float64, device=device)
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        t1 = (Ud[b0:b1, None, :] * Vd[None]).reshape(-1, rank) @ Wd.T
        t2 = (Wd[b0:b1, None, :] * Vd[None]).reshape(-1, rank) @ Ud.T
        C[b0:b1] = (t1 - t2).reshape(b1 - b0, n, n)
        del t1, t2
    if resid_scale != 0.0:
        G = torch.from_numpy(normal(seed, STREAM_G, 0, n ** 3)).to(device).reshape(n, n, n)
        for b0 in range(0, n, block):
            b1 = min(n, b0 + block)
            C[b0:b1] += resid_scale * (G[b0:b1] - G[:, :, b0:b1].permute(2, 1, 0))
        del G
    return C
