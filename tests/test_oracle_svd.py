"""Pins of the oracle's SVD-ROM (Sec. 4.4.2) on the CPU.

The SVD-ROM approximates the tensor's matricization over the advecting index
by its truncated SVD, C_ijk ~ sum_r U_jr sigma_r V[i][r][k], and evaluates
c_i = sum_r sigma_r (U^T u)_r sum_k V[i][r][k] u_k.  The pins: full rank
reproduces the dense contraction; the factored evaluation equals the
contraction of the reconstructed tensor (an independent einsum); a rank-one
tensor has a closed-form SVD; the singular values carry the Frobenius norm
and the truncation error (orthogonality of the SVD); skew tensors give skew
slices and a vanishing invariant; a planted layout mistake fails.
"""
import numpy as np
import pytest

import oracle
import synth


def _skew(n, seed):
    return synth.skew_normal_tensor(n, seed)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [3, 6, 9])
def test_full_rank_reproduces_dense_contraction(n):
    C = _skew(n, synth.seed_for(0) + 100 + n)
    u = synth.initial_condition(n, 5)[0]
    U, s, V = oracle.svd_factors(C, n)
    assert _rel(oracle.nonlinear_svd(U, s, V, u), oracle.nonlinear_full(C, u)) < 1e-12


@pytest.mark.parametrize("n,r", [(4, 1), (5, 3), (8, 8), (7, 11)])
def test_factored_evaluation_equals_reconstructed_contraction(n, r):
    rng = np.random.default_rng(n * 31 + r)
    U, s, V = rng.standard_normal((n, r)), rng.random(r) + 0.1, rng.standard_normal((n, r, n))
    u = rng.standard_normal(n)
    X = np.einsum("jm,m,imk->ijk", U, s, V)
    ref = np.einsum("ijk,j,k->i", X, u, u)
    assert _rel(oracle.nonlinear_svd(U, s, V, u), ref) < 1e-13


def test_rank_one_closed_form():
    n = 6
    rng = np.random.default_rng(3)
    a = rng.standard_normal(n)
    G = rng.standard_normal((n, n))
    M = G - G.T
    C = np.einsum("j,ik->ijk", a, M)  # C_ijk = a_j M_ik, skew in (i, k)
    U, s, V = oracle.svd_factors(C, n)
    assert s[0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(M), rel=1e-13)
    assert np.all(s[1:] < 1e-13 * s[0])
    u = rng.standard_normal(n)
    c1 = oracle.nonlinear_svd(U[:, :1], s[:1], V[:, :1, :], u)
    assert _rel(c1, (a @ u) * (M @ u)) < 1e-13


@pytest.mark.parametrize("n", [5, 8])
def test_singular_values_carry_norm_and_truncation_error(n):
    C = _skew(n, synth.seed_for(0) + 200 + n)
    U, s, V = oracle.svd_factors(C, n)
    assert np.sum(s ** 2) == pytest.approx(np.sum(C ** 2), rel=1e-13)
    for r in (1, n // 2, n - 1):
        X = oracle.svd_reconstruct(U[:, :r], s[:r], V[:, :r, :])
        assert np.sum((C - X) ** 2) == pytest.approx(np.sum(s[r:] ** 2), rel=1e-10, abs=1e-28)


def test_skew_tensor_gives_skew_slices_and_zero_invariant():
    n, r = 8, 5
    C = _skew(n, synth.seed_for(0) + 300)
    U, s, V = oracle.svd_factors(C, r)
    for m in range(r):
        assert np.max(np.abs(V[:, m, :] + V[:, m, :].T)) < 1e-13
    u = synth.initial_condition(n, 9)[0]
    c = oracle.nonlinear_svd(U, s, V, u)
    assert abs(u @ c) < 1e-14 * np.linalg.norm(u) * np.linalg.norm(c) * n


def test_planted_layout_mistake_is_caught():
    # reading V as V[k][r][i] (test and advected index swapped) must break
    # the full-rank reproduction
    n = 6
    C = _skew(n, synth.seed_for(0) + 400)
    u = synth.initial_condition(n, 2)[0]
    U, s, V = oracle.svd_factors(C, n)
    wrong = np.ascontiguousarray(V.transpose(2, 1, 0))
    assert _rel(oracle.nonlinear_svd(U, s, wrong, u), oracle.nonlinear_full(C, u)) > 0.5


def test_compression_ratio_formula():
    # CR_SVD = N^3 / (N^2 R) = N / R (Sec. 4.4.2)
    for n, r in ((64, 8), (1024, 16), (100, 3)):
        assert oracle.cr_svd(n, r) == pytest.approx(n ** 3 / (n ** 2 * r))


def test_full_rank_svd_rom_trajectory_equals_g_rom():
    n, steps = 6, 30
    C = _skew(n, synth.seed_for(0) + 500)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, 4)[0]
    full = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
    svd = oracle.Rom("svd", n, a, 1e-2, 1e-3, factors=oracle.svd_factors(C, n))
    hf, hs = full.initial_history(u0), svd.initial_history(u0)
    full.step(hf, steps)
    svd.step(hs, steps)
    assert _rel(hs[:n], hf[:n]) < 1e-12
