"""Pins of the oracle's CP contraction (Sec. 3.1, eq. tc_ap) and of the skew
CP structure (Sec. 3.3, eq. skew_abc_struct)."""
import numpy as np
import pytest

import oracle
import synth


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_reconstruct_matches_einsum(rng):
    n, r = 5, 4
    A, B, Cf = (rng.standard_normal((n, r)) for _ in range(3))
    X = oracle.cp_reconstruct(A, B, Cf)
    assert _rel(X, np.einsum("ir,jr,kr->ijk", A, B, Cf)) < 1e-14


@pytest.mark.parametrize("n,r", [(1, 1), (3, 2), (5, 6), (8, 3)])
def test_cp_equals_contraction_of_reconstruction(n, r, rng):
    # eq. tc_ap: contracting the CP sum equals contracting the tensor it builds.
    A, B, Cf = (rng.standard_normal((n, r)) for _ in range(3))
    u = rng.standard_normal(n)
    brute = oracle.nonlinear_full(oracle.cp_reconstruct(A, B, Cf), u)
    assert _rel(oracle.nonlinear_cp(A, B, Cf, u), brute) < 1e-13


def test_cp_closed_form(rng):
    n, r = 6, 4
    A, B, Cf = (rng.standard_normal((n, r)) for _ in range(3))
    u = rng.standard_normal(n)
    assert _rel(oracle.nonlinear_cp(A, B, Cf, u), A @ ((B.T @ u) * (Cf.T @ u))) < 1e-14


def test_skew_structure_reconstructs_skew_tensor(rng):
    # eq. skewsym_condition: [[A1, A2, A3]] = [[-A3, A2, A1]], i.e. X_ijk = -X_kji.
    n, r = 6, 3
    U, V, W = (rng.standard_normal((n, r)) for _ in range(3))
    A1, A2, A3 = oracle.cp_skew_expand(U, V, W)
    X = oracle.cp_reconstruct(A1, A2, A3)
    assert np.max(np.abs(X + X.transpose(2, 1, 0))) <= 1e-14 * np.max(np.abs(X))
    assert _rel(X, oracle.cp_reconstruct(-A3, A2, A1)) < 1e-14
    # and A2 has the repeated block, A3 = [W, -U]
    np.testing.assert_array_equal(A2[:, :r], A2[:, r:])
    np.testing.assert_array_equal(A3[:, r:], -U)


def test_skew_cp_closed_form_and_invariant(rng):
    n, r = 7, 5
    U, V, W = (rng.standard_normal((n, r)) for _ in range(3))
    u = rng.standard_normal(n)
    p, q, s = V.T @ u, W.T @ u, U.T @ u
    c = oracle.nonlinear_cp_skew(U, V, W, u)
    assert _rel(c, U @ (p * q) - W @ (p * s)) < 1e-13
    A1, A2, A3 = oracle.cp_skew_expand(U, V, W)
    brute = oracle.nonlinear_full(oracle.cp_reconstruct(A1, A2, A3), u)
    assert _rel(c, brute) < 1e-13
    assert abs(u @ c) < 1e-13 * np.sum(np.abs(u)) * np.sum(np.abs(U @ (p * q)) + np.abs(W @ (p * s)))


def test_generator_cp_tensor_matches_oracle_reconstruction():
    # Two independent builds of the CP-structured workload tensor agree.
    n, r = 9, 4
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    T = synth.cp_tensor(U, V, W, seed, 0.0)
    X = oracle.cp_reconstruct(*oracle.cp_skew_expand(U, V, W))
    assert _rel(T, X) < 1e-14
    # the residual is exactly skew and has the requested relative size
    U, V, W, s, seed = synth.cp_workload(32, 8, 1)
    full = synth.cp_tensor(U, V, W, seed, s)
    part = synth.cp_tensor(U, V, W, seed, 0.0)
    E = full - part
    assert abs(np.linalg.norm(E) / np.linalg.norm(part) - 1e-3) < 1e-4
    assert np.max(np.abs(E + E.transpose(2, 1, 0))) < 1e-15 * np.max(np.abs(full))
    assert np.max(np.abs(full + full.transpose(2, 1, 0))) < 1e-15 * np.max(np.abs(full))
