"""Pins of the oracle's CP fitting (Sec. 2.3 ALS, eq. cp_als; Sec. 3.3
ALS-skew, eq. skew_abc_struct / cp_als_quad).

Each ALS subproblem is a linear least-squares problem: the normal-equation
update must equal numpy's least-squares solution of the unfolded problem; an
exact rank-R tensor is a fixed point and is recovered from a nearby start;
plain ALS never increases the residual; ALS-skew keeps the skew structure
and its fitted tensor is exactly skew; a planted Khatri-Rao ordering mistake
breaks the least-squares identity.
"""
import numpy as np
import pytest

import oracle


def _cp(n, r, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n, r)) for _ in range(3)]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_update_is_the_least_squares_solution(mode):
    rng = np.random.default_rng(1 + mode)
    n, r = 6, 3
    X = rng.standard_normal((n, n, n))
    F = _cp(n, r, 2)
    # the subproblem written as lstsq on the unfolding: X_(mode) ~ B K^T
    others = [F[q] for q in range(3) if q != mode]
    K = np.einsum("ar,br->abr", *others).reshape(n * n, r)
    unf = np.moveaxis(X, mode, 0).reshape(n, n * n)
    B_ref = np.linalg.lstsq(K, unf.T, rcond=None)[0].T
    np.testing.assert_allclose(oracle.als_update(X, F, mode), B_ref, rtol=1e-9, atol=1e-11)


def test_exact_tensor_is_fixed_point_and_recovered():
    n, r = 7, 3
    F0 = _cp(n, r, 5)
    X = np.einsum("ir,jr,kr->ijk", *F0)
    F, res = oracle.cp_als(X, F0, 1)
    assert res[-1] < 1e-12
    rng = np.random.default_rng(6)
    start = [f + 1e-2 * rng.standard_normal(f.shape) for f in F0]
    F, res = oracle.cp_als(X, start, 30)
    assert res[-1] < 1e-9


def test_plain_als_residual_is_monotone():
    rng = np.random.default_rng(7)
    n, r = 8, 4
    X = rng.standard_normal((n, n, n))
    _, res = oracle.cp_als(X, _cp(n, r, 8), 15)
    assert all(b <= a + 1e-12 for a, b in zip(res, res[1:]))


def test_als_skew_keeps_structure_and_skew_fit():
    n, r = 8, 6
    rng = np.random.default_rng(9)
    S = rng.standard_normal((n, n, n))
    X = S - S.transpose(2, 1, 0)
    A1, B1 = rng.standard_normal((n, r)), rng.standard_normal((n, r // 2))
    (A1, B1), res = oracle.cp_als_skew(X, A1, B1, 10)
    F = oracle.skew_structure(A1, B1)
    Y = np.einsum("ir,jr,kr->ijk", *F)
    assert np.max(np.abs(Y + Y.transpose(2, 1, 0))) < 1e-12 * np.max(np.abs(Y))
    assert res[-1] < res[0]
    # for a skew tensor the unconstrained mode-2 update already has equal halves
    A2 = oracle.als_update(X, F, 1)
    np.testing.assert_allclose(A2[:, : r // 2], A2[:, r // 2:], rtol=1e-8, atol=1e-10)


def test_als_skew_recovers_exact_skew_cp_tensor():
    n, h = 7, 2
    rng = np.random.default_rng(10)
    A1s, B1s = rng.standard_normal((n, 2 * h)), rng.standard_normal((n, h))
    X = np.einsum("ir,jr,kr->ijk", *oracle.skew_structure(A1s, B1s))
    # the exact factors are a fixed point
    _, res = oracle.cp_als_skew(X, A1s, B1s, 3)
    assert max(res) < 1e-13
    # from a nearby start the residual falls steadily (ALS near an exact fit
    # converges slowly)
    start_A = A1s + 1e-3 * rng.standard_normal(A1s.shape)
    start_B = B1s + 1e-3 * rng.standard_normal(B1s.shape)
    _, res = oracle.cp_als_skew(X, start_A, start_B, 60)
    assert res[-1] < 0.05 * res[0] and res[-1] < 2e-5


def test_planted_khatri_rao_order_mistake_is_caught():
    n, r = 5, 2
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, n, n))
    F = _cp(n, r, 12)
    good = oracle.mttkrp(X, F, 0)
    wrong = X.reshape(n, -1) @ oracle.kr(F[2], F[1])  # factors in the wrong order
    assert np.linalg.norm(good - wrong) > 0.1 * np.linalg.norm(good)
