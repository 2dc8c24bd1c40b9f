"""The skew-packed storage rule, checked on the host (no GPU).

Row (i, j) of the packed tensor keeps the entries k = (i + d) mod n for
d = 1 .. floor(n/2), except that for even n the distance n/2 is kept only in
rows with i < n/2.  For a tensor skew in i and k (Sec. 3.2, C_ijk = -C_kji)
this stores every unordered pair {i, k}, i != k, exactly once, and
  c_i = sum_j u_j [ sum_d P_{i,j,d} u_{i+d} - sum_d P_{i-d,j,d} u_{i-d} ]
(indices mod n) equals the dense contraction sum_jk C_ijk u_j u_k.
"""
import numpy as np
import pytest

import oracle
import synth


def kept(n):
    """(i, d) pairs the packed layout stores."""
    h = n // 2
    return [(i, d) for i in range(n) for d in range(1, h + 1) if not (n % 2 == 0 and d == h and i >= h)]


@pytest.mark.parametrize("n", list(range(1, 41)))
def test_each_unordered_pair_stored_once(n):
    seen = {}
    for i, d in kept(n):
        key = frozenset((i, (i + d) % n))
        assert len(key) == 2  # never the diagonal
        seen[key] = seen.get(key, 0) + 1
    assert len(seen) == n * (n - 1) // 2
    assert all(v == 1 for v in seen.values())


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 10, 13])
def test_packed_formula_equals_dense_contraction(n):
    seed = synth.seed_for(0) + 8000 + n
    C = synth.skew_normal_tensor(n, seed)
    u = synth.initial_condition(n, seed)[0]
    h = n // 2
    P = np.zeros((n, n, max(h, 1)))
    for i, d in kept(n):
        P[i, :, d - 1] = C[i, :, (i + d) % n]
    c = np.zeros(n)
    for i, d in kept(n):
        k = (i + d) % n
        D = P[i, :, d - 1] @ u  # D_ik = sum_j u_j C_ijk
        c[i] += D * u[k]
        c[k] -= D * u[i]  # D_ki = -D_ik
    ref = oracle.nonlinear_full(C, u)
    assert np.allclose(c, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


def _packed(C):
    """P[i][j][p] = C[i][j][(i+1+p) mod n] on the kept distances, zero elsewhere."""
    n = C.shape[0]
    h = n // 2
    P = np.zeros((n, n, max(h, 1)))
    for i, d in kept(n):
        P[i, :, d - 1] = C[i, :, (i + d) % n]
    return P


@pytest.mark.parametrize("n", [2, 3, 8, 11, 16])
@pytest.mark.parametrize("batch", [1, 3])
def test_factored_form_equals_dense_contraction(n, batch):
    # the factored batched form on the packed layout: one product
    # D_i[p, b] = sum_j P[i][j][p] u_bj per test index feeds both entries of
    # every stored pair, c_i += D_i u_{b,k} and c_k -= D_i u_{b,i},
    # k = (i+1+p) mod n
    seed = synth.seed_for(0) + 8700 + n
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, batch)
    P = _packed(C)
    c = np.zeros((batch, n))
    for i in range(n):
        D = np.einsum("jp,bj->pb", P[i], U)
        for p in range(P.shape[2]):
            k = (i + 1 + p) % n
            c[:, i] += D[p] * U[:, k]
            c[:, k] -= D[p] * U[:, i]
    for b in range(batch):
        np.testing.assert_allclose(c[b], oracle.nonlinear_full(C, U[b]), rtol=1e-12, atol=1e-13)
        # both entries of a pair use the same D: u^T c vanishes to rounding
        assert abs(U[b] @ c[b]) <= 1e-13 * np.abs(U[b]) @ np.abs(c[b]) + 1e-15


@pytest.mark.parametrize("n,r", [(7, 3), (12, 5)])
def test_stacked_cp_factors_equal_the_cp_oracle(n, r):
    # the batched CP form on the tensor cores stacks the projections and the
    # expansion: [P; Q; S] = [V W U]^T u, c = [U, -W] [P o Q; P o S]
    # (general: [P; Q] = [B C]^T u, c = A (P o Q))
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    u = synth.initial_condition(n, seed)[0]
    PQS = np.vstack([V.T, W.T, U.T]) @ u
    P, Q, S = PQS[:r], PQS[r:2 * r], PQS[2 * r:]
    c = np.hstack([U, -W]) @ np.concatenate([P * Q, P * S])
    np.testing.assert_allclose(c, oracle.nonlinear_cp_skew(U, V, W, u), rtol=1e-12, atol=1e-14)
    A, B, Cf = U, V, W
    PQ = np.vstack([B.T, Cf.T]) @ u
    c = A @ (PQ[:r] * PQ[r:])
    np.testing.assert_allclose(c, oracle.nonlinear_cp(A, B, Cf, u), rtol=1e-12, atol=1e-14)
