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
