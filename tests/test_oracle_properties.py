"""Property checks of the oracle over random sizes and seeds (CPU only).

Complements the fixed-size pins: for any size and seed the oracle must keep
the invariants the paper's structure implies (Sec. 3.2: u^T C(u)u = 0 for a
skew tensor; Sec. 3.3: the skew CP structure equals its expanded rank-2R
general form), the contraction must be quadratic in u, and the BDFk/EXTk
coefficient tables must be consistent (sum beta = 0, sum alpha = 1) and exact
on polynomials of their order."""
import numpy as np
import pytest

import oracle
import synth

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None, derandomize=True)  # the same examples every run


@SETTINGS
@given(n=st.integers(1, 14), seed=st.integers(0, 2**31 - 1))
def test_skew_invariant_any_size(n, seed):
    C = synth.skew_normal_tensor(n, seed)
    u = synth.initial_condition(n, seed)[0]
    c = oracle.nonlinear_full(C, u)
    scale = np.abs(u) @ np.einsum("ijk,j,k->i", np.abs(C), np.abs(u), np.abs(u))
    assert abs(u @ c) <= 1e-13 * max(scale, 1e-300)


@SETTINGS
@given(n=st.integers(1, 12), seed=st.integers(0, 2**31 - 1), alpha=st.floats(-4.0, 4.0))
def test_contraction_is_quadratic(n, seed, alpha):
    C = synth.skew_normal_tensor(n, seed)
    u = synth.initial_condition(n, seed)[0]
    c1 = oracle.nonlinear_full(C, u)
    c2 = oracle.nonlinear_full(C, alpha * u)
    np.testing.assert_allclose(c2, alpha * alpha * c1, rtol=1e-12, atol=1e-14 * (1 + np.abs(c1).max()))


@SETTINGS
@given(n=st.integers(1, 10), r=st.integers(1, 6), seed=st.integers(0, 2**31 - 1))
def test_skew_cp_equals_its_expanded_general_form(n, r, seed):
    U, V, W = (synth.normal(seed, 40 + q, 0, n * r).reshape(n, r) for q in range(3))
    u = synth.normal(seed, 43, 0, n)
    A1, A2, A3 = oracle.cp_skew_expand(U, V, W)
    c_skew = oracle.nonlinear_cp_skew(U, V, W, u)
    c_gen = oracle.nonlinear_cp(A1, A2, A3, u)
    np.testing.assert_allclose(c_skew, c_gen, rtol=1e-12, atol=1e-12 * (1 + np.abs(c_gen).max()))
    # and the reconstructed tensor is skew in (i, k)
    X = oracle.cp_reconstruct(A1, A2, A3)
    np.testing.assert_allclose(X, -X.transpose(2, 1, 0), atol=1e-12 * (1 + np.abs(X).max()))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_bdf_ext_coefficients_are_consistent_and_exact(k):
    beta, alpha = oracle.bdf_ext_coefficients(k)
    # BDFk: sum_q beta_q u^{l+1-q} = dt u'(t_{l+1}) exactly for polynomials of degree <= k
    for deg in range(k + 1):
        t = np.array([1.0 - q for q in range(k + 1)])  # t_{l+1} = 1, step 1
        lhs = sum(beta[q] * t[q] ** deg for q in range(k + 1))
        rhs = deg * 1.0 ** (deg - 1) if deg > 0 else 0.0
        assert abs(lhs - rhs) <= 1e-13, (k, deg, lhs, rhs)
    # EXTk: sum_q alpha_q f(t_{l+1-q}) = f(t_{l+1}) exactly for degree <= k-1
    for deg in range(k):
        ext = sum(alpha[q - 1] * (1.0 - q) ** deg for q in range(1, k + 1))
        assert abs(ext - 1.0) <= 1e-13, (k, deg, ext)
    assert abs(sum(beta[: k + 1])) <= 1e-15
    assert abs(sum(alpha[:k]) - 1.0) <= 1e-15
