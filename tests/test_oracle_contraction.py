"""Pins of the oracle's dense contraction c_i = sum_jk C_ijk u_j u_k (Sec. 2.2, eq. Cu).

Each test checks the oracle against something other than itself: numpy's
einsum on brute-force inputs, the closed form for a rank-one tensor, the
skew-symmetry invariant of Sec. 3.2 and quadratic homogeneity.
"""
import numpy as np
import pytest

import oracle
import synth


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17])
def test_full_matches_einsum(n, rng):
    C = rng.standard_normal((n, n, n))
    u = rng.standard_normal(n)
    ref = np.einsum("ijk,j,k->i", C, u, u)
    assert _rel(oracle.nonlinear_full(C, u), ref) < 1e-13


def test_full_rank_one_closed_form(rng):
    # C = a o b o c  =>  c_i = a_i (b . u)(c . u): an index slip (test index
    # contracted with u, or u applied once) breaks this.
    n = 7
    a, b, c, u = (rng.standard_normal(n) for _ in range(4))
    C = np.einsum("i,j,k->ijk", a, b, c)
    got = oracle.nonlinear_full(C, u)
    assert _rel(got, a * (b @ u) * (c @ u)) < 1e-14


def test_full_row_slab_matches_whole(rng):
    n = 9
    C = rng.standard_normal((n, n, n))
    u = rng.standard_normal(n)
    whole = oracle.nonlinear_full(C, u)
    part = oracle.nonlinear_full_rows(C[3:7], 3, u)
    np.testing.assert_array_equal(part, whole[3:7])


@pytest.mark.parametrize("n", [4, 16, 64])
def test_skew_invariant(n, rng):
    # Sec. 3.2: C_ijk = -C_kji  =>  u^T C(u) u = 0 for every u.
    C = synth.skew_normal_tensor(n, synth.seed_for(0))
    for _ in range(3):
        u = rng.standard_normal(n)
        c = oracle.nonlinear_full(C, u)
        scale = np.sum(np.abs(u)) * np.sum(np.abs(np.einsum("ijk,j,k->ijk", C, u, u)))
        assert abs(u @ c) <= 8 * np.sqrt(n) * 2.0 ** -53 * scale
        assert np.linalg.norm(c) > 0


def test_homogeneity(rng):
    n = 6
    C = rng.standard_normal((n, n, n))
    u = rng.standard_normal(n)
    np.testing.assert_allclose(oracle.nonlinear_full(C, 2.0 * u), 4.0 * oracle.nonlinear_full(C, u), rtol=1e-14)


def test_pins_reject_planted_mistakes(rng):
    # Mutants of the definition, written here on the CPU: each must fail at
    # least one of the checks above, showing that the pins discriminate.
    n = 7
    a, b, c, u = (rng.standard_normal(n) for _ in range(4))
    C = np.einsum("i,j,k->ijk", a, b, c)
    closed = a * (b @ u) * (c @ u)
    mutants = {
        "test/advecting swapped": np.einsum("jik,j,k->i", C, u, u),
        "single u": np.einsum("ijk,k->i", C, u),
        "sign": -np.einsum("ijk,j,k->i", C, u, u),
    }
    for name, m in mutants.items():
        assert _rel(m, closed) > 1e-3, name
