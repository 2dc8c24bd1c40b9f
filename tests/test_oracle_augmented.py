"""Pins of the oracle's operators that include the zeroth mode (Sec. 2.2,
eq. nse_ode with the augmented vector ubar = (1, u); Sec. 4.2 "full" tensor).

The augmented contraction is checked against an independent einsum, against
the split form C(u)u + (C1 + C2)u + c0 read from eq. nse_d1 and eq.
zeroth_contribution (with C1_ik = Cbar_i0k, C2_ij = Cbar_ij0,
c0_i = Cbar_i00), and the stepper of the augmented model against the core
model stepped with that L and f.
"""
import numpy as np
import pytest

import oracle
import synth


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [1, 4, 9])
def test_augmented_contraction_against_einsum(n):
    Cbar = synth.augment_tensor(synth.skew_normal_tensor(n, 31 + n), 5)
    u = synth.initial_condition(n, 3)[0]
    ub = np.concatenate([[1.0], u])
    ref = np.einsum("ijk,j,k->i", Cbar, ub, ub)
    assert _rel(oracle.nonlinear_full_augmented(Cbar, u), ref) < 1e-13


@pytest.mark.parametrize("n", [3, 8])
def test_augmented_contraction_splits_into_core_linear_and_constant(n):
    C = synth.skew_normal_tensor(n, 40 + n)
    Cbar = synth.augment_tensor(C, 6)
    u = synth.initial_condition(n, 4)[0]
    C1, C2, c0 = Cbar[:, 0, 1:], Cbar[:, 1:, 0], Cbar[:, 0, 0]
    split = oracle.nonlinear_full(C, u) + (C1 + C2) @ u + c0
    assert _rel(oracle.nonlinear_full_augmented(Cbar, u), split) < 1e-13


def test_zero_zeroth_mode_reduces_to_core():
    n = 6
    C = synth.skew_normal_tensor(n, 50)
    Cbar = np.zeros((n, n + 1, n + 1))
    Cbar[:, 1:, 1:] = C
    u = synth.initial_condition(n, 1)[0]
    np.testing.assert_array_equal(oracle.nonlinear_full_augmented(Cbar, u), oracle.nonlinear_full(C, u))


@pytest.mark.parametrize("n,r", [(5, 3), (7, 10)])
def test_augmented_cp_against_reconstruction(n, r):
    rng = np.random.default_rng(n + r)
    A, B, Cf = rng.standard_normal((n, r)), rng.standard_normal((n + 1, r)), rng.standard_normal((n + 1, r))
    u = rng.standard_normal(n)
    ub = np.concatenate([[1.0], u])
    X = np.einsum("im,jm,km->ijk", A, B, Cf)
    ref = np.einsum("ijk,j,k->i", X, ub, ub)
    assert _rel(oracle.nonlinear_cp_augmented(A, B, Cf, u), ref) < 1e-13


def test_planted_swap_of_zeroth_planes_is_caught():
    # reading the zeroth mode at the end of the index range instead of index 0
    n = 5
    Cbar = synth.augment_tensor(synth.skew_normal_tensor(n, 60), 7)
    u = synth.initial_condition(n, 2)[0]
    wrong = np.roll(np.roll(Cbar, -1, axis=1), -1, axis=2)
    assert _rel(oracle.nonlinear_full_augmented(wrong, u), oracle.nonlinear_full_augmented(Cbar, u)) > 0.1


def test_augmented_stepper_equals_core_with_zeroth_terms():
    n, steps = 6, 40
    C = synth.skew_normal_tensor(n, 70)
    Cbar = synth.augment_tensor(C, 8)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, 9)[0]
    aug = oracle.Rom("full_aug", n, a, 1e-2, 1e-3, C=Cbar)
    core = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C, L=Cbar[:, 0, 1:] + Cbar[:, 1:, 0], f=Cbar[:, 0, 0])
    ha, hc = aug.initial_history(u0), core.initial_history(u0)
    aug.step(ha, steps)
    core.step(hc, steps)
    assert _rel(ha[:n], hc[:n]) < 1e-12
