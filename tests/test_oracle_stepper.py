"""Pins of the oracle's BDFk/EXTk reduced time-stepper (Sec. 2.2, eq. nse_d1).

The coefficients are pinned by their defining order conditions, the stepper
by closed-form solutions of linear systems (exponential decay, a matrix
exponential with a non-identity mass matrix, a forced steady state), by the
observed convergence orders, and the nonlinear stepper by an independent
classical RK4 integration written here.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth


@pytest.mark.parametrize("k", [1, 2, 3])
def test_coefficients_order_conditions(k):
    beta, alpha = oracle.bdf_ext_coefficients(k)
    q = np.arange(0, k + 1, dtype=float)
    # BDFk differentiates polynomials of degree <= k exactly at t^{l+1}.
    for m in range(0, k + 1):
        lhs = np.sum(beta[: k + 1] * (-q) ** m)
        assert abs(lhs - (1.0 if m == 1 else 0.0)) < 1e-14
    # EXTk extrapolates polynomials of degree <= k-1 exactly.
    for m in range(0, k):
        lhs = np.sum(alpha[:k] * (-q[1:]) ** m)
        assert abs(lhs - (1.0 if m == 0 else 0.0)) < 1e-14


def test_cholesky_against_numpy(rng):
    n = 12
    M = rng.standard_normal((n, n))
    H = M @ M.T + n * np.eye(n)
    L = oracle.cholesky(H)
    np.testing.assert_allclose(L, np.linalg.cholesky(H), rtol=1e-12, atol=1e-13)
    b = rng.standard_normal(n)
    np.testing.assert_allclose(oracle.cholesky_solve(L, b), np.linalg.solve(H, b), rtol=1e-11)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(-H)


def _zero_rom(n, a, nu, dt, **kw):
    return oracle.Rom("full", n, a, nu, dt, C=np.zeros((n, n, n)), **kw)


def test_first_step_is_backward_euler():
    n, nu, dt = 5, 0.3, 0.01
    a = np.linspace(0.5, 2.0, n)
    u0 = np.arange(1.0, n + 1)
    rom = _zero_rom(n, a, nu, dt)
    h = rom.initial_history(u0)
    rom.step(h, 1)
    np.testing.assert_allclose(h[:n], u0 / (1.0 + nu * a * dt), rtol=1e-15)
    assert h[6 * n] == 1.0


def _seeded_history(n, u_of_t, dt, nl=None):
    """History at t = 2 dt with exact states at 0, dt, 2 dt and 2 steps taken."""
    h = np.zeros(6 * n + 1)
    for q, t in enumerate((2 * dt, dt, 0.0)):
        h[q * n:(q + 1) * n] = u_of_t(t)
        if nl is not None:
            h[(3 + q) * n:(4 + q) * n] = nl(u_of_t(t))
    h[6 * n] = 2.0
    return h


def _order(errors):
    return np.log2(np.array(errors[:-1]) / np.array(errors[1:]))


def test_linear_decay_bdf3_order3_with_exact_history():
    n, nu, T = 4, 1.0, 1.0
    a = np.array([0.5, 1.0, 2.0, 3.0])
    u0 = np.ones(n)
    exact = lambda t: u0 * np.exp(-nu * a * t)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        rom = _zero_rom(n, a, nu, dt)
        h = _seeded_history(n, exact, dt)
        steps = int(round(T / dt)) - 2
        rom.step(h, steps)
        errs.append(np.max(np.abs(h[:n] - exact(T))))
    assert np.all(np.abs(_order(errs) - 3.0) < 0.15), errs


def test_linear_decay_with_startup_is_second_order():
    n, nu, T = 3, 1.0, 1.0
    a = np.array([0.5, 1.0, 2.0])
    u0 = np.ones(n)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        rom = _zero_rom(n, a, nu, dt)
        h = rom.initial_history(u0)
        rom.step(h, int(round(T / dt)))
        errs.append(np.max(np.abs(h[:n] - u0 * np.exp(-nu * a * T))))
    assert np.all(np.abs(_order(errs) - 2.0) < 0.2), errs


def test_ext3_explicit_channel_order3():
    # L = diag(l) enters only through EXT3; exact solution exp(-(nu a + l) t).
    n, nu, T = 3, 1.0, 1.0
    a = np.array([0.2, 0.5, 1.0])
    ell = np.array([0.7, -0.3, 1.1])
    u0 = np.array([1.0, -2.0, 0.5])
    exact = lambda t: u0 * np.exp(-(nu * a + ell) * t)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        rom = _zero_rom(n, a, nu, dt, L=ell)
        h = _seeded_history(n, exact, dt)
        rom.step(h, int(round(T / dt)) - 2)
        errs.append(np.max(np.abs(h[:n] - exact(T))))
    assert np.all(np.abs(_order(errs) - 3.0) < 0.2), errs


def test_mass_matrix_matrix_exponential(rng):
    # B du/dt = -nu A u with dense SPD A, B: u(t) = expm(-nu B^-1 A t) u0.
    n, nu, T = 5, 0.5, 1.0
    M1, M2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    A = M1 @ M1.T + np.eye(n)
    B = M2 @ M2.T + n * np.eye(n)
    u0 = rng.standard_normal(n)
    G = -nu * np.linalg.solve(B, A)
    exact = lambda t: scipy.linalg.expm(G * t) @ u0
    errs = []
    for dt in (0.02, 0.01, 0.005):
        rom = oracle.Rom("full", n, A, nu, dt, C=np.zeros((n, n, n)), B=B)
        h = _seeded_history(n, exact, dt)
        rom.step(h, int(round(T / dt)) - 2)
        errs.append(np.max(np.abs(h[:n] - exact(T))))
    assert np.all(np.abs(_order(errs) - 3.0) < 0.2), errs


def test_forcing_sign_steady_state():
    # du/dt = -nu a u - f has the fixed point u* = -f/(nu a), kept exactly by
    # BDF/EXT once reached; from any start the iteration contracts onto it.
    n, nu, dt = 3, 1.0, 0.05
    a = np.array([1.0, 2.0, 4.0])
    f = np.array([0.3, -1.0, 2.0])
    rom = _zero_rom(n, a, nu, dt, f=f)
    h = rom.initial_history(np.zeros(n))
    rom.step(h, 2000)
    np.testing.assert_allclose(h[:n], -f / (nu * a), rtol=1e-12)


def _rk4(fun, u, dt, steps):
    for _ in range(steps):
        k1 = fun(u)
        k2 = fun(u + 0.5 * dt * k1)
        k3 = fun(u + 0.5 * dt * k2)
        k4 = fun(u + dt * k3)
        u = u + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


def test_nonlinear_bdf3_ext3_against_rk4():
    # du/dt = -C(u)u - nu A u with the skew workload tensor; reference from
    # classical RK4 at a step 1/64 of the finest BDF step.
    n, nu, T = 6, 0.1, 0.4
    C = 3.0 * synth.skew_normal_tensor(n, synth.seed_for(0))
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, synth.seed_for(0))[0]
    rhs = lambda u: -np.einsum("ijk,j,k->i", C, u, u) - nu * a * u
    h_ref = 0.01 / 256
    ref = lambda t: _rk4(rhs, u0, h_ref, int(round(t / h_ref)))
    nl = lambda u: np.einsum("ijk,j,k->i", C, u, u)
    uT = ref(T)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        rom = oracle.Rom("full", n, a, nu, dt, C=C)
        h = _seeded_history(n, ref, dt, nl=nl)
        rom.step(h, int(round(T / dt)) - 2)
        errs.append(np.max(np.abs(h[:n] - uT)))
    assert np.all(np.abs(_order(errs) - 3.0) < 0.3), errs


def test_inviscid_energy_drift_is_third_order_with_exact_history():
    # nu = 0 with a skew tensor: E = u^T u / 2 is conserved by the ODE, so the
    # discrete drift E(T) - E(0) is the scheme's error alone.  With the history
    # seeded exactly (RK4 at a step 1/64 of the finest BDF step) it falls by 8
    # per halving of dt (BDF3/EXT3 is third order).  With the BDF1/BDF2
    # startup the first steps' errors dominate and the drift is second order.
    n, T = 6, 0.4
    C = 3.0 * synth.skew_normal_tensor(n, synth.seed_for(0) + 11)
    u0 = synth.initial_condition(n, synth.seed_for(0) + 11)[0]
    rhs = lambda u: -np.einsum("ijk,j,k->i", C, u, u)
    h_ref = 0.01 / 256
    ref = lambda t: _rk4(rhs, u0, h_ref, int(round(t / h_ref)))
    nl = lambda u: np.einsum("ijk,j,k->i", C, u, u)
    e0 = 0.5 * u0 @ u0
    drifts = []
    for dt in (0.04, 0.02, 0.01):
        rom = oracle.Rom("full", n, np.zeros(n), 0.0, dt, C=C)
        h = _seeded_history(n, ref, dt, nl=nl)
        e, _ = rom.step(h, int(round(T / dt)) - 2, want_energy=True)
        drifts.append(abs(e[-1] - e0))
    assert np.all(np.abs(_order(drifts) - 3.0) < 0.35), drifts
    started = []
    for dt in (0.04, 0.02, 0.01):
        rom = oracle.Rom("full", n, np.zeros(n), 0.0, dt, C=C)
        h = rom.initial_history(u0)
        e, _ = rom.step(h, int(round(T / dt)), want_energy=True)
        started.append(abs(e[-1] - e0))
    assert np.all(np.abs(_order(started) - 2.0) < 0.2), started


def test_scalar_cp_model_closed_form_and_blow_up():
    # n = 1, rank 1: c = a b c u^2, so du/dt = -k u^2 with k = abc, solved by
    # u(t) = u0 / (1 + k u0 t).  For k u0 > 0 the state decays, and the stepper
    # with its BDF1/BDF2 startup converges to it at order 2.  For k u0 < 0 the
    # solution blows up at t* = -1/(k u0), which the unstructured CP form can
    # do (Sec. 4.3: plain CPD-ROMs at low rank diverge, skew ones do not).
    u0, T = 1.0, 1.0
    one = np.ones((1, 1))
    errs = []
    for dt in (0.02, 0.01, 0.005):
        rom = oracle.Rom("cp", 1, np.zeros(1), 0.0, dt, factors=(2.0 * one, one, one))
        h = rom.initial_history(np.array([u0]))
        rom.step(h, int(round(T / dt)))
        errs.append(abs(h[0] - u0 / (1.0 + 2.0 * u0 * T)))
    assert np.all(np.abs(_order(errs) - 2.0) < 0.2), errs
    rom = oracle.Rom("cp", 1, np.zeros(1), 0.0, 1e-3, factors=(-one, one, one))
    h = rom.initial_history(np.array([u0]))
    rom.step(h, 900)  # t = 0.9 < t* = 1: still the closed form
    assert abs(h[0] - u0 / (1.0 - u0 * 0.9)) < 1e-3 * 10.0
    with np.errstate(all="ignore"):
        rom.step(h, 600)  # past t*
    assert not np.isfinite(h[0]) or abs(h[0]) > 1e6


def test_skew_cp_model_stays_bounded():
    # the skew CP structure conserves u^T u / 2 at nu = 0 (u^T c(u) = 0), so
    # even a large initial state only drifts by the scheme's error
    n, r = 4, 2
    U, V, W = (synth.normal(synth.seed_for(0) + 21, 40 + q, 0, n * r).reshape(n, r) for q in range(3))
    u0 = 3.0 * synth.initial_condition(n, synth.seed_for(0) + 21)[0]
    rom = oracle.Rom("cp_skew", n, np.zeros(n), 0.0, 1e-3, factors=(U, V, W))
    h = rom.initial_history(u0)
    e, inv = rom.step(h, 2000, want_energy=True, want_invariant=True)
    e0 = 0.5 * u0 @ u0
    assert np.all(np.isfinite(h)) and np.max(np.abs(e - e0)) <= 1e-4 * e0
    assert np.max(np.abs(inv)) <= 1e-12 * np.max(e)


def test_energy_and_invariant_outputs():
    n, dt = 8, 1e-3
    C = synth.skew_normal_tensor(n, synth.seed_for(0))
    u0 = synth.initial_condition(n, synth.seed_for(0))[0]
    # nu = 0: continuous energy is conserved; the drift shrinks with dt.
    drifts = []
    for dt_ in (4e-3, 2e-3, 1e-3):
        rom = oracle.Rom("full", n, np.zeros(n), 0.0, dt_, C=C)
        h = rom.initial_history(u0)
        e, inv = rom.step(h, int(round(0.2 / dt_)), want_energy=True, want_invariant=True)
        drifts.append(abs(e[-1] - 0.5 * u0 @ u0))
        assert np.max(np.abs(inv)) < 1e-13
    assert drifts[0] / drifts[1] > 3.0 and drifts[1] / drifts[2] > 3.0, drifts
    # nu > 0: energy decays monotonically for this dissipative model.
    rom = oracle.Rom("full", n, synth.diag_stiffness(n), 1.0, dt, C=C)
    h = rom.initial_history(u0)
    e, _ = rom.step(h, 200, want_energy=True)
    assert np.all(np.diff(e) < 0)


def test_history_is_resumable():
    n, dt = 5, 1e-3
    C = synth.skew_normal_tensor(n, 7)
    rom = oracle.Rom("full", n, synth.diag_stiffness(n), 1e-2, dt, C=C)
    u0 = synth.initial_condition(n, 7)[0]
    h1 = rom.initial_history(u0)
    rom.step(h1, 10)
    h2 = rom.initial_history(u0)
    rom.step(h2, 4)
    rom.step(h2, 6)
    np.testing.assert_array_equal(h1, h2)


def test_cp_forms_step_like_their_reconstruction():
    n, r, dt = 6, 3, 1e-3
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    A1, A2, A3 = oracle.cp_skew_expand(U, V, W)
    X = oracle.cp_reconstruct(A1, A2, A3)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, seed)[0]
    hs = []
    for rom in (oracle.Rom("full", n, a, 1e-2, dt, C=X),
                oracle.Rom("cp", n, a, 1e-2, dt, factors=(A1, A2, A3)),
                oracle.Rom("cp_skew", n, a, 1e-2, dt, factors=(U, V, W))):
        h = rom.initial_history(u0)
        rom.step(h, 50)
        hs.append(h)
    np.testing.assert_allclose(hs[1], hs[0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(hs[2], hs[0], rtol=1e-12, atol=1e-15)
