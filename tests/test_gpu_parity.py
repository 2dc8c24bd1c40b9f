"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances on the per-evaluation relative l2 error ||c - c_ref|| / ||c_ref||:
FP64 storage 1e-12, F32X2 (double-single) 1e-12, FP32 1e-5, BF16 2e-2.  The
oracle runs on the unrounded FP64 operators, so the FP32/BF16 errors include
the storage rounding.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}
# unit roundoff of the accumulation, for the invariant bound
U_ACC = {"f64": 2.0 ** -53, "f32x2": 2.0 ** -47, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grom.build()
    grom.load()
    assert torch.cuda.is_available()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _u_fed(u, storage):
    """The u the kernel multiplies with (rounded like the storage arithmetic)."""
    if storage in ("f32", "bf16"):
        return u.astype(np.float32).astype(np.float64)
    return u


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _full_rom(C, storage, max_batch=1, **kw):
    n = C.shape[0]
    return grom.Rom(n, "full", storage, tensor=C, stiffness=synth.diag_stiffness(n), max_batch=max_batch, **kw)


def _eval(rom, U):
    u = _dev(U)
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


# ------------------------------------------------------------------ full form
@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 100, 130])
def test_full_single(storage, n):
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + n)
    u = synth.initial_condition(n, synth.seed_for(0) + n)[0]
    rom = _full_rom(C, storage)
    c = _eval(rom, u[None, :])[0]
    ref = oracle.nonlinear_full(C, u)
    if n > 1:
        assert _rel(c, ref) <= TOL[storage], (storage, n, _rel(c, ref))
    else:
        assert abs(c[0]) < 1e-300 and ref[0] == 0.0  # C_000 = -C_000 = 0
    # skew invariant u^T c = 0, to the accumulation's rounding (storage rounding keeps C skew)
    uf = _u_fed(u, storage)
    scale = np.sum(np.abs(uf)) * np.sum(np.abs(np.einsum("ijk,j,k->ijk", C, uf, uf)))
    assert abs(uf @ c) <= 8 * np.sqrt(n) * U_ACC[storage] * scale + 1e-300


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
@pytest.mark.parametrize("batch", [2, 3, 8, 13])
def test_full_batched(storage, batch):
    n = 70
    C = synth.skew_normal_tensor(n, 99)
    U = synth.initial_condition(n, 99, 0, batch)
    rom = _full_rom(C, storage, max_batch=batch)
    c = _eval(rom, U)
    for b in range(batch):
        assert _rel(c[b], oracle.nonlinear_full(C, U[b])) <= TOL[storage], (storage, batch, b)


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_full_nonskew_general_tensor(storage, rng):
    # the ABI takes any dense tensor (inflow/outflow case of Sec. 3.2)
    n = 48
    C = rng.standard_normal((n, n, n)) / n
    u = rng.standard_normal(n)
    c = _eval(_full_rom(C, storage), u[None, :])[0]
    assert _rel(c, oracle.nonlinear_full(C, u)) <= TOL[storage]


def test_full_deferred_slab_upload():
    n = 40
    C = synth.skew_normal_tensor(n, 5)
    u = synth.initial_condition(n, 5)[0]
    rom = grom.Rom(n, "full", "f64", stiffness=synth.diag_stiffness(n), defer_tensor=True)
    with pytest.raises(grom.GromError):
        rom.nonlinear(_dev(u[None]), torch.empty((1, n), dtype=torch.float64, device="cuda"))
    for i0, i1 in ((0, 7), (7, 30), (30, 40)):
        rom.upload_slab(i0, np.ascontiguousarray(C[i0:i1]))
    c = _eval(rom, u[None, :])[0]
    assert _rel(c, oracle.nonlinear_full(C, u)) <= 1e-12


# -------------------------------------------------------------------- CP forms
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("n,r", [(1, 1), (5, 3), (33, 1), (64, 64), (100, 130), (257, 64)])
def test_cp_skew(storage, n, r):
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    u = synth.initial_condition(n, seed)[0]
    rom = grom.Rom(n, "cp_skew", storage, factors=(U, V, W), stiffness=synth.diag_stiffness(n))
    c = _eval(rom, u[None, :])[0]
    ref = oracle.nonlinear_cp_skew(U, V, W, u)
    if n > 1:
        assert _rel(c, ref) <= TOL[storage], (storage, n, r, _rel(c, ref))
    else:
        # n = 1: the two skew terms cancel exactly; only rounding is left
        p, q, s = V.T @ u, W.T @ u, U.T @ u
        scale = np.abs(U @ (p * q)).sum() + np.abs(W @ (p * s)).sum()
        assert np.max(np.abs(c)) <= 8 * U_ACC[storage] * scale


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("batch", [1, 3, 6])
def test_cp_general_batched(storage, batch, rng):
    n, r = 90, 37
    A, B, Cf = (rng.standard_normal((n, r)) / np.sqrt(r) for _ in range(3))
    U0 = rng.standard_normal((batch, n))
    rom = grom.Rom(n, "cp", storage, factors=(A, B, Cf), stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0)
    for b in range(batch):
        assert _rel(c[b], oracle.nonlinear_cp(A, B, Cf, U0[b])) <= TOL[storage]


# --------------------------------------------------------------------- stepper
def test_trajectory_n64_fp64_1000_steps():
    """Plain FP64 full G-ROM, N=64, 1000 BDF3/EXT3 steps, dt=1e-3, nu=1e-2."""
    n, dt, nu, steps = 64, 1e-3, 1e-2, 1000
    seed = synth.seed_for(0)
    C = synth.skew_normal_tensor(n, seed)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, seed)[0]
    ref = oracle.Rom("full", n, a, nu, dt, C=C)
    h_ref = ref.initial_history(u0)
    e_ref, i_ref = ref.step(h_ref, steps, want_energy=True, want_invariant=True)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a, nu=nu, dt=dt)
    tr = grom.Trajectories(rom, u0[None, :])
    energy = torch.empty((steps, 1), dtype=torch.float64, device="cuda")
    inv = torch.empty((steps, 1), dtype=torch.float64, device="cuda")
    tr.step(steps, energy, inv)
    code, bad = tr.status()
    assert code == 0 and bad == -1
    h = tr.get_state()[0]
    err = _rel(h[:n], h_ref[:n])
    assert err <= 1e-10, err
    assert h[6 * n] == steps
    np.testing.assert_allclose(energy.cpu().numpy()[:, 0], e_ref, rtol=1e-10)
    scale = np.max(np.abs(i_ref)) + 1e-14
    assert np.max(np.abs(inv.cpu().numpy()[:, 0] - i_ref)) < 1e-12 * max(1.0, scale)
    # the exported history matches the oracle's layout (u^l, u^l-1, u^l-2, n^l, n^l-1, n^l-2, l)
    assert _rel(h[:6 * n], h_ref[:6 * n]) <= 1e-10


@pytest.mark.parametrize("form,storage,tol", [("full", "bf16", 2e-2), ("full", "f32", 1e-5), ("full", "f32x2", 1e-10),
                                              ("cp_skew", "f64", 1e-10), ("cp_skew", "bf16", 2e-2)])
def test_trajectory_other_forms(form, storage, tol):
    n, r, dt, nu, steps = 48, 16, 1e-3, 1e-2, 300
    U, V, W, s, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, seed)[0]
    if form == "full":
        C = synth.cp_tensor(U, V, W, seed, s)
        ref = oracle.Rom("full", n, a, nu, dt, C=C)
        rom = grom.Rom(n, "full", storage, tensor=C, stiffness=a, nu=nu, dt=dt)
    else:
        ref = oracle.Rom("cp_skew", n, a, nu, dt, factors=(U, V, W))
        rom = grom.Rom(n, "cp_skew", storage, factors=(U, V, W), stiffness=a, nu=nu, dt=dt)
    h_ref = ref.initial_history(u0)
    ref.step(h_ref, steps)
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(steps)
    h = tr.get_state()[0]
    assert _rel(h[:n], h_ref[:n]) <= tol, _rel(h[:n], h_ref[:n])


def test_dense_operators_and_forcing(rng):
    n, dt, nu, steps = 12, 2e-3, 0.3, 60
    C = synth.skew_normal_tensor(n, 3)
    M1, M2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    A = M1 @ M1.T / n + np.eye(n)
    B = M2 @ M2.T / n + np.eye(n)
    L = 0.1 * rng.standard_normal((n, n))
    f = 0.05 * rng.standard_normal(n)
    u0 = rng.standard_normal(n)
    ref = oracle.Rom("full", n, A, nu, dt, C=C, B=B, L=L, f=f)
    h_ref = ref.initial_history(u0)
    e_ref, i_ref = ref.step(h_ref, steps, want_energy=True, want_invariant=True)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=A, mass=B, linear=L, forcing=f, nu=nu, dt=dt)
    tr = grom.Trajectories(rom, u0[None, :])
    energy = torch.empty((steps, 1), dtype=torch.float64, device="cuda")
    inv = torch.empty((steps, 1), dtype=torch.float64, device="cuda")
    tr.step(steps, energy, inv)
    h = tr.get_state()[0]
    assert _rel(h[:6 * n], h_ref[:6 * n]) <= 1e-11
    np.testing.assert_allclose(energy.cpu().numpy()[:, 0], e_ref, rtol=1e-11)
    np.testing.assert_allclose(inv.cpu().numpy()[:, 0], i_ref, rtol=1e-9, atol=1e-12)


def test_diagonal_mass_linear_forcing(rng):
    n, dt, nu, steps = 20, 1e-3, 0.5, 80
    C = synth.skew_normal_tensor(n, 4)
    a = synth.diag_stiffness(n)
    mb = 1.0 + rng.random(n)
    ell = 0.2 * rng.standard_normal(n)
    f = 0.1 * rng.standard_normal(n)
    u0 = rng.standard_normal(n)
    ref = oracle.Rom("full", n, a, nu, dt, C=C, B=np.diag(mb), L=ell, f=f)
    h_ref = ref.initial_history(u0)
    ref.step(h_ref, steps)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a, mass=mb, linear=ell, forcing=f, nu=nu, dt=dt)
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(steps)
    assert _rel(tr.get_state()[0][:6 * n], h_ref[:6 * n]) <= 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_lower_orders(order):
    n, dt, nu, steps = 16, 1e-3, 1e-2, 40
    C = synth.skew_normal_tensor(n, 8)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, 8)[0]
    ref = oracle.Rom("full", n, a, nu, dt, order=order, C=C)
    h_ref = ref.initial_history(u0)
    ref.step(h_ref, steps)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a, nu=nu, dt=dt, order=order)
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(steps)
    assert _rel(tr.get_state()[0][:n], h_ref[:n]) <= 1e-12


def test_batched_trajectories_match_single():
    n, batch, steps = 40, 5, 50
    C = synth.skew_normal_tensor(n, 11)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 11, 0, batch)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    H = tr.get_state()
    for b in range(batch):
        ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= 1e-12


def test_checkpoint_resume_is_bit_identical():
    n, steps = 50, 30
    C = synth.skew_normal_tensor(n, 12)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, 12)[0]
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a)
    t1 = grom.Trajectories(rom, u0[None, :])
    t1.step(steps)
    h_cont = t1.get_state()
    t2 = grom.Trajectories(rom, u0[None, :])
    t2.step(12)
    snap = t2.get_state()
    t3 = grom.Trajectories(rom, u0[None, :])
    t3.set_state(snap)
    t3.step(steps - 12)
    np.testing.assert_array_equal(t3.get_state(), h_cont)


def test_set_state_with_exact_history_seeding_matches_oracle():
    n, dt = 10, 1e-3
    C = synth.skew_normal_tensor(n, 13)
    a = synth.diag_stiffness(n)
    rng = np.random.default_rng(4)
    h0 = np.zeros(6 * n + 1)
    h0[:3 * n] = rng.standard_normal(3 * n)
    h0[6 * n] = 7.0
    for q in range(3):
        h0[(3 + q) * n:(4 + q) * n] = oracle.nonlinear_full(C, h0[q * n:(q + 1) * n])
    ref = oracle.Rom("full", n, a, 1e-2, dt, C=C)
    h_ref = h0.copy()
    ref.step(h_ref, 25)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a)
    tr = grom.Trajectories(rom, h0[None, :n])
    tr.set_state(h0[None, :])
    tr.step(25)
    assert _rel(tr.get_state()[0], h_ref) <= 1e-12


def test_nonfinite_state_is_reported():
    n, batch = 20, 4
    C = synth.skew_normal_tensor(n, 14)
    U0 = synth.initial_condition(n, 14, 0, batch)
    U0[2, 3] = np.nan
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(3)
    code, bad = tr.status()
    assert grom.ERRORS[code] == "NONFINITE" and bad == 2
    H = tr.get_state()
    assert np.all(np.isfinite(H[0])) and np.all(np.isfinite(H[1])) and np.all(np.isfinite(H[3]))


def test_invalid_arguments_are_rejected():
    n = 8
    C = synth.skew_normal_tensor(n, 1)
    with pytest.raises(grom.GromError) as ei:
        grom.Rom(n, "full", "f64", tensor=C, stiffness=synth.diag_stiffness(n), dt=-1.0)
    assert ei.value.name == "INVALID_ARG"
    with pytest.raises(grom.GromError) as ei:
        grom.Rom(n, "full", "f64", tensor=C, stiffness=-np.ones(n), nu=1e6)
    assert ei.value.name == "INVALID_ARG"
    rom = _full_rom(C, "f64", max_batch=2)
    u = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(grom.GromError):
        rom.nonlinear(u, torch.empty_like(u))


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("form", ["cp", "cp_skew"])
@pytest.mark.parametrize("batch", [16, 37, 70])
def test_cp_batched_gemm_path(storage, form, batch, rng):
    # batches of 16 or more run the register-tiled GEMM kernels
    n, r = 75, 29
    if form == "cp_skew":
        U, V, W, _, seed = synth.cp_workload(n, r, 1)
        factors = (U, V, W)
        ref_fn = lambda u: oracle.nonlinear_cp_skew(U, V, W, u)
    else:
        factors = tuple(rng.standard_normal((n, r)) / np.sqrt(r) for _ in range(3))
        ref_fn = lambda u: oracle.nonlinear_cp(*factors, u)
    U0 = synth.initial_condition(n, 9, 0, batch)
    rom = grom.Rom(n, form, storage, factors=factors, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0)
    for b in range(batch):
        assert _rel(c[b], ref_fn(U0[b])) <= TOL[storage], (storage, form, batch, b)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("bf16", 2e-2)])
def test_cp_batched_stepping_matches_oracle(storage, tol):
    n, r, batch, steps = 64, 24, 20, 30
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp_skew", storage, factors=(U, V, W), stiffness=a, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    H = tr.get_state()
    for b in (0, 11, batch - 1):
        ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(U, V, W))
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= tol


def test_cp_batched_varying_batch_sizes_share_scratch():
    # one ROM, batches of different sizes in turn (split counts differ)
    n, r, mb = 96, 40, 70
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=synth.diag_stiffness(n), max_batch=mb)
    for batch in (70, 20, 41, 16, 70):
        U0 = synth.initial_condition(n, batch, 0, batch)
        c = _eval(rom, U0)
        for b in (0, batch // 2, batch - 1):
            assert _rel(c[b], oracle.nonlinear_cp_skew(U, V, W, U0[b])) <= 1e-12, (batch, b)


def test_device_wait_timeout_is_reported_and_recoverable():
    # failure detection without a fault: a bounded wait on a barrier nothing
    # signals gives up after 20 ms, the status reports TIMEOUT once, and the
    # ROM keeps working
    n = 32
    C = synth.skew_normal_tensor(n, 2)
    u = synth.initial_condition(n, 2)[0]
    rom = _full_rom(C, "f64")
    rom.selftest_timeout(20_000_000)
    with pytest.raises(grom.GromError) as ei:
        rom.sync()
    assert ei.value.name == "TIMEOUT"
    rom.sync()  # reported once
    assert _rel(_eval(rom, u[None, :])[0], oracle.nonlinear_full(C, u)) <= 1e-12


@pytest.mark.parametrize("storage,batch,tol", [("f64", 2, 1e-11), ("f32", 3, 1e-5), ("bf16", 4, 2e-2), ("f64", 1, 1e-11)])
def test_cp_persistent_stepper_with_outputs(storage, batch, tol):
    # CP forms with a few trajectories step in one persistent cooperative launch
    n, r, dt, nu, steps = 80, 33, 1e-3, 1e-2, 37
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp_skew", storage, factors=(U, V, W), stiffness=a, nu=nu, dt=dt, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    energy = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    inv = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    tr.step(steps, energy, inv)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    for b in range(batch):
        ref = oracle.Rom("cp_skew", n, a, nu, dt, factors=(U, V, W))
        h = ref.initial_history(U0[b])
        e_ref, i_ref = ref.step(h, steps, want_energy=True, want_invariant=True)
        assert _rel(H[b][:n], h[:n]) <= tol
        assert H[b][6 * n] == steps
        np.testing.assert_allclose(energy.cpu().numpy()[:, b], e_ref, rtol=max(tol, 1e-12))
        # the skew CP structure conserves u^T c(u) = 0
        assert np.max(np.abs(inv.cpu().numpy()[:, b])) <= 1e-3 * np.max(e_ref) * (1e-6 if storage == "f64" else 1)


def test_cp_persistent_resume_is_bit_identical():
    n, r = 64, 20
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, seed)[0]
    rom = grom.Rom(n, "cp_skew", "bf16", factors=(U, V, W), stiffness=a)
    t1 = grom.Trajectories(rom, u0[None, :])
    t1.step(40)
    whole = t1.get_state()
    t2 = grom.Trajectories(rom, u0[None, :])
    t2.step(15)
    t3 = grom.Trajectories(rom, u0[None, :])
    t3.set_state(t2.get_state())
    t3.step(25)
    np.testing.assert_array_equal(t3.get_state(), whole)
