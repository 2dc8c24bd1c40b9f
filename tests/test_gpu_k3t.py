"""K3T, the batched CP-form contraction on the tcgen05 tensor cores (BF16
factors): the projections [B C]^T X (skew: [V W U]^T X) and the expansion
A Z (skew: [U, -W] Z) as two GEMMs with the states and the Hadamard products
split into BF16 hi/lo parts.  Checked against the FP64 oracle of the CP form,
against the SIMT kernels on the same stored factors, and through stepping."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grom.build()
    grom.load()
    assert torch.cuda.is_available()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _eval(rom, U):
    u = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _factors(form, n, r, seed):
    if form == "cp_skew":
        U, V, W, _, _ = synth.cp_workload(n, r, 1)
        return (U, V, W), (lambda u: oracle.nonlinear_cp_skew(U, V, W, u))
    A, B, Cf = (synth.normal(seed, 12 + q, 0, n * r).reshape(n, r) / np.sqrt(r) for q in range(3))
    return (A, B, Cf), (lambda u: oracle.nonlinear_cp(A, B, Cf, u))


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()


# ranks below, at and across the 64-wide padding; n across the 128-row tile;
# batches across the 16-column granule and the 128-column tile
@pytest.mark.parametrize("form", ["cp", "cp_skew"])
@pytest.mark.parametrize("n,r", [(17, 5), (64, 24), (130, 64), (200, 129)])
@pytest.mark.parametrize("batch", [1, 33, 130])
def test_k3t_matches_oracle_and_simt(form, n, r, batch):
    facs, ref_fn = _factors(form, n, r, 300 + n + r)
    U0 = synth.initial_condition(n, 300 + n, 0, batch)
    rom = grom.Rom(n, form, "bf16", factors=facs, stiffness=synth.diag_stiffness(n), max_batch=batch)
    rom.set_kernel("tensor")
    c = _eval(rom, U0)
    rom.set_kernel("stream")
    c_simt = _eval(rom, U0)
    # the oracle on the BF16 factors the kernels hold
    fr = tuple(_bf16(f) for f in facs)
    ref_r = (oracle.nonlinear_cp_skew if form == "cp_skew" else oracle.nonlinear_cp)
    F1, F2, F3 = (np.abs(f) for f in facs)
    for b in range(batch):
        # elementwise bounds on S_i, the contraction with absolute values (the
        # skew form cancels strongly, so no relative bound holds for every state)
        ua = np.abs(U0[b])
        if form == "cp_skew":  # (U, V, W): U (p o q) - W (p o s)
            S = F1 @ ((F2.T @ ua) * (F3.T @ ua)) + F3 @ ((F2.T @ ua) * (F1.T @ ua))
        else:  # (A, B, C): A (p o q)
            S = F1 @ ((F2.T @ ua) * (F3.T @ ua))
        # same stored factors: the states and products exact to ~2^-17, FP32 sums
        exact = ref_r(*fr, U0[b])
        assert np.all(np.abs(c[b] - exact) <= 2.0 ** -14 * S), (form, n, r, batch, b)
        assert np.all(np.abs(c[b] - c_simt[b]) <= 2.0 ** -14 * S), (form, n, r, batch, b)
        # against the FP64 factors: each factor's BF16 rounding (2^-9)
        ref = ref_fn(U0[b])
        assert np.all(np.abs(c[b] - ref) <= 2.0 ** -6 * S), (form, n, r, batch, b)
    rom.close()


@pytest.mark.parametrize("form", ["cp", "cp_skew"])
def test_k3t_is_the_auto_choice_and_steps(form):
    n, r, batch, steps = 96, 48, 40, 30
    facs, _ = _factors(form, n, r, 77)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 77, 0, batch)
    rom = grom.Rom(n, form, "bf16", factors=facs, stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    tr = grom.Trajectories(rom, U0)  # auto: batch >= 16 selects K3T
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    tr.close()
    for b in (0, batch - 1):
        ref = oracle.Rom(form, n, a, 1e-2, 1e-3, factors=facs)
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    rom.close()


def test_k3t_is_deterministic():
    n, r, batch = 200, 100, 256
    facs, _ = _factors("cp_skew", n, r, 5)
    U0 = synth.initial_condition(n, 5, 0, batch)
    rom = grom.Rom(n, "cp_skew", "bf16", factors=facs, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c1, c2 = _eval(rom, U0), _eval(rom, U0)
    np.testing.assert_array_equal(c1, c2)
    rom.close()


def test_k3t_augmented_cp_model():
    # the zeroth-mode CP model: the core through K3T, the zeroth-mode terms
    # through the stepper's L and f
    n, r, steps, batch = 40, 16, 25, 36
    seed = synth.seed_for(0) + 9900
    A, B, Cf = (synth.normal(seed, 12 + q, 0, n * r).reshape(n, r) / np.sqrt(r) for q in range(3))
    A, Bb, Cb = synth.augment_cp(A, B, Cf, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp", "bf16", factors=(A, Bb, Cb), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch,
                   augmented=True)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    H = tr.get_state()
    tr.close()
    ref = oracle.Rom("cp_aug", n, a, 1e-2, 1e-3, factors=(A, Bb, Cb))
    for b in (0, batch - 1):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    rom.close()


def test_tensor_kernel_needs_bf16_cp():
    n, r = 32, 8
    facs, _ = _factors("cp", n, r, 1)
    rom = grom.Rom(n, "cp", "f32", factors=facs, stiffness=synth.diag_stiffness(n), max_batch=40)
    with pytest.raises(grom.GromError) as e:
        rom.set_kernel("tensor")
    assert e.value.name == "UNSUPPORTED"
    rom.close()


# The persistent batched stepper: a call of two or more steps runs every step
# in one cooperative launch (projection, expansion and step phases between
# grid barriers); single-step calls run the per-step kernels.  The tiles, the
# split sums and the arithmetic are the same, so the states after K steps are
# bitwise equal either way, and so are the energy and invariant series.
@pytest.mark.parametrize("form", ["cp_skew", "cp"])
@pytest.mark.parametrize("n,r,batch", [(200, 129, 70), (256, 96, 16), (130, 64, 130)])
def test_persistent_stepper_is_bitwise_the_per_step_path(form, n, r, batch):
    facs, _ = _factors(form, n, r, 500 + n)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 600 + n, 0, batch)
    steps = 12
    rom = grom.Rom(n, form, "bf16", factors=facs, stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    one = grom.Trajectories(rom, U0)
    for _ in range(steps):
        one.step(1)
    many = grom.Trajectories(rom, U0)
    many.step(steps)
    assert many.status()[0] == 0 and one.status()[0] == 0
    np.testing.assert_array_equal(many.get_state(), one.get_state())
    # with the energy and invariant asked for (the standalone step blocks)
    e1 = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    i1 = torch.empty_like(e1)
    e2, i2 = torch.empty_like(e1), torch.empty_like(e1)
    for s in range(steps):
        one.step(1, e1[s:s + 1], i1[s:s + 1])
    many.step(steps, e2, i2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(many.get_state(), one.get_state())
    assert torch.equal(e1, e2) and torch.equal(i1, i2)
    one.close()
    many.close()
    rom.close()


def test_persistent_stepper_matches_oracle():
    n, r, batch, steps = 160, 80, 40, 25
    (U, V, W), _ = _factors("cp_skew", n, r, 0)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 77, 0, batch)
    rom = grom.Rom(n, "cp_skew", "bf16", factors=(U, V, W), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    assert tr.status()[0] == 0
    ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(U, V, W))
    for b in (0, batch - 1):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(tr.get_state()[b][:n], h[:n]) <= TOL_BF16, b
    tr.close()
    rom.close()


def test_persistent_stepper_serving_pool_masks_and_budgets():
    # a pool of uneven requests: quanta of 8 steps (persistent launches) give
    # the same final states, bit for bit, as quanta of one step (per-step kernels)
    n, r = 96, 48
    (U, V, W), _ = _factors("cp_skew", n, r, 0)
    rom = grom.Rom(n, "cp_skew", "bf16", factors=(U, V, W), stiffness=synth.diag_stiffness(n), max_batch=24)
    rng = np.random.default_rng(5)
    count = 40
    horizons = rng.integers(3, 60, count)
    arrivals = np.sort(rng.random(count) * 0.01)
    u0s = [synth.initial_condition(n, 900 + q)[0] for q in range(count)]
    finals = []
    for quantum in (8, 1):
        srv = grom.Server(150 * 2 ** 30, quantum=quantum)
        mid = srv.add_rom(rom, 24)
        out = srv.serve([mid] * count, horizons, arrivals, u0s, want_final=True)
        assert np.all(out["status"] == 0)
        np.testing.assert_array_equal(out["steps"], horizons)
        finals.append(out["final"])
        srv.close()
    for q in range(count):
        np.testing.assert_array_equal(finals[0][q], finals[1][q], err_msg="request %d" % q)
    rom.close()
