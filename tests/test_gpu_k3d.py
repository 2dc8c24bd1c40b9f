"""K3D, the batched CP form of FP64 ROMs in double-single FP32 arithmetic
(Sec. 3.1 eq. tc_ap; skew structure Sec. 3.3), against the FP64 oracle:
per-evaluation relative l2 error within the FP64 tolerance (1e-12), the
exact-FP64 GEMMs (K3g, GROM_KERNEL_STREAM) on the same factors, stepping,
determinism, and the split-K reduction (sizes with several K splits)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _factors(form, n, r, seed):
    if form == "cp_skew":
        U, V, W, _, _ = synth.cp_workload(n, r, 1)
        return (U, V, W), lambda u: oracle.nonlinear_cp_skew(U, V, W, u)
    rng = np.random.default_rng(seed)
    A, B, C = (rng.standard_normal((n, r)) / np.sqrt(r) for _ in range(3))
    return (A, B, C), lambda u: oracle.nonlinear_cp(A, B, C, u)


def _eval(rom, U0, kernel="auto"):
    rom.set_kernel(kernel)
    ud = torch.from_numpy(U0).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    return cd.cpu().numpy()


@pytest.mark.parametrize("form", ["cp_skew", "cp"])
@pytest.mark.parametrize("n,r,batch", [(17, 5, 16), (100, 33, 17), (200, 129, 70), (300, 260, 20), (64, 64, 130)])
def test_k3d_matches_oracle(form, n, r, batch):
    grom.build()
    fac, ref = _factors(form, n, r, 7 + n)
    U0 = synth.initial_condition(n, 11 + n, 0, batch)
    rom = grom.Rom(n, form, "f64", factors=fac, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0)
    c_fp64 = _eval(rom, U0, "stream")  # the FP64 GEMMs
    for b in range(batch):
        rb = ref(U0[b])
        assert _rel(c[b], rb) <= 1e-12, (b, _rel(c[b], rb))
        assert _rel(c[b], c_fp64[b]) <= 1e-12, b
    # deterministic: a second evaluation gives the same bits
    np.testing.assert_array_equal(_eval(rom, U0), c)
    rom.close()


@pytest.mark.parametrize("form", ["cp_skew", "cp"])
def test_k3d_n1024_large_rank(form):
    # N = 1024 and R = 768, several column tiles and K splits (AUTO takes the
    # tensor-core path, K3O, from N R B = 2^24 on)
    grom.build()
    n, batch = 1024, 16
    fac, ref = _factors(form, n, 768, 5)
    U0 = synth.initial_condition(n, 3, 0, batch)
    rom = grom.Rom(n, form, "f64", factors=fac, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0)
    for b in (0, 1, batch // 2, batch - 1):
        assert _rel(c[b], ref(U0[b])) <= 1e-12, b
    rom.close()


def test_k3d_stepping_matches_oracle():
    grom.build()
    n, r, batch, steps = 96, 40, 24, 30
    (U, V, W), _ = _factors("cp_skew", n, r, 0)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 5, 0, batch)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(U, V, W))
    for b in (0, batch - 1):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(tr.get_state()[b][:n], h[:n]) <= 1e-12, b
    tr.close()
    rom.close()


@pytest.mark.parametrize("form", ["cp_skew", "cp"])
@pytest.mark.parametrize("steps", [6, 17])
def test_k3d_fused_step_bitwise(form, steps):
    # Stepping sums the expansion's splits in the step kernel, which also
    # writes the next state's hi/lo planes; a call prepares the planes from
    # the ring only at its first step.  One call of several steps (graph
    # replays included) equals single-step calls bit for bit, and the first
    # step's advection term equals the evaluation entry point's.
    grom.build()
    n, r, batch = 200, 129, 70
    fac, _ = _factors(form, n, r, 3)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 9, 0, batch)
    rom = grom.Rom(n, form, "f64", factors=fac, stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    c = _eval(rom, U0)
    t1 = grom.Trajectories(rom, U0)
    t1.step(steps)
    t2 = grom.Trajectories(rom, U0)
    for _ in range(steps):
        t2.step(1)
    assert t1.status()[0] == 0 and t2.status()[0] == 0
    np.testing.assert_array_equal(t1.get_state(), t2.get_state())
    t3 = grom.Trajectories(rom, U0)
    t3.step(1)
    np.testing.assert_array_equal(t3.get_state()[:, 4 * n:5 * n], c)
    for t in (t1, t2, t3):
        t.close()
    rom.close()


@pytest.mark.parametrize("batch", [16, 70])
def test_k3d_stepping_energy_invariant(batch):
    # the fused step with energy and invariant asked for (the step kernel's
    # full variant summing the expansion splits) against the oracle stepper
    grom.build()
    n, r, steps = 150, 100, 23
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    energy = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    inv = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    tr.step(steps, energy, inv)
    assert tr.status()[0] == 0
    H = tr.get_state()
    for b in (0, batch // 2, batch - 1):
        ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(U, V, W))
        h = ref.initial_history(U0[b])
        e_ref, _ = ref.step(h, steps, want_energy=True, want_invariant=True)
        assert _rel(H[b][:n], h[:n]) <= 1e-11, b
        assert H[b][6 * n] == steps
        np.testing.assert_allclose(energy.cpu().numpy()[:, b], e_ref, rtol=1e-12)
        # the skew CP structure conserves u^T c(u) = 0 to rounding
        assert np.max(np.abs(inv.cpu().numpy()[:, b])) <= 1e-9 * np.max(e_ref)
    tr.close()
    rom.close()
