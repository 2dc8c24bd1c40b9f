"""K3O, the batched CP form of FP64 ROMs on the BF16 tensor cores with every
operand split into 7- or 6-bit integer digit slices (Sec. 3.1 eq. tc_ap; skew
structure Sec. 3.3), against the FP64 oracle: per-evaluation relative l2
error within the FP64 tolerance (1e-12), agreement with the double-single
kernels (K3D) on the same factors, stepping with energy and invariant, the
fused combine-and-step kernel against the plain evaluation (bitwise), and
determinism."""
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


def _eval(rom, U0, kernel):
    rom.set_kernel(kernel)
    ud = torch.from_numpy(U0).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    return cd.cpu().numpy()


@pytest.mark.parametrize("form", ["cp_skew", "cp"])
@pytest.mark.parametrize("n,r,batch", [(17, 5, 16), (100, 33, 17), (200, 129, 70), (300, 260, 20), (64, 64, 130)])
def test_k3o_matches_oracle(form, n, r, batch):
    grom.build()
    fac, ref = _factors(form, n, r, 7 + n)
    U0 = synth.initial_condition(n, 11 + n, 0, batch)
    rom = grom.Rom(n, form, "f64", factors=fac, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0, "tensor")
    c_ds = _eval(rom, U0, "auto")  # K3D on the same factors
    for b in range(batch):
        rb = ref(U0[b])
        assert _rel(c[b], rb) <= 1e-12, (b, _rel(c[b], rb))
        assert _rel(c[b], c_ds[b]) <= 1e-12, b
    # deterministic: a second evaluation gives the same bits
    np.testing.assert_array_equal(_eval(rom, U0, "tensor"), c)
    rom.close()


@pytest.mark.parametrize("form", ["cp_skew", "cp"])
def test_k3o_n1024_rank_n(form):
    grom.build()
    n, batch = 1024, 64
    fac, ref = _factors(form, n, n, 5)
    U0 = synth.initial_condition(n, 3, 0, batch)
    rom = grom.Rom(n, form, "f64", factors=fac, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, U0, "tensor")
    for b in (0, 1, batch // 2, batch - 1):
        assert _rel(c[b], ref(U0[b])) <= 1e-12, b
    rom.close()


def test_k3o_stepping_energy_invariant():
    grom.build()
    n, r, batch, steps = 150, 100, 40, 23
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch)
    rom.set_kernel("tensor")
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
        assert np.max(np.abs(inv.cpu().numpy()[:, b])) <= 1e-9 * np.max(e_ref)
    tr.close()
    rom.close()


# Stepping runs the expansion's combine and the step as one kernel; it forms c
# with the plain evaluation's arithmetic, so after a step the ring's c slot
# holds the evaluation of the state the step was taken at, bitwise.  One and
# four elements per thread (40 and 70 trajectories); with and without the
# energy and invariant (the two step variants).
@pytest.mark.parametrize("batch", [40, 70])
@pytest.mark.parametrize("sums", [False, True])
def test_k3o_fused_step_ring_holds_the_plain_evaluation(batch, sums):
    grom.build()
    n, r = 150, 100
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=synth.diag_stiffness(n), nu=1e-2, dt=1e-3,
                   max_batch=batch)
    rom.set_kernel("tensor")
    tr = grom.Trajectories(rom, U0)

    def step():
        if sums:
            e = torch.empty((1, batch), dtype=torch.float64, device="cuda")
            tr.step(1, e, torch.empty_like(e))
        else:
            tr.step(1)
        assert tr.status()[0] == 0
        return tr.get_state()

    # get_state exports newest first: u^l, u^(l-1), u^(l-2), then the c of
    # each (that of u^l evaluated by the export itself), then l
    H1 = step()
    np.testing.assert_array_equal(H1[:, n:2 * n], U0)
    np.testing.assert_array_equal(H1[:, 4 * n:5 * n], _eval(rom, U0, "tensor"))  # written by the fused step
    H2 = step()
    np.testing.assert_array_equal(H2[:, 4 * n:5 * n], _eval(rom, np.ascontiguousarray(H1[:, :n]), "tensor"))
    assert np.all(H2[:, 6 * n] == 2)
    tr.close()
    rom.close()


def test_k3o_serving_alone_equals_mix():
    # a serving pool on K3O: every trajectory's digits, slice products and
    # sums depend on its own state only, so a request's result is bitwise
    # the same alone and in the mix; and it matches the oracle stepper
    grom.build()
    n, r, slots = 96, 64, 20
    U, V, W, _, seed = synth.cp_workload(n, r, 1)
    a = synth.diag_stiffness(n)
    rom = grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=a, nu=1e-2, dt=1e-3, max_batch=slots)
    rom.set_kernel("tensor")
    rng = np.random.default_rng(5)
    count = 40
    horizons = rng.integers(5, 60, count)
    arrivals = np.sort(rng.random(count) * 0.01)
    u0s = [synth.initial_condition(n, 300 + q)[0] for q in range(count)]
    srv = grom.Server(150 * 2 ** 30, quantum=8)
    mid = srv.add_rom(rom, slots)
    out = srv.serve([mid] * count, horizons, arrivals, u0s, want_final=True)
    assert np.all(out["status"] == 0), out["status"]
    assert out["stats"]["peak_active"] > 1
    srv.close()
    alone = grom.Server(150 * 2 ** 30, quantum=8)
    aid = alone.add_rom(rom, slots)
    for q in range(0, count, 4):
        one = alone.serve([aid], [horizons[q]], [0.0], [u0s[q]], want_final=True)
        assert one["status"][0] == 0
        np.testing.assert_array_equal(one["final"][0], out["final"][q], err_msg="request %d" % q)
    alone.close()
    for q in range(0, count, 8):
        ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(U, V, W))
        h = ref.initial_history(u0s[q])
        ref.step(h, int(horizons[q]))
        assert _rel(out["final"][q], h[:n]) <= 1e-11, q
    rom.close()
