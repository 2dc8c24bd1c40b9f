"""The autotuner (grom_autotune / grom_set_tuning): every configuration of a
ROM's tune space computes the contraction within the bounds of its kernel,
against the FP64 oracle and against the rules' configuration on the same
stored values; autotune installs one of them; stepping runs through it."""
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


def _sm():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _eval(rom, U):
    u = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _model(kind, n, r, batch, seed):
    """ROM, the oracle of its form, and the absolute-value contraction S(u)
    that bounds rounding elementwise."""
    a = synth.diag_stiffness(n)
    if kind in ("dense", "skew_packed"):
        C = synth.skew_normal_tensor(n, seed)
        rom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=a, max_batch=batch, layout=kind)
        absC = np.abs(C)
        return rom, (lambda u: oracle.nonlinear_full(C, u)), (lambda u: np.einsum("ijk,j,k->i", absC, np.abs(u),
                                                                                     np.abs(u)))
    if kind == "cp_skew":
        U, V, W, _, _ = synth.cp_workload(n, r, 1)
        rom = grom.Rom(n, "cp_skew", "bf16", factors=(U, V, W), stiffness=a, max_batch=batch)
        F1, F2, F3 = np.abs(U), np.abs(V), np.abs(W)
        return rom, (lambda u: oracle.nonlinear_cp_skew(U, V, W, u)), (
            lambda u: F1 @ ((F2.T @ np.abs(u)) * (F3.T @ np.abs(u))) + F3 @ ((F2.T @ np.abs(u)) * (F1.T @ np.abs(u))))
    A, B, Cf = (synth.normal(seed, 12 + q, 0, n * r).reshape(n, r) / np.sqrt(r) for q in range(3))
    rom = grom.Rom(n, "cp", "bf16", factors=(A, B, Cf), stiffness=a, max_batch=batch)
    F1, F2, F3 = np.abs(A), np.abs(B), np.abs(Cf)
    return rom, (lambda u: oracle.nonlinear_cp(A, B, Cf, u)), (lambda u: F1 @ ((F2.T @ np.abs(u)) * (F3.T @ np.abs(u))))


CASES = [("dense", 96, 0, 40), ("dense", 130, 0, 130), ("skew_packed", 96, 0, 40), ("skew_packed", 200, 0, 130),
         ("cp", 512, 64, 40), ("cp_skew", 512, 256, 130)]


@pytest.mark.parametrize("kind,n,r,batch", CASES)
def test_every_configuration_of_the_space_is_correct(kind, n, r, batch):
    rom, ref_fn, abs_fn = _model(kind, n, r, batch, 4100 + n)
    form = "full" if kind in ("dense", "skew_packed") else kind
    layout = kind if form == "full" else "dense"
    space = grom.tune_space(form, "bf16", n, batch, max_batch=batch, rank=r, layout=layout, sm_count=_sm())
    assert len(space) > 2
    U = synth.initial_condition(n, 4100 + n, 0, batch)
    rows = (0, batch // 2, batch - 1)
    refs = {b: ref_fn(U[b]) for b in rows}
    bounds = {b: abs_fn(U[b]) for b in rows}
    rom.set_tuning(space[0])
    c_rule = _eval(rom, U)
    rule_family = space[0]["kernel"]
    for e in space:
        rom.set_tuning(e)
        assert rom.get_tuning(batch)["kernel"] == e["kernel"]
        c = _eval(rom, U)
        for b in rows:
            assert _rel(c[b], refs[b]) <= TOL_BF16, (e, b)
            if e["kernel"] == rule_family:
                # same kernel, another launch shape: FP32 summation order only
                assert np.all(np.abs(c[b] - c_rule[b]) <= 2.0 ** -12 * bounds[b]), (e, b)
        if e["kernel"] == "tensor":  # the tensor-core kernels are deterministic
            np.testing.assert_array_equal(c, _eval(rom, U))
    rom.close()


@pytest.mark.parametrize("kind,n,r,batch", [("skew_packed", 128, 0, 48), ("cp_skew", 512, 256, 64),
                                            ("dense", 128, 0, 24)])
def test_autotune_installs_a_configuration_and_steps(kind, n, r, batch):
    rom, ref_fn, _ = _model(kind, n, r, batch, 4200 + n)
    form = "full" if kind in ("dense", "skew_packed") else kind
    layout = kind if form == "full" else "dense"
    space = grom.tune_space(form, "bf16", n, batch, max_batch=batch, rank=r, layout=layout, sm_count=_sm())
    keys = [(e["kernel"], e["tile_m"], e["split_a"], e["split_b"]) for e in space]
    assert rom.get_tuning(batch)["kernel"] == "auto"
    t = rom.autotune(batch, reps=3)
    assert (t["kernel"], t["tile_m"], t["split_a"], t["split_b"]) in keys
    assert t["timed"] == len(space) and t["ms"] > 0 and t["ms_rule"] > 0
    assert t["ms"] <= t["ms_rule"]
    got = rom.get_tuning(batch)
    assert (got["kernel"], got["tile_m"], got["split_a"], got["split_b"]) == (t["kernel"], t["tile_m"], t["split_a"],
                                                                              t["split_b"])
    # the entry serves its whole bucket and nothing else
    assert rom.get_tuning((batch - 1) // 16 * 16 + 1)["kernel"] == t["kernel"]
    # stepping through the tuned configuration
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 4200 + n, 0, batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(20)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    tr.close()
    if form == "full":
        ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=synth.skew_normal_tensor(n, 4200 + n))
    else:
        Uf, Vf, Wf, _, _ = synth.cp_workload(n, r, 1)
        ref = oracle.Rom("cp_skew", n, a, 1e-2, 1e-3, factors=(Uf, Vf, Wf))
    for b in (0, batch - 1):
        h = ref.initial_history(U0[b])
        ref.step(h, 20)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    # removing the entry restores the rules
    rom.set_tuning({"batch": batch, "kernel": "auto"})
    assert rom.get_tuning(batch)["kernel"] == "auto"
    c = _eval(rom, U0)
    for b in (0, batch - 1):
        assert _rel(c[b], ref_fn(U0[b])) <= TOL_BF16
    rom.close()


def test_set_tuning_rejects_what_the_plans_do_not_admit():
    n, batch = 96, 40
    rom, _, _ = _model("skew_packed", n, 0, batch, 4300)
    for bad in ({"batch": batch, "kernel": "tensor", "tile_m": 40}, {"batch": batch, "kernel": "tensor", "tile_m": 4},
                {"batch": batch, "kernel": "tensor", "split_a": 3}, {"batch": batch, "kernel": "stream", "tile_m": 16},
                {"batch": batch + 1, "kernel": "tensor"}):
        with pytest.raises(grom.GromError) as e:
            rom.set_tuning(bad)
        assert e.value.name == "INVALID_ARG"
    assert rom.get_tuning(batch)["kernel"] == "auto"
    rom.close()
    C = synth.skew_normal_tensor(n, 4301)
    f64 = grom.Rom(n, "full", "f64", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=batch)
    with pytest.raises(grom.GromError):
        f64.set_tuning({"batch": batch, "kernel": "tensor"})
    t = f64.autotune(batch, reps=2)  # one configuration: the streaming kernel
    assert t["kernel"] == "stream" and t["timed"] == 1
    f64.close()
