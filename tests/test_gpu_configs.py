"""The paper-shaped workloads other than the benchmark line, as parity cases
against the FP64 oracle (trajectory errors are also written to
$GROM_REPORT_DIR/configs.json when that variable is set).

* N = 512, one trajectory, 2000 BDF3/EXT3 steps: FP64 full G-ROM and FP64
  CPD-ROM with R = 128 and 512 (skew CP factors of the CP-structured tensor),
  each against its oracle, plus the model gap between them.
* N = 1024: the 1000-step trajectory error and u^T c(u) of every storage type,
  for the full G-ROM and for the skew CPD-ROM with R = N (factors of the
  CP-structured tensor), each against the oracle of the same form.
* N = 2048: per-evaluation parity of every output and the invariant (BF16, FP64).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu
NU, DT = 1e-2, 1e-3
REPORT = {}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _record(key, value):
    REPORT[key] = value
    d = os.environ.get("GROM_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "configs.json"), "w") as fh:
            json.dump(REPORT, fh, indent=1)


@pytest.fixture(scope="module", autouse=True)
def _setup():
    grom.build()
    oracle.set_threads(os.cpu_count() or 1)


def _gpu_traj(rom, u0, steps):
    tr = grom.Trajectories(rom, u0[None, :])
    inv = torch.empty((steps, 1), dtype=torch.float64, device="cuda")
    tr.step(steps, None, inv)
    code, _ = tr.status()
    assert code == 0
    h = tr.get_state()[0]
    tr.close()
    return h, inv.cpu().numpy()[:, 0]


def test_n512_full_vs_cpd_2000_steps():
    n, steps = 512, 2000
    a = synth.diag_stiffness(n)
    U, V, W, s, seed = synth.cp_workload(n, 512, 1)
    C = synth.cp_tensor(U, V, W, seed, s)
    u0 = synth.initial_condition(n, seed)[0]
    ref = oracle.Rom("full", n, a, NU, DT, C=C)
    h_full = ref.initial_history(u0)
    ref.step(h_full, steps)
    rom = grom.Rom(n, "full", "f64", tensor=C, stiffness=a, nu=NU, dt=DT)
    h, _ = _gpu_traj(rom, u0, steps)
    err_full = _rel(h[:n], h_full[:n])
    assert err_full <= 1e-9, err_full
    rom.close()
    out = {"full_f64_traj_rel_err": err_full}
    for R in (128, 512):
        Ur, Vr, Wr, _, _ = synth.cp_workload(n, R, 1)
        ref = oracle.Rom("cp_skew", n, a, NU, DT, factors=(Ur, Vr, Wr))
        h_cp = ref.initial_history(u0)
        ref.step(h_cp, steps)
        rom = grom.Rom(n, "cp_skew", "f64", factors=(Ur, Vr, Wr), stiffness=a, nu=NU, dt=DT)
        h, _ = _gpu_traj(rom, u0, steps)
        err = _rel(h[:n], h_cp[:n])
        assert err <= 1e-9, (R, err)
        out["cpd_f64_R%d_traj_rel_err" % R] = err
        out["cpd_R%d_vs_full_model_gap" % R] = _rel(h_cp[:n], h_full[:n])
        rom.close()
    _record("n512_2000_steps", out)


def test_n1024_precision_sweep_1000_steps():
    n, steps = 1024, 1000
    a = synth.diag_stiffness(n)
    seed = synth.seed_for(2) + 2000
    C = synth.skew_normal_tensor(n, seed)
    u0 = synth.initial_condition(n, seed)[0]
    ref = oracle.Rom("full", n, a, NU, DT, C=C)
    h_ref = ref.initial_history(u0)
    _, inv_ref = ref.step(h_ref, steps, want_invariant=True)
    tol = {"f64": 1e-9, "f32x2": 1e-9, "f32": 1e-4, "bf16": 5e-2}
    out = {}
    for storage in ("f64", "f32x2", "f32", "bf16"):
        rom = grom.Rom(n, "full", storage, tensor=C, stiffness=a, nu=NU, dt=DT)
        h, inv = _gpu_traj(rom, u0, steps)
        err = _rel(h[:n], h_ref[:n])
        out[storage] = {"traj_rel_err_1000": err, "max_abs_uTc": float(np.max(np.abs(inv))),
                        "energy_final": float(0.5 * h[:n] @ h[:n])}
        assert err <= tol[storage], (storage, err)
        rom.close()
    out["oracle_max_abs_uTc"] = float(np.max(np.abs(inv_ref)))
    _record("n1024_1000_steps", out)


def test_n1024_cpd_precision_sweep_1000_steps():
    # the CPD half of the precision sweep (Sec. 3.1 eq. tc_ap with the skew
    # structure of Sec. 3.3): factors stored in FP64, FP32 and BF16, FP32
    # accumulation below FP64, FP64 state; the oracle steps the FP64 factors
    n, steps = 1024, 1000
    a = synth.diag_stiffness(n)
    U, V, W, _, seed = synth.cp_workload(n, n, 2)
    u0 = synth.initial_condition(n, seed)[0]
    ref = oracle.Rom("cp_skew", n, a, NU, DT, factors=(U, V, W))
    h_ref = ref.initial_history(u0)
    _, inv_ref = ref.step(h_ref, steps, want_invariant=True)
    # scale of the invariant: ||u0|| * ||c(u0)|| (both decay along the trajectory)
    norm0 = float(np.linalg.norm(u0) * np.linalg.norm(oracle.nonlinear_cp_skew(U, V, W, u0)))
    tol = {"f64": 1e-9, "f32": 1e-4, "bf16": 5e-2}
    inv_tol = {"f64": 1e-13, "f32": 1e-5, "bf16": 1e-5}
    out = {}
    for storage in ("f64", "f32", "bf16"):
        rom = grom.Rom(n, "cp_skew", storage, factors=(U, V, W), stiffness=a, nu=NU, dt=DT)
        h, inv = _gpu_traj(rom, u0, steps)
        err = _rel(h[:n], h_ref[:n])
        out[storage] = {"traj_rel_err_1000": err, "max_abs_uTc": float(np.max(np.abs(inv))),
                        "max_abs_uTc_over_norms0": float(np.max(np.abs(inv)) / norm0),
                        "energy_final": float(0.5 * h[:n] @ h[:n])}
        assert err <= tol[storage], (storage, err)
        assert np.max(np.abs(inv)) <= inv_tol[storage] * norm0, (storage, out[storage])
        rom.close()
    out["oracle_max_abs_uTc"] = float(np.max(np.abs(inv_ref)))
    out["cpd_vs_full_note"] = "each form against the oracle of the same form"
    _record("n1024_cpd_1000_steps", out)


def test_n2048_all_rows():
    # every output at N = 2048 (the FP64 tensor is 69 GB) against the oracle,
    # elementwise against the contraction with absolute values (computed in
    # slabs of rows so that no second full-size array is held)
    n = 2048
    seed = synth.seed_for(2) + 3000
    C = synth.skew_normal_tensor(n, seed)
    u = synth.initial_condition(n, seed)[0]
    ref = oracle.nonlinear_full(C, u)
    slab = 128
    scale = np.concatenate([oracle.nonlinear_full_rows(np.abs(C[i:i + slab]), i, np.abs(u))
                            for i in range(0, n, slab)])
    out = {}
    for storage, tol, elem in (("bf16", 2e-2, 2.0 ** -8), ("f64", 1e-12, 2.0 ** -42)):
        rom = grom.Rom(n, "full", storage, tensor=C, stiffness=synth.diag_stiffness(n))
        ud = torch.from_numpy(u[None, :].copy()).cuda()
        cd = torch.empty_like(ud)
        rom.nonlinear(ud, cd)
        torch.cuda.synchronize()
        c = cd.cpu().numpy()[0]
        err = _rel(c, ref)
        assert err <= tol, (storage, err)
        worst = float(np.max(np.abs(c - ref) / scale))
        assert worst <= elem, (storage, worst)
        uf = u.astype(np.float32).astype(np.float64) if storage == "bf16" else u
        out[storage] = {"rel_err_all_rows": err, "max_abs_err_over_abs_contraction": worst,
                        "uTc_over_norms": float(abs(uf @ c) / (np.linalg.norm(uf) * np.linalg.norm(c)))}
        rom.close()
    _record("n2048_all_rows", out)
