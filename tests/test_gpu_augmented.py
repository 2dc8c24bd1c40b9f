"""GPU parity of operators that include the zeroth mode (Sec. 4.2 "full"
tensor; grom_desc.augmented): the library keeps the core and moves the
zeroth-mode terms into the stepper's L and f; the oracle steps the augmented
model directly with ubar = (1, u)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grom.build()
    grom.load()
    assert torch.cuda.is_available()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _traj(rom, U0, steps):
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    tr.close()
    return H


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32x2", 1e-11), ("bf16", 2e-2)])
def test_augmented_full_trajectory(layout, storage, tol):
    n, steps, batch = 40, 30, 2
    seed = synth.seed_for(0) + 9500
    C = synth.skew_normal_tensor(n, seed)
    Cbar = synth.augment_tensor(C, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "full", storage, tensor=Cbar, stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch, layout=layout,
                   augmented=True)
    H = _traj(rom, U0, steps)
    ref = oracle.Rom("full_aug", n, a, 1e-2, 1e-3, C=Cbar)
    for b in range(batch):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= tol, (layout, storage, b)
    # the evaluation alone is the core contraction
    u = torch.from_numpy(U0.copy()).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    assert _rel(c.cpu().numpy()[0], oracle.nonlinear_full(C, U0[0])) <= (1e-12 if storage != "bf16" else 2e-2)
    rom.close()


def test_augmented_with_callers_linear_and_forcing():
    # the caller's own L and f add to the zeroth-mode terms
    n, steps = 24, 25
    seed = synth.seed_for(0) + 9600
    Cbar = synth.augment_tensor(synth.skew_normal_tensor(n, seed), seed)
    a = synth.diag_stiffness(n)
    ell = 0.3 * np.arange(1, n + 1) / n
    f = synth.normal(seed, 11, 0, n) * 0.1
    u0 = synth.initial_condition(n, seed)
    rom = grom.Rom(n, "full", "f64", tensor=Cbar, stiffness=a, linear=ell, forcing=f, augmented=True)
    H = _traj(rom, u0, steps)
    ref = oracle.Rom("full_aug", n, a, 1e-2, 1e-3, C=Cbar, L=ell, f=f)
    h = ref.initial_history(u0[0])
    ref.step(h, steps)
    assert _rel(H[0][:n], h[:n]) <= 1e-11
    rom.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("bf16", 2e-2)])
@pytest.mark.parametrize("batch", [1, 20])
def test_augmented_cp_trajectory(storage, tol, batch):
    n, r, steps = 48, 12, 30
    seed = synth.seed_for(0) + 9700
    A, B, Cf = (synth.normal(seed, 12 + q, 0, n * r).reshape(n, r) / np.sqrt(r) for q in range(3))
    A, Bb, Cb = synth.augment_cp(A, B, Cf, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "cp", storage, factors=(A, Bb, Cb), stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch,
                   augmented=True)
    H = _traj(rom, U0, steps)
    ref = oracle.Rom("cp_aug", n, a, 1e-2, 1e-3, factors=(A, Bb, Cb))
    for b in sorted({0, batch - 1}):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= tol, (storage, batch, b)
    rom.close()


def test_augmented_rejected_where_undefined():
    n, r = 16, 4
    U, V, W, _, _ = synth.cp_workload(n, r, 1)
    with pytest.raises(grom.GromError) as e:
        grom.Rom(n, "cp_skew", "f64", factors=(U, V, W), stiffness=synth.diag_stiffness(n), augmented=True)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(grom.GromError) as e:
        grom.Rom(n, "full", "f64", stiffness=synth.diag_stiffness(n), defer_tensor=True, augmented=True)
    assert e.value.name == "INVALID_ARG"
