"""Parity at the benchmark's full size (N = 1024) in the launch configuration
bench.py times: sampled outputs against the FP64 oracle computed row by row,
and the skew invariant (a property that holds at any size).

The tensor is the counter-based skew normal workload, generated identically
for both sides (the oracle only regenerates the sampled rows)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

N = 1024
SEED = synth.seed_for(2) + 1000
ROWS = [0, 1, 2, 511, 512, 777, 1000, 1022, 1023]
TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tensor():
    grom.build()
    oracle.set_threads(16)
    return synth.skew_normal_tensor(N, SEED)


# the sampled rows, regenerated independently from the counter-based generator
_SLABS = {}


def _oracle_rows(u):
    out = []
    for i in ROWS:
        if i not in _SLABS:
            _SLABS[i] = synth.skew_normal_tensor(N, SEED, i, i + 1)
        out.append(oracle.nonlinear_full_rows(_SLABS[i], i, u))
    return np.concatenate(out)


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("storage", ["bf16", "f64", "f32x2", "f32"])
def test_full_size_single_trajectory(tensor, storage, layout):
    u = synth.initial_condition(N, SEED)[0]
    rom = grom.Rom(N, "full", storage, tensor=tensor, stiffness=synth.diag_stiffness(N), layout=layout)
    ud = torch.from_numpy(u[None, :].copy()).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    c = cd.cpu().numpy()[0]
    ref = _oracle_rows(u)
    got = c[ROWS]
    # relative error on the sampled rows, measured against the sampled oracle values
    assert _rel(got, ref) <= TOL[storage], (storage, _rel(got, ref))
    # invariant u^T c = 0 to the accumulation's rounding (the stored tensor is exactly skew)
    uf = u.astype(np.float32).astype(np.float64) if storage in ("f32", "bf16") else u
    u_acc = {"f64": 2.0 ** -53, "f32x2": 2.0 ** -47, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}[storage]
    scale = np.sum(np.abs(uf)) * np.sum(oracle.nonlinear_full(np.abs(tensor), np.abs(uf)))
    assert abs(uf @ c) <= 8 * np.sqrt(N) * u_acc * scale
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
def test_full_size_stepping_headline_configuration(tensor, layout):
    # the bench's headline: BF16 storage, one trajectory, BDF3/EXT3 with graphs
    steps = 24
    a = synth.diag_stiffness(N)
    u0 = synth.initial_condition(N, SEED)[0]
    rom = grom.Rom(N, "full", "bf16", tensor=tensor, stiffness=a, nu=1e-2, dt=1e-3, layout=layout)
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    h = tr.get_state()[0]
    ref = oracle.Rom("full", N, a, 1e-2, 1e-3, C=tensor)
    hr = ref.initial_history(u0)
    ref.step(hr, steps)
    assert _rel(h[:N], hr[:N]) <= 2e-2
    assert h[6 * N] == steps
    tr.close()
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("batch", [16, 256])
def test_full_size_batched_tensor_cores(tensor, batch, layout):
    # dense: K2 over the Khatri-Rao product; skew-packed: the factored K2P
    U0 = synth.initial_condition(N, SEED, 0, batch)
    rom = grom.Rom(N, "full", "bf16", tensor=tensor, stiffness=synth.diag_stiffness(N), max_batch=batch,
                   layout=layout)
    rom.set_kernel("tensor")
    ud = torch.from_numpy(U0).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    c = cd.cpu().numpy()
    for b in (0, batch // 3, batch - 1):
        assert _rel(c[b][ROWS], _oracle_rows(U0[b])) <= 2e-2, b
    rom.close()


@pytest.mark.parametrize("storage", ["bf16", "f64"])
@pytest.mark.parametrize("batch", [1, 64])
def test_full_size_cp_rank_n(storage, batch):
    grom.build()
    U, V, W, _, seed = synth.cp_workload(N, N, 2)
    U0 = synth.initial_condition(N, seed, 0, batch)
    rom = grom.Rom(N, "cp_skew", storage, factors=(U, V, W), stiffness=synth.diag_stiffness(N), max_batch=batch)
    ud = torch.from_numpy(U0).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    c = cd.cpu().numpy()
    for b in sorted({0, batch - 1}):
        assert _rel(c[b], oracle.nonlinear_cp_skew(U, V, W, U0[b])) <= TOL[storage]
    rom.close()
