"""Parity at the benchmark's full size (N = 1024) in the launch configuration
bench.py times: every output against the FP64 oracle, element by element,
and the skew invariant (a property that holds at any size).

Per output the bound is |c_i - ref_i| <= E * sum_jk |C_ijk u_j u_k| (the
contraction with absolute values, which bounds what any rounding of the
tensor or of the sums can move c_i), with E = 2^-8 for BF16 storage (one
rounding of each tensor entry, 2^-9), 2^-20 for FP32, 2^-40 for F32X2 (its
double-single sums of N = 1024 terms: the worst element seen on GB300 was
2^-41.9 before the accumulators were renormalised per chunk) and 2^-42 for
FP64;
the relative l2 error of the whole vector must stay within the per-evaluation
tolerance (1e-12 FP64 / F32X2, 1e-5 FP32, 2e-2 BF16).  A partition or
chunk-boundary fault anywhere in the 1024 outputs fails the elementwise bound.

The tensor is the counter-based skew normal workload, generated identically
for both sides."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

N = 1024
SEED = synth.seed_for(2) + 1000
TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}
ELEM = {"f64": 2.0 ** -42, "f32x2": 2.0 ** -40, "f32": 2.0 ** -20, "bf16": 2.0 ** -8}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tensor():
    grom.build()
    oracle.set_threads(16)
    return synth.skew_normal_tensor(N, SEED)


@pytest.fixture(scope="module")
def abs_tensor(tensor):
    return np.abs(tensor)


_REF = {}


def _reference(tensor, abs_tensor, u, key):
    """The oracle's c and the absolute-value contraction for state u."""
    if key not in _REF:
        _REF[key] = (oracle.nonlinear_full(tensor, u), oracle.nonlinear_full(abs_tensor, np.abs(u)))
    return _REF[key]


def _check_all_rows(c, ref, scale, storage, what):
    err = _rel(c, ref)
    assert err <= TOL[storage], (what, storage, err)
    bad = np.nonzero(np.abs(c - ref) > ELEM[storage] * scale)[0]
    assert bad.size == 0, (what, storage, bad[:10], (np.abs(c - ref) / scale)[bad[:10]])
    return err


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("storage", ["bf16", "f64", "f32x2", "f32"])
def test_full_size_single_trajectory(tensor, abs_tensor, storage, layout):
    u = synth.initial_condition(N, SEED)[0]
    rom = grom.Rom(N, "full", storage, tensor=tensor, stiffness=synth.diag_stiffness(N), layout=layout)
    ud = torch.from_numpy(u[None, :].copy()).cuda()
    cd = torch.empty_like(ud)
    rom.nonlinear(ud, cd)
    torch.cuda.synchronize()
    c = cd.cpu().numpy()[0]
    ref, scale = _reference(tensor, abs_tensor, u, "u0")
    _check_all_rows(c, ref, scale, storage, "nonlinear")
    # invariant u^T c = 0 to the accumulation's rounding (the stored tensor is exactly skew)
    uf = u.astype(np.float32).astype(np.float64) if storage in ("f32", "bf16") else u
    u_acc = {"f64": 2.0 ** -53, "f32x2": 2.0 ** -47, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}[storage]
    assert abs(uf @ c) <= 8 * np.sqrt(N) * u_acc * np.sum(np.abs(uf)) * np.sum(scale)
    rom.close()


@pytest.mark.parametrize("storage", ["f32x2", "bf16", "f64"])
def test_full_size_persistent_stepper_one_step(tensor, abs_tensor, storage):
    # bench.py's timed configuration (one trajectory, skew-packed tensor, the
    # persistent cooperative stepper): after one step the history holds
    # n^0 = C(u^0)u^0 at [4N, 5N) of the canonical state, every row checked
    a = synth.diag_stiffness(N)
    u0 = synth.initial_condition(N, SEED)[0]
    rom = grom.Rom(N, "full", storage, tensor=tensor, stiffness=a, nu=1e-2, dt=1e-3, layout="skew_packed")
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(1)
    code, _ = tr.status()
    assert code == 0
    h = tr.get_state()[0]
    ref, scale = _reference(tensor, abs_tensor, u0, "u0")
    _check_all_rows(h[4 * N:5 * N], ref, scale, storage, "persistent step")
    # and the new state against the oracle's first step
    ro = oracle.Rom("full", N, a, 1e-2, 1e-3, C=tensor)
    hr = ro.initial_history(u0)
    ro.step(hr, 1)
    assert _rel(h[:N], hr[:N]) <= TOL[storage]
    tr.close()
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("storage", ["f32x2", "bf16"])
def test_full_size_stepping_headline_configuration(tensor, storage, layout):
    # the bench's models: one trajectory, BDF3/EXT3, persistent stepper
    # (skew-packed) or captured graphs (dense), 24 steps
    steps = 24
    a = synth.diag_stiffness(N)
    u0 = synth.initial_condition(N, SEED)[0]
    rom = grom.Rom(N, "full", storage, tensor=tensor, stiffness=a, nu=1e-2, dt=1e-3, layout=layout)
    tr = grom.Trajectories(rom, u0[None, :])
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    h = tr.get_state()[0]
    ref = oracle.Rom("full", N, a, 1e-2, 1e-3, C=tensor)
    hr = ref.initial_history(u0)
    ref.step(hr, steps)
    assert _rel(h[:N], hr[:N]) <= {"f32x2": 1e-11, "bf16": 2e-2}[storage]
    assert h[6 * N] == steps
    tr.close()
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("batch", [16, 256])
def test_full_size_batched_tensor_cores(tensor, abs_tensor, batch, layout):
    # dense: K2 over the Khatri-Rao product; skew-packed: the factored K2P;
    # every output of three trajectories
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
        ref, scale = _reference(tensor, abs_tensor, U0[b], ("batch", b, batch))
        _check_all_rows(c[b], ref, scale, "bf16", "batched b=%d" % b)
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
