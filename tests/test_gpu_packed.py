"""GPU parity of the skew-packed tensor layout (one entry of each pair
C_ijk = -C_kji stored) against the FP64 oracle on the full tensor.

The packed model is the dense model exactly when the tensor is skew, so the
tolerances are the dense ones: per-evaluation relative l2 error 1e-12 (FP64,
F32X2), 1e-5 (FP32), 2e-2 (BF16).  Sizes cover odd and even n, rows shorter
than one 64-element tile, several streaming chunks per test index, CTAs that
split a test index, and batches larger than one kernel pass.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}
U_ACC = {"f64": 2.0 ** -53, "f32x2": 2.0 ** -47, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}


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


def _rom(C, storage, layout="skew_packed", max_batch=1, **kw):
    n = C.shape[0]
    return grom.Rom(n, "full", storage, tensor=C, stiffness=synth.diag_stiffness(n), max_batch=max_batch,
                    layout=layout, **kw)


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 96, 129, 200])
def test_packed_matches_oracle(storage, n):
    seed = synth.seed_for(0) + 7000 + n
    C = synth.skew_normal_tensor(n, seed)
    batch = 3
    U = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, storage, max_batch=batch)
    c = _eval(rom, U)
    for b in range(batch):
        ref = oracle.nonlinear_full(C, U[b])
        if np.linalg.norm(ref) == 0.0:  # n = 1: a skew tensor is zero
            assert np.all(c[b] == 0.0)
            continue
        assert _rel(c[b], ref) <= TOL[storage], (storage, n, b, _rel(c[b], ref))
        uf = U[b].astype(np.float32).astype(np.float64) if storage in ("f32", "bf16") else U[b]
        scale = np.sum(np.abs(uf)) * np.sum(oracle.nonlinear_full(np.abs(C), np.abs(uf)))
        assert abs(uf @ c[b]) <= 8 * np.sqrt(n) * U_ACC[storage] * scale
    rom.close()


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_packed_equals_dense(storage):
    # same stored values (rounding is odd-symmetric), different summation order
    n = 160
    seed = synth.seed_for(0) + 7100
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, 2)
    dense = _rom(C, storage, layout="dense", max_batch=2)
    packed = _rom(C, storage, max_batch=2)
    cd, cp = _eval(dense, U), _eval(packed, U)
    bound = 1e-13 if storage == "f64" else 1e-5
    for b in range(2):
        assert _rel(cp[b], cd[b]) <= bound
    dense.close()
    packed.close()


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
def test_packed_many_passes(storage):
    # batch larger than the trajectories of one kernel pass
    n, batch = 96, 19
    seed = synth.seed_for(0) + 7200
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, storage, max_batch=batch)
    c = _eval(rom, U)
    for b in (0, 7, 8, 18):
        assert _rel(c[b], oracle.nonlinear_full(C, U[b])) <= TOL[storage], b
    rom.close()


def test_packed_cp_structured_tensor_accepted():
    # skew only to FP64 rounding of its entries: the probe accepts it
    n, R = 48, 24
    U, V, W, s, seed = synth.cp_workload(n, R, 1)
    C = synth.cp_tensor(U, V, W, seed, s)
    u = synth.initial_condition(n, seed)
    rom = _rom(C, "f64")
    assert _rel(_eval(rom, u)[0], oracle.nonlinear_full(C, u[0])) <= 1e-12
    rom.close()


@pytest.mark.parametrize("asym", [1.0, 1e-6])
def test_packed_rejects_non_skew(asym):
    n = 40
    seed = synth.seed_for(0) + 7300
    C = synth.skew_normal_tensor(n, seed)
    S = synth.normal(seed, 9, 0, n ** 3).reshape(n, n, n)
    S = S + S.transpose(2, 1, 0)  # symmetric in (i, k)
    bad = C + asym * np.linalg.norm(C) / np.linalg.norm(S) * S
    with pytest.raises(grom.GromError) as e:
        _rom(bad, "bf16")
    assert e.value.name == "INVALID_ARG"
    assert "skew" in str(e.value)


def test_packed_slab_upload():
    n = 70
    seed = synth.seed_for(0) + 7400
    C = synth.skew_normal_tensor(n, seed)
    u = synth.initial_condition(n, seed)
    rom = grom.Rom(n, "full", "f32x2", stiffness=synth.diag_stiffness(n), defer_tensor=True, layout="skew_packed")
    for i0, i1 in ((0, 30), (30, 31), (31, 70)):
        rom.upload_slab(i0, np.ascontiguousarray(C[i0:i1]))
    assert _rel(_eval(rom, u)[0], oracle.nonlinear_full(C, u[0])) <= 1e-12
    with pytest.raises(grom.GromError):
        rom.upload_slab(0, np.ascontiguousarray(C[0:1]))
    rom.close()


def test_packed_kernel_choice():
    # BF16 packed ROMs have the factored tensor-core kernel (K2P, tested in
    # test_gpu_k2p.py); the other storage types have none
    n = 64
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + 7500)
    rom = _rom(C, "f32", max_batch=32)
    with pytest.raises(grom.GromError) as e:
        rom.set_kernel("tensor")
    assert e.value.name == "UNSUPPORTED"
    rom.close()
    # batches beyond the tensor-core threshold, forced onto the streaming kernel
    rom = _rom(C, "bf16", max_batch=32)
    rom.set_kernel("stream")
    U = synth.initial_condition(n, 11, 0, 32)
    c = _eval(rom, U)
    for b in (0, 31):
        assert _rel(c[b], oracle.nonlinear_full(C, U[b])) <= 2e-2
    rom.close()


def test_packed_halves_the_footprint():
    n = 256
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + 7600)
    dense, packed = _rom(C, "bf16", layout="dense"), _rom(C, "bf16")
    tensor_dense = n * n * 256 * 2
    tensor_packed = n * n * 128 * 2
    assert dense.nbytes - packed.nbytes >= tensor_dense - tensor_packed - (64 << 20)
    dense.close()
    packed.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32x2", 1e-11), ("bf16", 2e-2)])
@pytest.mark.parametrize("batch", [1, 5])
def test_packed_trajectory_matches_oracle(storage, tol, batch):
    n, steps = 64, 40
    seed = synth.seed_for(0) + 7700
    C = synth.skew_normal_tensor(n, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, storage, max_batch=batch, nu=1e-2, dt=1e-3)
    tr = grom.Trajectories(rom, U0)
    E = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    inv = torch.empty_like(E)
    tr.step(steps, E, inv)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
    for b in range(batch):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= tol, (storage, b)
        assert H[b][6 * n] == steps
    tr.close()
    rom.close()


@pytest.mark.parametrize("layout", ["dense"])
def test_profiling_inside_graph_replays(layout):
    # 19 steps = two replays of the 8-step graph + 3 direct steps; every
    # streaming launch is timed, and timing does not change the result
    n = 96
    seed = synth.seed_for(0) + 7800
    C = synth.skew_normal_tensor(n, seed)
    u0 = synth.initial_condition(n, seed)
    rom = _rom(C, "bf16", layout=layout)
    t1 = grom.Trajectories(rom, u0)
    t1.step(19)
    rom.profile(True)
    t2 = grom.Trajectories(rom, u0)
    t2.step(19)
    ms, launches = rom.profile_read()
    rom.profile(False)
    assert launches == 19
    assert ms > 0.0
    np.testing.assert_array_equal(t1.get_state(), t2.get_state())
    t1.close()
    t2.close()
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
def test_step_host_paths_agree(layout):
    # grom_step_host with pinned buffers (one captured graph per call), with
    # device buffers (graph) and with pageable numpy buffers (direct launches)
    # gives the state grom_step gives, bit for bit
    n, batch = 80, 2
    seed = synth.seed_for(0) + 7900
    C = synth.skew_normal_tensor(n, seed)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, "bf16", layout=layout, max_batch=batch)
    ref = grom.Trajectories(rom, U0)
    ref.step(5)
    want = ref.get_state()[:, :n]

    pinned = torch.from_numpy(U0.copy()).pin_memory()
    t1 = grom.Trajectories(rom, U0)
    t1.step_host(1, pinned, pinned)
    t1.step_host(1, pinned, pinned)   # graph reused
    other = torch.empty_like(pinned).pin_memory()
    t1.step_host(3, pinned, other)    # new buffers and count: graph captured again
    np.testing.assert_array_equal(other.numpy(), want)

    dev = torch.from_numpy(U0.copy()).cuda()
    t2 = grom.Trajectories(rom, U0)
    for _ in range(5):
        t2.step_host(1, dev, dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), want)

    host = U0.copy()
    t3 = grom.Trajectories(rom, U0)
    for _ in range(5):
        t3.step_host(1, host, host)
    np.testing.assert_array_equal(host, want)
    for t in (ref, t1, t2, t3):
        t.close()
    rom.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32x2", 1e-12), ("f32", 1e-6), ("bf16", 1e-4)])
@pytest.mark.parametrize("batch", [1, 3])
def test_persistent_stepper_matches_single_steps(storage, tol, batch):
    # 40 steps in one persistent launch vs 40 single steps on the per-step
    # kernels (the finalize sums run in different orders: agreement to rounding)
    n = 96
    seed = synth.seed_for(0) + 8100
    C = synth.skew_normal_tensor(n, seed)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, storage, max_batch=batch, nu=1e-2, dt=1e-3)
    t1 = grom.Trajectories(rom, U0)
    t1.step(40)
    rom.set_kernel("stream")  # the streaming kernel and a separate finalize/step launch
    t2 = grom.Trajectories(rom, U0)
    for _ in range(40):
        t2.step(1)
    rom.set_kernel("auto")
    t3 = grom.Trajectories(rom, U0)
    for _ in range(40):
        t3.step(1)  # single-step calls on the persistent stepper: the bits of one long launch
    np.testing.assert_array_equal(t3.get_state(), t1.get_state())
    t3.close()
    H1, H2 = t1.get_state(), t2.get_state()
    for b in range(batch):
        assert _rel(H1[b][:n], H2[b][:n]) <= tol, (storage, b)
        assert H1[b][6 * n] == 40
    t1.close()
    t2.close()
    rom.close()


def test_persistent_stepper_outputs_and_chaining():
    # energies and invariants of a persistent launch against the oracle, and
    # three chained launches equal to one (the barrier word is reused)
    n, batch = 128, 2
    seed = synth.seed_for(0) + 8200
    C = synth.skew_normal_tensor(n, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, "f64", max_batch=batch, nu=1e-2, dt=1e-3)
    tr = grom.Trajectories(rom, U0)
    E = torch.empty((24, batch), dtype=torch.float64, device="cuda")
    inv = torch.empty_like(E)
    tr.step(24, E, inv)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
    for b in range(batch):
        h = ref.initial_history(U0[b])
        e_ref, inv_ref = ref.step(h, 24, want_energy=True, want_invariant=True)
        assert _rel(H[b][:n], h[:n]) <= 1e-11
        np.testing.assert_allclose(E.cpu().numpy()[:, b], e_ref, rtol=1e-11)
        assert np.max(np.abs(inv.cpu().numpy()[:, b])) <= 1e-10 * np.max(e_ref)
    t2 = grom.Trajectories(rom, U0)
    for _ in range(3):
        t2.step(8)
    np.testing.assert_array_equal(t2.get_state(), H)
    t2.close()
    tr.close()
    rom.close()


def test_persistent_stepper_falls_back_when_it_does_not_fit():
    # FP64 with 4 trajectories needs more shared memory than one CTA has: the
    # call takes the graph path and still matches the oracle
    n, batch = 1024, 4
    seed = synth.seed_for(0) + 8300
    C = synth.skew_normal_tensor(n, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, "f64", max_batch=batch, nu=1e-2, dt=1e-3)
    tr = grom.Trajectories(rom, U0)
    tr.step(8)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
    h = ref.initial_history(U0[3])
    ref.step(h, 8)
    assert _rel(H[3][:n], h[:n]) <= 1e-11
    tr.close()
    rom.close()
