"""GPU parity of the SVD-ROM (Sec. 4.4.2) against the FP64 oracle.

The library streams the slices V[i][r][k] with the middle index weighted by
beta = sigma o (U^T u); tolerances are the per-evaluation ones of the dense
contraction (1e-12 FP64 and F32X2, 1e-5 FP32, 2e-2 BF16).  Cases cover
dense and skew-packed slices, ranks below and above one streaming chunk,
odd n, batches beyond one kernel pass, stepping, and the full-rank SVD of a
tensor (which reproduces the G-ROM).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}


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


def _rom(n, factors, storage, layout="dense", max_batch=1, **kw):
    return grom.Rom(n, "svd", storage, factors=factors, stiffness=synth.diag_stiffness(n), max_batch=max_batch,
                    layout=layout, **kw)


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
@pytest.mark.parametrize("n,rank", [(2, 1), (17, 5), (64, 64), (129, 40), (96, 300)])
def test_svd_matches_oracle(layout, storage, n, rank):
    seed = synth.seed_for(0) + 9000 + n + rank
    f = synth.svd_workload(n, rank, seed)
    batch = 3
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(n, f, storage, layout, max_batch=batch)
    c = _eval(rom, U0)
    for b in range(batch):
        ref = oracle.nonlinear_svd(*f, U0[b])
        assert _rel(c[b], ref) <= TOL[storage], (layout, storage, n, rank, b, _rel(c[b], ref))
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
def test_svd_many_passes(layout):
    n, rank, batch = 80, 24, 13
    seed = synth.seed_for(0) + 9100
    f = synth.svd_workload(n, rank, seed)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(n, f, "f32", layout, max_batch=batch)
    c = _eval(rom, U0)
    for b in (0, 7, 8, 12):
        assert _rel(c[b], oracle.nonlinear_svd(*f, U0[b])) <= 1e-5, b
    rom.close()


@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
def test_full_rank_svd_reproduces_g_rom(layout):
    # factors of the exact SVD of a skew tensor (oracle helper): the SVD-ROM
    # at full rank is the G-ROM
    n = 24
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + 9200)
    f = oracle.svd_factors(C, n)
    u = synth.initial_condition(n, 3)
    rom = _rom(n, f, "f64", layout)
    assert _rel(_eval(rom, u)[0], oracle.nonlinear_full(C, u[0])) <= 1e-12
    rom.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("bf16", 2e-2)])
@pytest.mark.parametrize("layout", ["dense", "skew_packed"])
@pytest.mark.parametrize("batch", [1, 3])
def test_svd_trajectory_matches_oracle(storage, tol, layout, batch):
    n, rank, steps = 64, 16, 40
    seed = synth.seed_for(0) + 9300
    f = synth.svd_workload(n, rank, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(n, f, storage, layout, max_batch=batch, nu=1e-2, dt=1e-3)
    tr = grom.Trajectories(rom, U0)
    E = torch.empty((steps, batch), dtype=torch.float64, device="cuda")
    tr.step(steps, E)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    ref = oracle.Rom("svd", n, a, 1e-2, 1e-3, factors=f)
    for b in range(batch):
        h = ref.initial_history(U0[b])
        e_ref, _ = ref.step(h, steps, want_energy=True)
        assert _rel(H[b][:n], h[:n]) <= tol, (storage, layout, b)
        np.testing.assert_allclose(E.cpu().numpy()[:, b], e_ref, rtol=max(tol, 1e-12))
    tr.close()
    rom.close()


def test_svd_packed_rejects_non_skew_slices():
    n, rank = 30, 4
    U, s, V = synth.svd_workload(n, rank, 11)
    V = V + np.abs(V)  # no longer skew
    with pytest.raises(grom.GromError) as e:
        _rom(n, (U, s, np.ascontiguousarray(V)), "bf16", "skew_packed")
    assert e.value.name == "INVALID_ARG"
