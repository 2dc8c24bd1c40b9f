"""K2, the tcgen05 tensor-core contraction over the Khatri-Rao product of the
states (BF16 storage, FP32 accumulation in tensor memory), against the FP64
oracle and against the streaming kernel on the same stored tensor."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _eval(rom, U):
    u = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("n", [64, 100, 200])
@pytest.mark.parametrize("batch", [1, 5, 16, 17, 48, 130, 256, 300])
def test_k2_matches_oracle(n, batch):
    C = synth.skew_normal_tensor(n, 500 + n)
    U = synth.initial_condition(n, 500 + n, 0, batch)
    rom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=batch)
    rom.set_kernel("tensor")
    c = _eval(rom, U)
    rom.set_kernel("stream")
    c_stream = _eval(rom, U)
    for b in range(batch):
        ref = oracle.nonlinear_full(C, U[b])
        assert _rel(c[b], ref) <= TOL_BF16, (n, batch, b, _rel(c[b], ref))
        # same stored tensor: the two kernels differ only by the BF16 rounding of u_j u_k
        assert _rel(c[b], c_stream[b]) <= 1e-2
    rom.close()


def test_k2_cp_structured_workload_and_invariant():
    n, batch = 128, 40
    U, V, W, s, seed = synth.cp_workload(n, n, 2)
    C = synth.cp_tensor(U, V, W, seed, s)
    X = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=batch)
    c = _eval(rom, X)  # auto: batch > 8 selects the tensor-core kernel
    for b in range(batch):
        ref = oracle.nonlinear_full(C, X[b])
        assert _rel(c[b], ref) <= TOL_BF16
        # invariant u^T c(u) = 0 holds to the BF16 rounding of the KR products
        scale = np.abs(X[b]) @ np.abs(c[b]) + np.linalg.norm(X[b]) * np.linalg.norm(ref)
        assert abs(X[b] @ c[b]) <= 2.0 ** -7 * scale


def test_k2_stepping_batch_matches_oracle():
    n, batch, steps = 96, 24, 40
    C = synth.skew_normal_tensor(n, 77)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, 77, 0, batch)
    rom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=a, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    for b in (0, 7, batch - 1):
        ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16


def test_k2_is_deterministic():
    n, batch = 80, 33
    C = synth.skew_normal_tensor(n, 3)
    U = synth.initial_condition(n, 3, 0, batch)
    rom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=batch)
    rom.set_kernel("tensor")
    np.testing.assert_array_equal(_eval(rom, U), _eval(rom, U))
