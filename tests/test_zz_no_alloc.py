"""The allocation-free contraction entry point (grom_nonlinear_full_noalloc).

Some callers cannot let a library allocate device memory: programs whose HBM
is owned by another allocator (a framework's caching allocator that reserves
memory up front, a fixed start-up budget) and real-time loops, where an
allocation can synchronise the device or stall for an unbounded time.  The
entry point runs the same streaming kernel as grom_nonlinear with its
scratch in a fixed array inside the library.  Its results must equal the
FP64 oracle within the parity tolerances and grom_nonlinear bit for bit
(same plan, same fixed summation order), on consecutive calls of different
sizes that share the fixed array.  This file sorts last so that a run
stopping at the first failure has run every other test first; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
def test_noalloc_matches_oracle_and_nonlinear_on_consecutive_calls(storage):
    # sizes alternate so that a call reading partial sums left by the
    # previous one (another n, another partition) would show
    grom.build()
    cases = {}
    for n in (200, 96):
        C = synth.skew_normal_tensor(n, 1234 + n)
        rom = grom.Rom(n, "full", storage, tensor=C, stiffness=synth.diag_stiffness(n), max_batch=1)
        cases[n] = (C, rom, grom.stored_layout(torch.from_numpy(C).cuda(), storage))
    for call, n in enumerate((200, 96, 200, 96)):
        C, rom, stored = cases[n]
        u_h = synth.initial_condition(n, 99 + call)[0]
        u = torch.from_numpy(u_h.copy()).cuda()
        c_ref = torch.empty_like(u)
        rom.nonlinear(u[None], c_ref[None])
        c = torch.full_like(u, float("nan"))
        grom.nonlinear_full_noalloc(n, storage, stored, u, c)
        grom.nonlinear_full_noalloc_status()
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        assert np.isfinite(got).all()
        assert torch.equal(c, c_ref), (storage, n, call, float((c - c_ref).abs().max()))
        err = _rel(got, oracle.nonlinear_full(C, u_h))
        assert err <= TOL[storage], (storage, n, call, err)
    for _, rom, _ in cases.values():
        rom.close()


def test_noalloc_rejects_bad_arguments():
    grom.build()
    n = 8
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    t = torch.zeros(n * n * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(grom.GromError):
        grom.nonlinear_full_noalloc(0, "f64", t, u, u.clone())
    with pytest.raises(grom.GromError):  # full length but 8 bytes off a 16-byte boundary (library check)
        t2 = torch.zeros(n * n * 64 + 1, dtype=torch.float64, device="cuda")
        grom.nonlinear_full_noalloc(n, "f64", t2[1:], u, u.clone())
    with pytest.raises(grom.GromError):  # too short for n*n stored rows (binding check)
        grom.nonlinear_full_noalloc(n, "f64", t[: n * n * 64 - 64], u, u.clone())
    with pytest.raises(grom.GromError):  # state on the host
        grom.nonlinear_full_noalloc(n, "f64", t, u.cpu(), u.clone())
    with pytest.raises(grom.GromError):  # wrong state length
        grom.nonlinear_full_noalloc(n, "f64", t, u[: n - 1], u.clone())
    with pytest.raises(grom.GromError):
        grom.nonlinear_full_noalloc(n, "f64", t, u, torch.zeros(n + 1, dtype=torch.float64, device="cuda"))
    c = torch.full_like(u, float("nan"))
    grom.nonlinear_full_noalloc(n, "f64", t, u, c)  # the zero tensor gives c = 0
    grom.nonlinear_full_noalloc_status()
    assert torch.equal(c, torch.zeros_like(c))
