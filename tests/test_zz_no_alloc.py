"""The allocation-free contraction entry point (grom_nonlinear_full_noalloc).

It exists for callers that cannot let a library allocate device memory
(HBM owned by another allocator, real-time loops).  It must give the same
result as grom_nonlinear on the same tensor, within the tolerances of the
parity tests, on consecutive calls that share its fixed scratch array.
This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32", "bf16"])
@pytest.mark.parametrize("n", [96, 200])
def test_noalloc_matches_nonlinear_on_two_calls(storage, n):
    grom.build()
    C = synth.skew_normal_tensor(n, 1234 + n)
    U = synth.initial_condition(n, 1234 + n, 0, 2)
    rom = grom.Rom(n, "full", storage, tensor=C, stiffness=synth.diag_stiffness(n))
    stored = grom.stored_layout(torch.from_numpy(C).cuda(), storage)
    for call in range(2):
        u = torch.from_numpy(U[call].copy()).cuda()
        c_ref = torch.empty_like(u)
        rom.nonlinear(u[None], c_ref[None])
        c = torch.full_like(u, float("nan"))
        grom.nonlinear_full_noalloc(n, storage, stored, u, c)
        torch.cuda.synchronize()
        assert torch.isfinite(c).all()
        assert _rel(c, c_ref) <= TOL[storage], (storage, n, call, _rel(c, c_ref))
    rom.close()


def test_noalloc_rejects_bad_arguments():
    grom.build()
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    t = torch.zeros(8 * 8 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(grom.GromError):
        grom.nonlinear_full_noalloc(0, "f64", t, u, u.clone())
    with pytest.raises(grom.GromError):
        grom.nonlinear_full_noalloc(8, "f64", t[1:], u, u.clone())  # misaligned tensor
