"""grom_serve on the GPU: continuous batching of mixed-model requests.  Each
result is bitwise the same as the same request served alone by a server with
the same pools (every quantum steps a pool as one batch of all its slots, so
the kernels' plan and summation order do not depend on the other requests),
and equals the request stepped on its own (batch 1, another kernel plan)
within the parity tolerance."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2311_03694_gb300 as grom  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def models():
    grom.build()
    nf, nc, r = 64, 48, 12
    Cf = synth.skew_normal_tensor(nf, 21)
    U, V, W, _, seed = synth.cp_workload(nc, r, 1)
    s1, s2, s3, s4 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    roms = {
        "full_bf16": grom.Rom(nf, "full", "bf16", tensor=Cf, stiffness=synth.diag_stiffness(nf), max_batch=12,
                              stream=s1),
        "cp_f64": grom.Rom(nc, "cp_skew", "f64", factors=(U, V, W), stiffness=synth.diag_stiffness(nc),
                           max_batch=20, stream=s2),
        "full_f64": grom.Rom(nf, "full", "f64", tensor=Cf, stiffness=synth.diag_stiffness(nf), max_batch=4,
                             stream=s3),
        # skew-packed BF16: 12 slots step through the factored tensor-core kernel
        "packed_bf16": grom.Rom(nf, "full", "bf16", tensor=Cf, stiffness=synth.diag_stiffness(nf), max_batch=12,
                                stream=s4, layout="skew_packed"),
    }
    return roms, (Cf, (U, V, W))


def test_mixed_requests_match_alone(models):
    roms, (Cf, fac) = models
    srv = grom.Server(150 * 2 ** 30, quantum=8)
    ids = [srv.add_rom(roms["full_bf16"], 12), srv.add_rom(roms["cp_f64"], 20), srv.add_rom(roms["full_f64"], 4),
           srv.add_rom(roms["packed_bf16"], 12)]
    rng = np.random.default_rng(3)
    count = 80
    which = rng.integers(0, 4, count)
    horizons = rng.integers(5, 120, count)
    arrivals = np.sort(rng.random(count) * 0.02)
    n_of = [64, 48, 64, 64]
    u0s = [synth.initial_condition(n_of[w], 100 + q)[0] for q, w in enumerate(which)]
    out = srv.serve([ids[w] for w in which], horizons, arrivals, u0s, want_final=True)
    assert np.all(out["status"] == 0), out["status"]
    np.testing.assert_array_equal(out["steps"], horizons)
    assert out["stats"]["peak_active"] > 1
    names = ["full_bf16", "cp_f64", "full_f64", "packed_bf16"]
    tol = {"full_bf16": 1e-5, "cp_f64": 1e-11, "full_f64": 1e-12, "packed_bf16": 1e-5}
    alone_srv = grom.Server(150 * 2 ** 30, quantum=8)
    alone_ids = [alone_srv.add_rom(roms["full_bf16"], 12), alone_srv.add_rom(roms["cp_f64"], 20),
                 alone_srv.add_rom(roms["full_f64"], 4), alone_srv.add_rom(roms["packed_bf16"], 12)]
    for q in range(0, count, 3):
        one = alone_srv.serve([alone_ids[which[q]]], [horizons[q]], [0.0], [u0s[q]], want_final=True)
        assert one["status"][0] == 0
        np.testing.assert_array_equal(one["final"][0], out["final"][q], err_msg="request %d (%s)" % (
            q, names[which[q]]))
    alone_srv.close()
    for q in range(0, count, 3):
        rom = roms[names[which[q]]]
        tr = grom.Trajectories(rom, u0s[q][None, :])
        tr.step(int(horizons[q]))
        alone = tr.get_state()[0][:rom.n]
        tr.close()
        assert _rel(out["final"][q], alone) <= tol[names[which[q]]], (q, names[which[q]])
    # and against the FP64 oracle for the FP64 models
    for q in range(count):
        if names[which[q]] == "full_f64" and horizons[q] < 60:
            ref = oracle.Rom("full", 64, synth.diag_stiffness(64), 1e-2, 1e-3, C=Cf)
            h = ref.initial_history(u0s[q])
            ref.step(h, int(horizons[q]))
            assert _rel(out["final"][q], h[:64]) <= 1e-11
    srv.close()


def test_budget_limits_admission_on_gpu(models):
    roms, _ = models
    rom = roms["cp_f64"]
    slot = 8 * (7 * rom.n + 4)
    budget = rom.nbytes + 20 * slot + 2 * slot  # room for two trajectory states
    srv = grom.Server(budget, quantum=8)
    m = srv.add_rom(rom, 20)
    count = 6
    u0s = [synth.initial_condition(rom.n, 7 + q)[0] for q in range(count)]
    out = srv.serve([m] * count, [16] * count, [0.0] * count, u0s, want_final=True)
    assert np.all(out["status"] == 0)
    assert out["stats"]["peak_active"] == 2
    srv.close()
