"""Host-side logic of the serving loop (grom_serve) in its simulation mode:
no GPU is touched, a batched step costs step_seconds of virtual time."""
import numpy as np
import pytest

import paper_2311_03694_gb300 as grom


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grom.build()
    grom.load()


def _slot_bytes(n):
    return 8 * (7 * n + 4)


def test_every_request_completes_with_its_horizon():
    s = grom.Server(10 ** 9, quantum=8, simulate=True)
    a = s.add_simulated(16, 10_000, 4, 1e-4)
    b = s.add_simulated(32, 20_000, 2, 2e-4)
    rng = np.random.default_rng(0)
    count = 40
    models = rng.integers(0, 2, count)
    horizons = rng.integers(1, 60, count)
    arrivals = np.sort(rng.random(count) * 0.01)
    u0 = [np.zeros(s.n[m]) for m in models]
    out = s.serve(models, horizons, arrivals, u0)
    assert np.all(out["status"] == 0)
    np.testing.assert_array_equal(out["steps"], horizons)
    assert np.all(out["t_admit"] >= arrivals - 1e-12)
    assert np.all(out["t_done"] >= out["t_admit"])
    assert out["stats"]["trajectory_steps"] == horizons.sum()
    assert out["stats"]["peak_active"] <= 6
    assert a == 0 and b == 1


def test_fifo_per_model_and_slot_limit():
    s = grom.Server(10 ** 9, quantum=4, simulate=True)
    s.add_simulated(8, 0, 2, 1e-3)
    count = 6
    out = s.serve([0] * count, [8] * count, [0.0] * count, [np.zeros(8)] * count)
    # two slots: requests are admitted in arrival order, two at a time
    adm = out["t_admit"]
    assert np.all(np.diff(adm) >= 0)
    assert adm[0] == adm[1] < adm[2] == adm[3] < adm[4] == adm[5]
    assert out["stats"]["peak_active"] == 2


def test_budget_bounds_concurrency():
    n = 8
    rom_bytes = 1000
    budget = rom_bytes + 4 * _slot_bytes(n) + 3 * _slot_bytes(n)  # pool of 4 + room for 3 states
    s = grom.Server(budget, quantum=4, simulate=True)
    s.add_simulated(n, rom_bytes, 4, 1e-3)
    out = s.serve([0] * 8, [12] * 8, [0.0] * 8, [np.zeros(n)] * 8)
    assert np.all(out["status"] == 0)
    assert out["stats"]["peak_active"] == 3
    assert out["stats"]["peak_bytes"] <= budget


def test_model_over_budget_is_refused():
    s = grom.Server(10_000, quantum=4, simulate=True)
    with pytest.raises(grom.GromError) as ei:
        s.add_simulated(64, 9_000, 8, 1e-3)
    assert ei.value.name == "BUDGET"


def test_request_that_can_never_fit_is_rejected():
    n = 8
    s = grom.Server(1000 + 2 * _slot_bytes(n) + _slot_bytes(n) - 1, quantum=4, simulate=True)
    s.add_simulated(n, 1000, 2, 1e-3)
    out = s.serve([0, 0], [4, 4], [0.0, 0.0], [np.zeros(n)] * 2)
    assert list(out["status"]) == [6, 6]  # GROM_ERR_BUDGET


def test_continuous_batching_admits_while_others_run():
    s = grom.Server(10 ** 9, quantum=4, simulate=True)
    s.add_simulated(8, 0, 4, 1e-3)
    # a long request starts alone; a short one arriving later joins it and
    # finishes first
    out = s.serve([0, 0], [400, 8], [0.0, 0.05], [np.zeros(8)] * 2)
    assert out["t_admit"][1] < out["t_done"][0]
    assert out["t_done"][1] < out["t_done"][0]


def test_idle_server_waits_for_arrivals():
    s = grom.Server(10 ** 9, quantum=4, simulate=True)
    s.add_simulated(8, 0, 4, 1e-3)
    out = s.serve([0], [4], [2.5], [np.zeros(8)])
    assert out["t_admit"][0] == pytest.approx(2.5)
    assert out["t_done"][0] == pytest.approx(2.5 + 4e-3)


def test_bad_requests_are_rejected():
    s = grom.Server(10 ** 9, quantum=4, simulate=True)
    s.add_simulated(8, 0, 4, 1e-3)
    with pytest.raises(grom.GromError):
        s.serve([1], [4], [0.0], [np.zeros(8)])  # unknown model
    with pytest.raises(grom.GromError):
        s.serve([0], [0], [0.0], [np.zeros(8)])  # horizon < 1
