"""GPU parity of CP fitting (Sec. 2.3 ALS, Sec. 3.3 ALS-skew) against the
oracle's numpy ALS.

The test tensors hold multiples of 1/64 with at most 8 significant bits,
exactly representable in BF16, so the GPU's BF16 copy is the oracle's tensor and the
remaining differences are the hi/lo split of the Khatri-Rao operand (~2^-17)
and FP32 accumulation: one iteration agrees to 1e-4 relative.
"""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bf16_exact(shape, seed, skew=False):
    z = synth.normal(seed, 13, 0, int(np.prod(shape))).reshape(shape)
    lim = 127 if skew else 255  # at most 8 significant bits after the difference
    X = np.clip(np.round(z * 64.0), -lim, lim) / 64.0
    if skew:
        X = X - X.transpose(2, 1, 0)  # multiples of 1/64 up to 254/64: exact in BF16
    return X


def _factors(n, r, seed, k=3):
    return [synth.normal(seed, 20 + q, 0, n * r).reshape(n, r) for q in range(k)]


@pytest.mark.parametrize("n,r", [(24, 4), (64, 16), (40, 264)])
def test_one_plain_iteration_matches_oracle(n, r):
    X = _bf16_exact((n, n, n), 100 + n)
    F0 = _factors(n, r, 200 + r)
    als = grom.Als(X)
    F, res = als.fit(F0, 1)
    Fo, reso = oracle.cp_als(X, F0, 1)
    for q in range(3):
        assert _rel(F[q], Fo[q]) <= 1e-4, (n, r, q, _rel(F[q], Fo[q]))
    assert res[0] == pytest.approx(reso[0], rel=1e-4)
    als.close()


def test_plain_residuals_track_oracle_and_decrease():
    n, r, iters = 32, 6, 6
    X = _bf16_exact((n, n, n), 300)
    F0 = _factors(n, r, 301)
    als = grom.Als(X)
    F, res = als.fit(F0, iters)
    _, reso = oracle.cp_als(X, F0, iters)
    np.testing.assert_allclose(res, reso, rtol=1e-3)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(res, res[1:]))
    # continuing from the returned factors continues the same sequence
    _, res2 = als.fit(F, 2)
    _, reso2 = oracle.cp_als(X, F0, iters + 2)
    np.testing.assert_allclose(res2, reso2[iters:], rtol=1e-3)
    als.close()


@pytest.mark.parametrize("lam,subiters", [(0.5, 1), (0.25, 3)])
def test_als_skew_matches_oracle(lam, subiters):
    n, r, iters = 28, 8, 3
    X = _bf16_exact((n, n, n), 400, skew=True)
    A1, B1 = _factors(n, r, 401, 1)[0], _factors(n, r // 2, 402, 1)[0]
    als = grom.Als(X)
    (A1g, B1g), res = als.fit((A1, B1), iters, method="skew", lam=lam, subiters=subiters)
    (A1o, B1o), reso = oracle.cp_als_skew(X, A1, B1, iters, lam=lam, subiters=subiters)
    assert _rel(A1g, A1o) <= 1e-3 and _rel(B1g, B1o) <= 1e-3
    np.testing.assert_allclose(res, reso, rtol=1e-3)
    als.close()


def test_als_rejects_bad_arguments():
    n = 16
    X = _bf16_exact((n, n, n), 500, skew=True)
    als = grom.Als(X)
    with pytest.raises(grom.GromError) as e:
        als.fit((_factors(n, 3, 1, 1)[0], _factors(n, 1, 2, 1)[0]), 1, method="skew")
    assert e.value.name == "INVALID_ARG"
    als.close()


def test_one_context_many_ranks():
    # scratch and factor buffers follow the rank up and down
    n = 40
    X = _bf16_exact((n, n, n), 600)
    als = grom.Als(X)
    for r in (40, 4, 264, 16):
        F0 = _factors(n, r, 700 + r)
        F, res = als.fit(F0, 1)
        Fo, reso = oracle.cp_als(X, F0, 1)
        assert _rel(F[0], Fo[0]) <= 1e-4, r
        assert res[0] == pytest.approx(reso[0], rel=1e-4)
    ms, calls, solve = als.stats()
    assert calls == 16 and ms > 0.0 and solve > 0.0  # 3 updates + 1 residual MTTKRP per iteration
    als.close()


@pytest.mark.parametrize("method", ["plain", "skew"])
def test_ridge_matches_oracle(method):
    n, r, iters, ridge = 30, 8, 2, 1e-3
    X = _bf16_exact((n, n, n), 800, skew=method == "skew")
    als = grom.Als(X)
    if method == "plain":
        F0 = _factors(n, r, 801)
        F, res = als.fit(F0, iters, ridge=ridge)
        Fo, reso = oracle.cp_als(X, F0, iters, ridge=ridge)
        for q in range(3):
            assert _rel(F[q], Fo[q]) <= 1e-4, q
    else:
        A1, B1 = _factors(n, r, 802, 1)[0], _factors(n, r // 2, 803, 1)[0]
        (A1g, B1g), res = als.fit((A1, B1), iters, method="skew", ridge=ridge)
        (A1o, B1o), reso = oracle.cp_als_skew(X, A1, B1, iters, ridge=ridge)
        assert _rel(A1g, A1o) <= 1e-3 and _rel(B1g, B1o) <= 1e-3
    np.testing.assert_allclose(res, reso, rtol=1e-3)
    als.close()
