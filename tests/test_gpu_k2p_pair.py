"""K2P on SM pairs: the factored tensor-core contraction of the skew-packed
BF16 layout with one 256-row MMA (cta_group::2) over a cluster of two CTAs,
each holding its own 128-position block and one half (hi or lo) of the
states.  Checked against the FP64 oracle with the same elementwise bounds as
the single-CTA kernel, bitwise against the single-CTA kernel at the same tile
height (the same K=16 MMAs in the same order give each D entry, the epilogue
is the same), through
stepping and the skew invariant, and on block counts that need a padding
block (odd counts) or whose last block is half outside the stored row."""
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
    grom.load()
    assert torch.cuda.is_available()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()


def _rom(C, max_batch):
    n = C.shape[0]
    return grom.Rom(n, "full", "bf16", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=max_batch,
                    layout="skew_packed")


def _use(rom, batch, ctas, m=0):
    """Install the K2P kernel choice (1: single CTAs, 2: SM pairs) and tile
    height (0: the plan's rule) for the batch's bucket.  The height sets how
    the mirrored entries are grouped into FP32 window sums, so bitwise
    comparisons fix it."""
    rom.set_tuning({"batch": batch, "kernel": "tensor", "tile_m": m, "split_a": 0, "split_b": ctas})


def _common_height(rom, batch):
    """The tallest tile height both kernels admit for this batch (the least
    scratch); installs nothing that stays."""
    for m in range(32, 7, -1):
        try:
            _use(rom, batch, 1, m)
            _use(rom, batch, 2, m)
            return m
        except grom.GromError:
            continue
    raise AssertionError("no tile height admitted by both kernels")


def _eval(rom, U):
    u = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


# stored rows of 192 positions (n = 300: two blocks, the second half outside
# the row), 320 (n = 520: three blocks, the third half outside, and a padding
# block), 384 (n = 700: three blocks and a padding block); batches below, at
# and across the 16-column granule and the 128-column tile.  Four full blocks
# (n = 1024) are the full-size batched test's 256 trajectories.
@pytest.mark.parametrize("n,batch", [(300, 1), (300, 33), (520, 16), (520, 130), (700, 24)])
def test_pair_kernel_matches_oracle_and_single_ctas(n, batch):
    seed = synth.seed_for(0) + 8600 + n
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, batch)
    m = _common_height(rom, batch)
    _use(rom, batch, 1, m)
    c1 = _eval(rom, U)
    _use(rom, batch, 2, m)
    np.testing.assert_array_equal(_eval(rom, U), c1)
    _use(rom, batch, 2)  # the pair plan's own height
    c2 = _eval(rom, U)
    Cr = _bf16(C)
    absC = np.abs(C)
    for b in sorted({0, batch // 2, batch - 1}):
        A = np.einsum("ijk,j,k->i", absC, np.abs(U[b]), np.abs(U[b]))
        ref = oracle.nonlinear_full(C, U[b])
        ref_r = oracle.nonlinear_full(Cr, U[b])
        assert np.all(np.abs(c2[b] - ref_r) <= 2.0 ** -14 * A), (n, batch, b)
        assert np.all(np.abs(c2[b] - ref) <= 2.0 ** -8 * A), (n, batch, b)
        assert _rel(c2[b], ref) <= TOL_BF16, (n, batch, b, _rel(c2[b], ref))
    rom.close()


def test_pair_kernel_is_the_rule_and_deterministic():
    n, batch = 400, 300  # three column tiles, the last one ragged
    seed = synth.seed_for(0) + 8700
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, batch)
    c_rule = _eval(rom, U)
    np.testing.assert_array_equal(c_rule, _eval(rom, U))
    _use(rom, batch, 2)
    np.testing.assert_array_equal(_eval(rom, U), c_rule)
    m = _common_height(rom, batch)
    _use(rom, batch, 1, m)
    c1 = _eval(rom, U)
    _use(rom, batch, 2, m)
    np.testing.assert_array_equal(_eval(rom, U), c1)
    for b in (0, 150, batch - 1):
        assert _rel(c_rule[b], oracle.nonlinear_full(C, U[b])) <= TOL_BF16
    rom.close()


def test_pair_kernel_keeps_the_invariant_and_steps():
    n, batch, steps = 300, 40, 30
    seed = synth.seed_for(0) + 8800
    C = synth.skew_normal_tensor(n, seed)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, batch)
    _use(rom, batch, 2)
    c = _eval(rom, U0)
    Cr = _bf16(C)
    for b in (0, batch - 1):
        u32 = U0[b].astype(np.float32).astype(np.float64)
        D = np.einsum("ijk,j->ik", Cr, u32)
        scale = float(np.abs(u32) @ np.abs(D) @ np.abs(u32))
        assert abs(u32 @ c[b]) <= 2.0 ** -16 * scale, (b, abs(u32 @ c[b]) / scale)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    tr.close()
    a = synth.diag_stiffness(n)
    for b in (0, batch - 1):
        ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    rom.close()
