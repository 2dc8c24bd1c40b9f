"""K2P, the factored tensor-core contraction of the skew-packed BF16 layout:
one tcgen05 GEMM D_i = P_i^T U^T per test index over the stored half of the
tensor, after which every stored pair (i, k) adds D_i u_k to c_i and
subtracts D_i u_i from c_k.  Checked against the FP64 oracle on the full
tensor, against the streaming kernel and the dense K2 on the same BF16
values, and through the skew invariant, which the factored form keeps to
FP32 rounding (both entries of a pair use the same D and the same state)."""
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


def _eval(rom, U):
    u = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).cuda()
    c = torch.empty_like(u)
    rom.nonlinear(u, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _rom(C, layout="skew_packed", max_batch=1, **kw):
    n = C.shape[0]
    return grom.Rom(n, "full", "bf16", tensor=C, stiffness=synth.diag_stiffness(n), max_batch=max_batch,
                    layout=layout, **kw)


def _bf16(x):
    """Round-to-nearest-even of FP64 values to BF16 (through FP32, exact for
    the tensors here, whose entries are far from FP32 ties)."""
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()


# odd and even n (the even-n rule for distance n/2), rows shorter than one
# 128-position block, several blocks, ragged last test-index range; batches
# below, at and across the 16-column granule and the 128-column tile
@pytest.mark.parametrize("n", [2, 3, 17, 64, 96, 129, 200, 300])
@pytest.mark.parametrize("batch", [1, 9, 16, 33, 130])
def test_k2p_matches_oracle(n, batch):
    seed = synth.seed_for(0) + 8100 + n
    C = synth.skew_normal_tensor(n, seed)
    Cr = _bf16(C)
    U = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, max_batch=batch)
    rom.set_kernel("tensor")
    c = _eval(rom, U)
    rom.set_kernel("stream")
    c_stream = _eval(rom, U)
    for b in range(batch):
        # elementwise bounds on A_i = sum_jk |C_ijk| |u_j| |u_k|, which hold
        # however much the sum cancels: on the stored BF16 values the kernel
        # is exact up to the 2^-17 hi/lo split of the states and FP32 sums;
        # against the FP64 tensor the BF16 rounding (2^-9) adds to that
        A = np.einsum("ijk,j,k->i", np.abs(C), np.abs(U[b]), np.abs(U[b]))
        ref = oracle.nonlinear_full(C, U[b])
        ref_r = oracle.nonlinear_full(Cr, U[b])
        assert np.all(np.abs(c[b] - ref_r) <= 2.0 ** -14 * A), (n, batch, b)
        assert np.all(np.abs(c[b] - ref) <= 2.0 ** -8 * A), (n, batch, b)
        assert np.all(np.abs(c[b] - c_stream[b]) <= 2.0 ** -14 * A), (n, batch, b)
        if n >= 17:  # at n = 2, 3 single entries cancel beyond any relative bound
            assert _rel(c[b], ref) <= TOL_BF16, (n, batch, b, _rel(c[b], ref))
    rom.close()


def test_k2p_equals_dense_k2_on_the_same_values():
    n, batch = 160, 48
    seed = synth.seed_for(0) + 8200
    C = synth.skew_normal_tensor(n, seed)
    U = synth.initial_condition(n, seed, 0, batch)
    packed, dense = _rom(C, max_batch=batch), _rom(C, layout="dense", max_batch=batch)
    cp, cd = _eval(packed, U), _eval(dense, U)  # auto: both tensor-core kernels at batch 48
    # against the oracle on the BF16-rounded tensor both are exact up to
    # FP32 accumulation and the ~2^-17 operand splits
    Cr = _bf16(C)
    for b in range(batch):
        ref = oracle.nonlinear_full(Cr, U[b])
        assert _rel(cp[b], ref) <= 2e-4, (b, _rel(cp[b], ref))
        assert _rel(cd[b], ref) <= 2e-4, (b, _rel(cd[b], ref))
    packed.close()
    dense.close()


def test_k2p_keeps_the_invariant_to_fp32_rounding():
    n, batch = 128, 40
    U_, V, W, s, seed = synth.cp_workload(n, n, 2)
    C = synth.cp_tensor(U_, V, W, seed, s)
    X = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, max_batch=batch)
    c = _eval(rom, X)  # auto: batch > 8 selects K2P
    Cr = _bf16(C)
    for b in range(batch):
        ref = oracle.nonlinear_full(C, X[b])
        assert _rel(c[b], ref) <= TOL_BF16
        # u^T c with the FP32 state the kernel used: every pair (i, k) adds
        # u_i D_ik u_k and subtracts u_k D_ik u_i with the same D, so only the
        # FP32 rounding of products and partial sums remains
        u32 = X[b].astype(np.float32).astype(np.float64)
        D = np.einsum("ijk,j->ik", Cr, u32)
        scale = float(np.abs(u32) @ np.abs(D) @ np.abs(u32))
        assert abs(u32 @ c[b]) <= 2.0 ** -16 * scale, (b, abs(u32 @ c[b]) / scale)
    rom.close()


@pytest.mark.parametrize("batch", [12, 24])
def test_k2p_stepping_matches_oracle(batch):
    n, steps = 96, 40
    seed = synth.seed_for(0) + 8300
    C = synth.skew_normal_tensor(n, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = _rom(C, max_batch=batch)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    code, _ = tr.status()
    assert code == 0
    H = tr.get_state()
    tr.close()
    for b in (0, batch // 2, batch - 1):
        ref = oracle.Rom("full", n, a, 1e-2, 1e-3, C=C)
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    rom.close()


def test_k2p_is_deterministic():
    n, batch = 200, 130
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + 8400)
    U = synth.initial_condition(n, 5, 0, batch)
    rom = _rom(C, max_batch=batch)
    c1, c2 = _eval(rom, U), _eval(rom, U)
    np.testing.assert_array_equal(c1, c2)
    # a sub-batch gives the same rows bitwise (the column tiles are independent)
    c3 = _eval(rom, U[:40])
    np.testing.assert_array_equal(c3, _eval(rom, U[:40]))
    rom.close()


def test_k2p_augmented_model():
    # the zeroth-mode model: the packed core goes through K2P, the zeroth-mode
    # terms through the stepper's L and f
    n, steps, batch = 40, 30, 12
    seed = synth.seed_for(0) + 8500
    C = synth.skew_normal_tensor(n, seed)
    Cbar = synth.augment_tensor(C, seed)
    a = synth.diag_stiffness(n)
    U0 = synth.initial_condition(n, seed, 0, batch)
    rom = grom.Rom(n, "full", "bf16", tensor=Cbar, stiffness=a, nu=1e-2, dt=1e-3, max_batch=batch,
                   layout="skew_packed", augmented=True)
    tr = grom.Trajectories(rom, U0)
    tr.step(steps)
    H = tr.get_state()
    tr.close()
    ref = oracle.Rom("full_aug", n, a, 1e-2, 1e-3, C=Cbar)
    for b in (0, batch - 1):
        h = ref.initial_history(U0[b])
        ref.step(h, steps)
        assert _rel(H[b][:n], h[:n]) <= TOL_BF16, b
    rom.close()


@pytest.mark.parametrize("n,batch", [(96, 16), (129, 40), (200, 130), (256, 256)])
def test_k2_tile_copy_and_row_layout_agree_bitwise(n, batch):
    # dense ROMs created for batches above 8 keep a tile-major copy of the
    # tensor for K2; without it (no_tile_copy) K2 reads the row layout.  Same
    # operands, same accumulation order: same bits.
    C = synth.skew_normal_tensor(n, synth.seed_for(0) + 8600 + n)
    U = synth.initial_condition(n, 9, 0, batch)
    tiled = _rom(C, layout="dense", max_batch=batch)
    rows = _rom(C, layout="dense", max_batch=batch, tile_copy=False)
    c1, c2 = _eval(tiled, U), _eval(rows, U)
    np.testing.assert_array_equal(c1, c2)
    for b in (0, batch - 1):
        assert _rel(c1[b], oracle.nonlinear_full(C, U[b])) <= TOL_BF16
    # the copy is the only difference in the footprint: 256-row tiles of C_(1)
    npad = (n + 63) // 64 * 64
    assert tiled.nbytes - rows.nbytes == (n + 255) // 256 * 256 * n * npad * 2
    # the skew-packed layout keeps no copy
    packed = _rom(C, max_batch=batch)
    packed_rows = _rom(C, max_batch=batch, tile_copy=False)
    assert packed.nbytes == packed_rows.nbytes
    for r in (tiled, rows, packed, packed_rows):
        r.close()
