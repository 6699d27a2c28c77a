"""The allocation-free tile entry point (bsmm_split_tile_noalloc).

Callers that cannot allocate device memory where they need the product use
bsmm_split_tile_noalloc: its scratch is a fixed device array inside the library,
so it must give the same bits as the allocating path (bsmm_execute on a 1 x 1 x 1
plan) and as the split oracle, call after call, although every call reuses (and
leaves behind) the previous call's scratch contents. This file is collected last so
that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

import bsmm_gen as G
from oracle import split as OS
import paper_1504_05046_gb300 as P

pytestmark = pytest.mark.gpu


def _reference(A, B, C0, m, n, k, s, alpha, beta):
    """The same tile task through a 1 x 1 x 1 plan and bsmm_execute."""
    import torch
    plan = P.bsmm_plan([m], [n], [k], np.ones((1, 1), np.uint8), np.ones((1, 1), np.uint8),
                       mode=P.BSMM_SPLIT_BF16, nslices=s)
    C = C0.clone()
    zero = torch.zeros(1, dtype=torch.int64, device="cuda")
    P.bsmm_execute(plan, alpha, A, zero, B, zero, beta, C, zero)
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    return C


def _oracle(A, B, C0, m, n, k, s, alpha, beta):
    """The split oracle on the 1 x 1 x 1 tiling (numpy arrays)."""
    one = np.ones((1, 1), np.uint8)
    z = np.zeros((1, 1), np.int64)
    prob = G.Problem("tile", np.array([m], np.int32), np.array([n], np.int32), np.array([k], np.int32), one, one,
                     z, z, A.reshape(-1).copy(), B.reshape(-1).copy(), alpha, beta)
    C = C0.reshape(-1).copy()
    OS.bsmm_split(prob, one, C, z, s)
    return C.reshape(m, n)


@pytest.mark.parametrize("shape", [(200, 150, 300, 6), (256, 256, 512, 6), (37, 70, 29, 3), (5, 33, 17, 1),
                                   (130, 40, 64, 2)])
def test_noalloc_matches_execute_and_oracle_on_two_calls(shape):
    import torch
    m, n, k, s = shape
    rng = np.random.default_rng(m + n + k)
    for call, (alpha, beta) in enumerate([(1.0, 0.0), (-0.5, 2.0)]):
        # two calls in a row with different data: the second must not see the first's scratch
        A = torch.from_numpy(rng.uniform(-1, 1, (m, k)) * 2.0 ** (call * 9)).cuda()
        B = torch.from_numpy(rng.uniform(-1, 1, (k, n))).cuda()
        C0 = torch.from_numpy(rng.uniform(-1, 1, (m, n))).cuda()
        want = _reference(A, B, C0, m, n, k, s, alpha, beta)
        got = C0.clone()
        P.bsmm_split_tile_noalloc(m, n, k, s, alpha, A, B, beta, got)
        assert torch.equal(got, want), f"call {call}: max diff {float((got - want).abs().max())}"
        ref = _oracle(A.cpu().numpy(), B.cpu().numpy(), C0.cpu().numpy(), m, n, k, s, alpha, beta)
        assert np.array_equal(got.cpu().numpy(), ref), f"call {call}: differs from the split oracle"
        # and the method's accuracy against an FP64 product
        exact = alpha * (A.cpu().numpy() @ B.cpu().numpy()) + (beta * C0.cpu().numpy() if beta else 0.0)
        err = np.linalg.norm(got.cpu().numpy() - exact) / np.linalg.norm(exact)
        assert err <= {1: 1e-1, 2: 1e-3, 3: 1e-5, 6: 1e-11}[s]


def test_noalloc_empty_inner_dimension_scales_c():
    """k = 0: C = beta * C, after a call that left a full tile's scratch behind."""
    import torch
    rng = np.random.default_rng(5)
    A = torch.from_numpy(rng.uniform(-1, 1, (64, 64))).cuda()
    B = torch.from_numpy(rng.uniform(-1, 1, (64, 64))).cuda()
    C = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    P.bsmm_split_tile_noalloc(64, 64, 64, 6, 1.0, A, B, 0.0, C)
    C0 = torch.from_numpy(rng.uniform(-1, 1, (40, 24))).cuda()
    got = C0.clone()
    P.bsmm_split_tile_noalloc(40, 24, 0, 6, 3.0, None, None, -0.5, got)
    assert torch.equal(got, -0.5 * C0)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_noalloc_reports_non_finite_input(bad):
    """A non-finite element in A is reported as BSMM_ERR_DEVICE (the error word read back
    from the library's array); the next call with finite data succeeds."""
    import torch
    rng = np.random.default_rng(6)
    A = torch.from_numpy(rng.uniform(-1, 1, (48, 32))).cuda()
    B = torch.from_numpy(rng.uniform(-1, 1, (32, 40))).cuda()
    C = torch.zeros((48, 40), dtype=torch.float64, device="cuda")
    A[7, 3] = bad
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_split_tile_noalloc(48, 40, 32, 6, 1.0, A, B, 0.0, C)
    assert ei.value.status == 6
    A[7, 3] = 0.25
    P.bsmm_split_tile_noalloc(48, 40, 32, 6, 1.0, A, B, 0.0, C)
    ref = _oracle(A.cpu().numpy(), B.cpu().numpy(), np.zeros((48, 40)), 48, 40, 32, 6, 1.0, 0.0)
    assert np.array_equal(C.cpu().numpy(), ref)


def test_noalloc_rejects_out_of_range_sizes():
    import torch
    A = torch.zeros((300, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((600, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((300, 8), dtype=torch.float64, device="cuda")
    for args in ((300, 8, 8, 6), (8, 8, 513, 6), (8, 300, 8, 6), (8, 8, 8, 0), (8, 8, 8, 7), (-1, 8, 8, 6)):
        with pytest.raises(P.BsmmError) as ei:
            P.bsmm_split_tile_noalloc(*args, 1.0, A, B, 0.0, C)
        assert ei.value.status == 1, args


def test_noalloc_wrapper_checks_tensors():
    """The binding refuses what the C entry point cannot check: a float32, host, strided
    or too small tensor never reaches the kernels."""
    import torch
    A = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    C = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    for bad in (A.float(), A.cpu(), torch.zeros((16, 32), dtype=torch.float64, device="cuda")[:, ::2],
                torch.zeros(100, dtype=torch.float64, device="cuda")):
        with pytest.raises(P.BsmmError) as ei:
            P.bsmm_split_tile_noalloc(16, 16, 16, 6, 1.0, bad, A, 0.0, C)
        assert ei.value.status == 1
