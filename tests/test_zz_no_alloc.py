"""The allocation-free tile entry point (bsmm_split_tile_noalloc) against the
plan-based entry point (bsmm_execute) on the same tile task.

Callers that cannot allocate device memory where they need the product use
bsmm_split_tile_noalloc: its scratch is a fixed device array inside the library,
so it must give the same bits as the allocating path, call after call, although
every call reuses (and leaves behind) the previous call's scratch contents.
This file is collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("shape", [(200, 150, 300, 6), (256, 256, 512, 6), (37, 70, 29, 3)])
def test_noalloc_matches_execute_on_two_calls(shape):
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
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}: max diff {float((got - want).abs().max())}"
        # and the method's accuracy against an FP64 product
        exact = alpha * (A.cpu().numpy() @ B.cpu().numpy()) + (beta * C0.cpu().numpy() if beta else 0.0)
        err = np.linalg.norm(got.cpu().numpy() - exact) / np.linalg.norm(exact)
        assert err <= (1e-11 if s == 6 else 1e-5)


def test_noalloc_rejects_oversize():
    import torch
    A = torch.zeros((300, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((300, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_split_tile_noalloc(300, 8, 8, 6, 1.0, A, B, 0.0, C)
    assert ei.value.status == 1
    with pytest.raises(P.BsmmError):
        P.bsmm_split_tile_noalloc(8, 8, 513, 6, 1.0, A, B, 0.0, C)
