"""The kernels' bounded waits, exercised on the GPU without a fault, trap or hang: a
kernel whose mbarriers no thread arrives at runs out of its short limit, reports
BSMM_ERR_TIMEOUT through the device error word, and the abort flag releases the other
waiting warps long before their own (longer) limit; the context then runs a product
correctly."""
import time

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_release_every_warp():
    import torch
    limit = 50_000_000  # 50 ms; the other warps wait up to 1 s unless the abort reaches them
    with pytest.raises(P.BsmmError) as ei:  # first call also loads the module
        P.bsmm_selftest_wait(limit)
    assert ei.value.status == 4
    t0 = time.perf_counter()
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_selftest_wait(limit)
    dt = time.perf_counter() - t0
    assert ei.value.status == 4
    assert 0.045 <= dt < 0.5, dt
    torch.cuda.synchronize()


def test_context_usable_after_timeout():
    from gpu_helpers import run_lib
    with pytest.raises(P.BsmmError):
        P.bsmm_selftest_wait(2_000_000)
    prob = G.random_small(5, max_blocks=5, max_size=50)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(0))
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6)
    got, _ = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=6)
    assert np.array_equal(struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want))
