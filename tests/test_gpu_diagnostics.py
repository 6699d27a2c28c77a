"""GPU diagnostics through the C ABI: the measured FP64 rates (the FP64 path's roofline
denominators) and the per-kernel times a profiled plan averages over its executes."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
import paper_1504_05046_gb300 as P
from helpers import c_arena

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    """GB300: 152 SMs at up to 2.07 GHz. The FP64 rates must be positive and below a
    generous ceiling (a rate far above it would mean the kernels did no work); so must
    the INT8 mma.sync rate (far below the 4.5 POP/s that dense FP8 reaches on tcgen05)."""
    r = P.bsmm_measure_rates()
    for key in ("dfma", "dmma"):
        assert 0.05 < r[key] < 5.0, r
    assert 1.0 < r["imma"] < 5000.0, r


def test_kernel_ms_means_over_the_executes_since_the_last_read():
    import torch
    from gpu_helpers import to_dev
    prob = G.make_problem("nonuniform_dense", 3, 1500, lo=64, hi=200)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, profile=1)
    A, B, ao, bo, co = to_dev(prob.A), to_dev(prob.B), to_dev(prob.a_off), to_dev(prob.b_off), to_dev(off)
    C = to_dev(C0)
    with pytest.raises(P.BsmmError):
        P.bsmm_plan_kernel_ms(plan)  # nothing recorded yet
    singles = []
    for _ in range(4):
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
        singles.append(P.bsmm_plan_kernel_ms(plan))
    again = P.bsmm_plan_kernel_ms(plan)  # no execute since: the last execute's times
    assert np.allclose(again, singles[-1])
    for _ in range(4):
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
    mean4 = np.array(P.bsmm_plan_kernel_ms(plan))
    assert len(mean4) == len(singles[0]) == 3  # exponents/scales/classes, slicing, contraction
    assert (mean4 > 0).all()
    # the mean of four executes lies within the range the single executes span (generously)
    lo, hi = np.min(singles, axis=0), np.max(singles, axis=0)
    assert (mean4 >= 0.5 * lo).all() and (mean4 <= 2.0 * hi).all()
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
