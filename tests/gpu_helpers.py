"""Helpers for the GPU tests: run a generated problem through the C ABI."""
from __future__ import annotations

import numpy as np

import paper_1504_05046_gb300 as P


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_lib(prob, c_struct, C0, c_off, *, mode=P.BSMM_FP64, nslices=6, c_mask=None, schedule=P.BSMM_SCHED_FLOPS,
            max_ctas=0, ctas=None, costs=None, debug=1, plan=None, record_timings=0, cluster=0, stages=0,
            split_scale=0, ksplit=0, store_warps=0):
    """Plan (unless given) and execute on the GPU; returns (C result numpy, plan)."""
    import torch
    if plan is None:
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, c_mask,
                           mode=mode, nslices=nslices, schedule=schedule, max_ctas=max_ctas, debug_checks=debug,
                           record_timings=record_timings, cluster=cluster, stages=stages,
                           transa=int(getattr(prob, "transa", False)), transb=int(getattr(prob, "transb", False)),
                           split_scale=split_scale, ksplit=ksplit, store_warps=store_warps)
    if ctas is not None:
        P.bsmm_plan_set_ctas(plan, ctas)
    if costs is not None:
        P.bsmm_plan_set_costs(plan, costs)
    q = P.bsmm_plan_query(plan)
    assert np.array_equal(q["c_mask"], c_struct), "plan's C structure differs from the oracle's"
    A = to_dev(prob.A if prob.A.size else np.zeros(2))
    B = to_dev(prob.B if prob.B.size else np.zeros(2))
    C = to_dev(C0 if C0.size else np.zeros(2))
    ao, bo, co = to_dev(prob.a_off.astype(np.int64)), to_dev(prob.b_off.astype(np.int64)), to_dev(c_off.astype(np.int64))
    P.bsmm_execute(plan, prob.alpha, A, ao, B, bo, prob.beta, C, co)
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    out = C.cpu().numpy()
    return (out if C0.size else C0.copy()), plan
