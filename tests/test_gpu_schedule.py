"""What the learned cost model gains: trained on unit timings of clustered products
(irregular log-uniform blocks, dense clusters of tiles), evaluated on a held-out
product against the flop-count schedule, at the clustered workload's full size (M = N =
24576, K = 49152). The makespans are medians of 5 timed runs each; the learned schedule
must be no slower than the flop-count one, and the result bits are the same either way."""
import json
import os

import numpy as np
import pytest

import bsmm_gen as G
import paper_1504_05046_gb300 as P
from paper_1504_05046_gb300 import costmodel as CM

pytestmark = pytest.mark.gpu
N = 24576


def _setup(seed):
    import torch
    prob = G.make_problem("clustered", seed, N, lo=16, hi=512, nclusters=40, cluster_density=0.10)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, record_timings=1, profile=1)
    q = P.bsmm_plan_query(plan)
    off, tot = G.layout_arena(q["c_mask"], prob.row_sizes, prob.col_sizes)
    d = lambda x: torch.from_numpy(x).cuda()
    A, B, ao, bo, co = d(prob.A), d(prob.B), d(prob.a_off), d(prob.b_off), d(off)
    C = torch.zeros(max(tot, 2), dtype=torch.float64, device="cuda")

    def run():
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
    return plan, run, C


def test_learned_schedule_vs_flop_count():
    rows = []
    for seed in (11, 12, 13):
        plan, run, _ = _setup(seed)
        run()
        rows.append(CM.training_rows(plan, CM.unit_times(plan, run, repeats=3)))
    mlp, loss = CM.fit(rows, steps=2000, lr=3e-3)
    assert loss < 0.5

    plan, run, C = _setup(14)
    run()
    times = CM.unit_times(plan, run, repeats=3)
    _, flops = P.bsmm_plan_features(plan)
    CM.apply_flops(plan)
    t_flops = CM.makespan_ms(plan, run, repeats=5)
    ref = C.cpu().numpy().copy()
    CM.apply(plan, mlp)
    t_mlp = CM.makespan_ms(plan, run, repeats=5)
    assert np.array_equal(C.cpu().numpy(), ref), "the schedule changed result bits"
    # predicted costs as the plan now holds them
    import torch
    feats, _ = P.bsmm_plan_features(plan)
    y = torch.zeros(len(feats), dtype=torch.float32, device="cuda")
    P.bsmm_mlp_predict(mlp, torch.from_numpy(feats).cuda(), y)
    err_mlp = CM.prediction_error(plan, times, np.exp(y.cpu().numpy().astype(np.float64)))
    err_flops = CM.prediction_error(plan, times, np.maximum(flops, 1.0))
    record = {"workload": f"clustered M=N={N} K={2 * N}, log-uniform blocks [16,512], 40 clusters at 10%",
              "train_seeds": [11, 12, 13], "eval_seed": 14, "train_loss": loss, "makespan_ms_flops": t_flops,
              "makespan_ms_mlp": t_mlp, "log_rms_err_flops": err_flops, "log_rms_err_mlp": err_mlp}
    out = os.environ.get("BSMM_SCHEDULE_RECORD")
    if out:
        with open(out, "w") as f:
            json.dump(record, f, indent=1)
    print(record)
    assert err_mlp < err_flops
    assert t_mlp <= t_flops


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_unit_records_of_column_block_groups(cluster):
    """Timing records of groups of 1, 2 or 4 CTAs: every unit that ran has a start and a
    positive time (the longest of its group's CTAs), no longer than the whole contraction,
    and the records are rewritten, not accumulated, by the next execute."""
    import torch
    prob = G.make_problem("clustered", 3, 2000, lo=16, hi=160, nclusters=5, cluster_density=0.3)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, record_timings=1, profile=1, cluster=cluster)
    q = P.bsmm_plan_query(plan)
    off, tot = G.layout_arena(q["c_mask"], prob.row_sizes, prob.col_sizes)
    d = lambda x: torch.from_numpy(x).cuda()
    A, B, ao, bo, co = d(prob.A), d(prob.B), d(prob.a_off), d(prob.b_off), d(off)
    C = torch.zeros(max(tot, 2), dtype=torch.float64, device="cuda")
    spans = []
    for _ in range(2):
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
        torch.cuda.synchronize()
        s, e, cta = P.bsmm_plan_timings(plan)
        ms = P.bsmm_plan_kernel_ms(plan)[2]
        ran = s > 0
        assert ran.all()
        assert (e[ran] > s[ran]).all()
        assert ((e[ran] - s[ran]) <= ms * 1e6 * 1.05 + 1e4).all()
        spans.append((e - s)[ran].sum())
    assert spans[1] < 1.5 * spans[0]
