"""Learned task-cost schedule: collect unit timings, train the MLP, re-pack a plan.

Host orchestration only: the timings come from the contraction kernels' own
%globaltimer records (bsmm_plan_timings), training runs in the library's MLP kernels
(bsmm_mlp_fit) and prediction in its inference kernel (bsmm_plan_predict_costs).
"""
from __future__ import annotations

import numpy as np

from . import (bsmm_mlp_create, bsmm_mlp_fit, bsmm_plan_features, bsmm_plan_kernel_ms, bsmm_plan_predict_costs,
               bsmm_plan_query, bsmm_plan_set_costs, bsmm_plan_timings)


def unit_times(plan, run, repeats: int = 3) -> np.ndarray:
    """Median duration (ns) of every work unit over `repeats` runs; `run()` executes the
    plan once (built with record_timings=1)."""
    import torch
    rows = []
    for _ in range(repeats):
        run()
        torch.cuda.synchronize()
        s, e, _ = bsmm_plan_timings(plan)
        rows.append((e - s).astype(np.float64))
    return np.median(np.stack(rows), axis=0)


def training_rows(plan, times_ns):
    """(features float32 [n x F], log unit time float32 [n]) for the units that ran."""
    feats, _ = bsmm_plan_features(plan)
    ok = times_ns > 0
    return feats[ok].astype(np.float32), np.log(times_ns[ok]).astype(np.float32)


def fit(rows, steps: int = 2000, lr: float = 3e-3, seed: int = 0):
    """Train a fresh model on the concatenated rows [(X, t), ...]; returns (mlp, loss)."""
    import torch
    X = torch.from_numpy(np.concatenate([r[0] for r in rows])).cuda()
    t = torch.from_numpy(np.concatenate([r[1] for r in rows])).cuda()
    mlp = bsmm_mlp_create(seed)
    loss = bsmm_mlp_fit(mlp, X, t, steps, lr)
    return mlp, loss


def apply(plan, mlp):
    """Re-pack `plan` with the model's predicted unit times as costs."""
    bsmm_plan_predict_costs(plan, mlp)


def apply_flops(plan):
    """Re-pack `plan` with the flop-count costs (the fallback schedule)."""
    _, flops = bsmm_plan_features(plan)
    bsmm_plan_set_costs(plan, np.maximum(flops, 1.0))


def makespan_ms(plan, run, repeats: int = 5) -> float:
    """Median device time of the contraction kernel (last kernel of the plan's execute;
    the plan must be built with profile=1)."""
    import torch
    ms = []
    for _ in range(repeats):
        run()
        torch.cuda.synchronize()
        ms.append(bsmm_plan_kernel_ms(plan)[-1])
    return float(np.median(ms))


def prediction_error(plan, times_ns, costs) -> float:
    """RMS error of log(cost) against log(measured time) after the best constant offset
    (a cost model only has to rank and proportion the units)."""
    ok = times_ns > 0
    d = np.log(np.asarray(costs, np.float64)[ok]) - np.log(times_ns[ok])
    return float(np.sqrt(np.mean((d - d.mean()) ** 2)))


__all__ = ["unit_times", "training_rows", "fit", "apply", "apply_flops", "makespan_ms", "prediction_error",
           "bsmm_plan_query"]
