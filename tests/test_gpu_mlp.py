"""The cost-model MLP kernels against the FP64 oracle: loss and gradient, forward
pass, an Adam step, reproducibility, and plans re-packed by its predictions."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import mlp as OM
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu
F, H = P.BSMM_NFEATURES, 32


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, F)).astype(np.float32)
    t = (np.tanh(X[:, 0] - 0.5 * X[:, 2]) + 0.2 * X[:, 7] + 0.05 * rng.normal(0, 1, n)).astype(np.float32)
    return X, t


def _identity_norm(mlp):
    P.bsmm_mlp_set_norm(mlp, np.zeros(F), np.ones(F), 0.0, 1.0)


@pytest.mark.parametrize("n", [1, 100, 1000, 4099])
def test_loss_and_gradient_match_oracle(n):
    import torch
    X, t = _data(n, n)
    mlp = P.bsmm_mlp_create(3)
    _identity_norm(mlp)
    theta = P.bsmm_mlp_get_params(mlp).astype(np.float64)
    loss, g = P.bsmm_mlp_loss_grad(mlp, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    L, gref = OM.loss_and_grad(theta, X.astype(np.float64), t.astype(np.float64), F, H)
    assert abs(loss - L) <= 1e-5 * max(1.0, L)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_forward_matches_oracle_with_standardisation():
    import torch
    X, _ = _data(5, 777)
    X = X * 3.0 + 1.5
    mlp = P.bsmm_mlp_create(9)
    mu, sd = X.mean(0), X.std(0)
    P.bsmm_mlp_set_norm(mlp, mu, sd, 2.0, 0.5)
    y = torch.zeros(777, dtype=torch.float32, device="cuda")
    P.bsmm_mlp_predict(mlp, torch.from_numpy(X).cuda(), y)
    theta = P.bsmm_mlp_get_params(mlp).astype(np.float64)
    ref = OM.forward(theta, (X.astype(np.float64) - mu) / sd, F, H) * 0.5 + 2.0
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_adam_step_matches_oracle():
    import torch
    X, t = _data(11, 500)
    mlp = P.bsmm_mlp_create(4)
    theta0 = P.bsmm_mlp_get_params(mlp).astype(np.float64)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    P.bsmm_mlp_fit(mlp, Xd, td, 1, 0.01)
    # fit standardises from the data first; replay that in FP64 and take one Adam step
    mu, sd = OM.standardise(X)
    tm, ts = float(t.astype(np.float64).mean()), float(t.astype(np.float64).std())
    _, g = OM.loss_and_grad(theta0, (X - mu) / sd, (t - tm) / ts, F, H)
    want, _, _ = OM.adam_step(theta0, np.zeros_like(theta0), np.zeros_like(theta0), g, 1, 0.01)
    got = P.bsmm_mlp_get_params(mlp).astype(np.float64)
    # the first Adam step moves each coordinate by about lr * sign(g): exact agreement
    # wherever the gradient is clearly nonzero, and never more than lr anywhere
    big = np.abs(g) > 1e-5
    assert np.max(np.abs(got - want)[big]) <= 1e-6
    assert np.max(np.abs(got - theta0)) <= 0.01 * (1 + 1e-5)


def test_training_is_reproducible_and_learns():
    import torch
    X, t = _data(2, 3000)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    outs = []
    for _ in range(2):
        mlp = P.bsmm_mlp_create(7)
        loss = P.bsmm_mlp_fit(mlp, Xd, td, 400, 3e-3)
        outs.append((loss, P.bsmm_mlp_get_params(mlp)))
    assert outs[0][0] == outs[1][0] and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][0] < 0.1  # standardised MSE of a smooth target


def test_predicted_costs_repack_without_changing_bits():
    from gpu_helpers import run_lib
    import torch
    prob = G.make_problem("clustered", 3, 1500, lo=16, hi=200, nclusters=8, cluster_density=0.2)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(0))
    base, plan = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16)
    feats, _ = P.bsmm_plan_features(plan)
    mlp = P.bsmm_mlp_create(1)
    rng = np.random.default_rng(0)
    P.bsmm_mlp_fit(mlp, torch.from_numpy(feats).cuda(), torch.from_numpy(rng.normal(0, 1, len(feats)).astype(np.float32)).cuda(), 50, 1e-2)
    P.bsmm_plan_predict_costs(plan, mlp)
    again, _ = run_lib(prob, cs, C0, off, plan=plan)
    assert np.array_equal(struct_elements(prob, cs, off, base), struct_elements(prob, cs, off, again))
