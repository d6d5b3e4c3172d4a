"""GPU checks of the schedule cost model and plan search: the library's MLP
forward/backward kernels against the FP64 oracle, training on the GPU, the
planner's use of an installed model, and the exhaustive autotuner."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import costmodel
from gpu_util import pinned, pinned_from

pytestmark = pytest.mark.gpu


def _data(n=300, seed=11):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, 16)).astype(np.float32)
    t = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 8]).astype(np.float32)
    return X, t


def test_forward_matches_oracle(ooc):
    X, _ = _data()
    p = costmodel.init(3)
    got = ooc.ooc_mlp_forward(p, X)
    ref, _ = costmodel.forward(p, X)
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


def test_loss_gradient_matches_oracle(ooc):
    X, t = _data(257)
    p = costmodel.init(4)
    loss, g = ooc.ooc_mlp_loss_grad(p, X, t)
    ref_loss, ref_g = costmodel.loss_grad(p.astype(np.float64), X, t)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)


def test_training_reduces_loss(ooc):
    from paper_1808_05056_gb300 import tune
    X, t = _data(600)
    p0 = tune.init_params(2)
    l0, _ = ooc.ooc_mlp_loss_grad(p0, X, t)
    p, l1 = ooc.ooc_mlp_train(p0, X, t, epochs=200, batch=64, lr=3e-3, seed=5)
    assert l1 < 0.05 * l0
    # the trained parameters reproduce the reported loss through the oracle
    assert abs(costmodel.loss(p.astype(np.float64), X, t) - l1) <= 1e-3 * max(l1, 1e-6) + 1e-7


def test_planner_follows_installed_model(ooc):
    # a hand-built model: prediction = -10 * feature[8] (log2 mb), so the planner must pick the largest mb
    d = costmodel.unpack(np.zeros(costmodel.NPARAM))
    d["W1"][0, 8] = 1.0
    d["W2"][0, 0] = 1.0
    d["W3"][0] = -10.0
    p = costmodel.pack(d).astype(np.float32)
    M, N, K, budget = 3000, 2000, 1500, 16 << 20
    cands = ooc.ooc_plan_candidates(M, N, K, 8, 0, budget, capacity=64)
    assert len(cands) > 1
    ooc.ooc_costmodel_set(p)
    try:
        plan = ooc.ooc_plan(M, N, K, 8, 0, budget, ooc.make_opts(flags=ooc.OOC_PLAN_MODEL))
    finally:
        ooc.ooc_costmodel_set(None)
    assert plan["mb"] == max(c.mb for c in cands)
    heur = ooc.ooc_plan(M, N, K, 8, 0, budget)
    assert (heur["mb"], heur["nb"], heur["kb"]) == (cands[0].mb, cands[0].nb, cands[0].kb)


def test_autotune_times_every_candidate(ooc):
    M, N, K = 1024, 768, 512
    A = pinned_from(12, 0, M, K, synth.UNIFORM)
    B = pinned_from(12, 1, K, N, synth.UNIFORM)
    C = pinned(M, N)
    d = ooc.gemm_desc("N", "N", A, B, C, 1.0, 0.0)
    res = ooc.ooc_autotune(d, 8, 2 << 20, ooc.make_opts(form=ooc.OOC_FORM_FP64), max_candidates=6)
    assert 1 <= len(res) <= 6
    assert all(s > 0 for _, s in res)
    # the last run left a correct product in C (element by element against the oracle)
    ref = oracle.gemm("N", "N", 1.0, A.numpy().astype(np.float64), B.numpy().astype(np.float64), 0.0, None)
    np.testing.assert_allclose(C.numpy(), ref, rtol=1e-12, atol=1e-12)


def test_trained_model_gains_over_analytic_planner(ooc):
    """On autotuner timings recorded on GB300 (93 problems x 16 candidate plans),
    a model trained on the GPU with the library's kernels picks plans whose
    held-out regret (measured time / best measured time - 1) is lower on average
    than the analytic planner's, without its worst picks."""
    from paper_1808_05056_gb300 import tune
    recs = tune.load_records()
    assert len(recs) >= 60
    rm, rh = [], []
    for k in range(3):
        train, test = tune.split(recs, 1 + k)
        params, _ = tune.train(train, seed=1 + k)
        rm.append(tune.regret(test, params))
        rh.append(tune.heuristic_regret(test))
    rm, rh = np.concatenate(rm), np.concatenate(rh)
    assert rm.mean() < rh.mean()
    assert rm.max() < 0.5 and np.mean(rm <= 0.05) >= 0.8
