"""Plan search tools on top of the C ABI: autotuner data collection, cost-model
training on the GPU (the library's MLP kernels), regret measurement, and model
files.

The cost model maps the 16 features of a (problem, candidate plan) pair (see
ooc_plan_candidates) to log2 of the measured seconds; the planner, given
OOC_PLAN_MODEL and an installed model, keeps the candidate with the smallest
prediction.  The exhaustive autotuner (ooc_autotune) stays the reference: the
regret of a model pick is its measured time over the best measured time, minus 1.
"""
import os

import numpy as np

from . import (OOC_ERR_BUDGET, OOC_FORM_BF16X3, OOC_FORM_FP64, OOC_FORM_OZAKI, OOC_MLP_PARAMS, OocError, gemm_desc,
               make_opts, ooc_autotune, ooc_costmodel_set, ooc_mlp_forward, ooc_mlp_train)

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "costmodel_gb300.f32")


def training_problems(seed, count, lo=512, hi=8192):
    """Seeded problems: (form, M, N, K, budget bytes), dims log-uniform in [lo, hi],
    budgets between 1/8 and 2x the operands' size (so most run out of core)."""
    rng = np.random.default_rng(seed)
    forms = [OOC_FORM_FP64, OOC_FORM_BF16X3, OOC_FORM_OZAKI]
    out = []
    for i in range(count):
        form = forms[i % 3]
        m, n, k = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
        es = 4 if form == OOC_FORM_BF16X3 else 8
        size = (m * k + k * n + m * n) * es
        budget = int(size * np.exp(rng.uniform(np.log(1 / 8), np.log(2))))
        out.append((form, m, n, k, max(budget, 8 << 20)))
    return out


def collect(problems, max_candidates=12, seed=7, log=None):
    """Autotune every problem on scratch operands; returns a list of
    (features [n_cand, 16] float32, seconds [n_cand] float64, problem)."""
    import torch
    import synth
    recs = []
    for q, (form, m, n, k, budget) in enumerate(problems):
        dt = torch.float32 if form == OOC_FORM_BF16X3 else torch.float64
        A = torch.empty((m, k), dtype=dt, pin_memory=True)
        B = torch.empty((k, n), dtype=dt, pin_memory=True)
        C = torch.empty((m, n), dtype=dt, pin_memory=True)
        synth.fill(A, seed + q, 0, synth.UNIFORM)
        synth.fill(B, seed + q, 1, synth.UNIFORM)
        d = gemm_desc("N", "N", A, B, C, 1.0, 0.0)
        try:
            res = ooc_autotune(d, 4 if form == OOC_FORM_BF16X3 else 8, budget, make_opts(form=form), max_candidates)
        except OocError as e:
            if e.code != OOC_ERR_BUDGET:
                raise
            if log:
                log("problem %d skipped: %s" % (q, e))
            continue
        feats = np.array([list(c.features) for c, _ in res], dtype=np.float32)
        secs = np.array([s for _, s in res], dtype=np.float64)
        recs.append((feats, secs, (form, m, n, k, budget)))
        if log:
            log("problem %d form %d %dx%dx%d budget %.0f MB: %d candidates, best %.4f s, heuristic %.4f s" % (
                q, form, m, n, k, budget / 2 ** 20, len(secs), secs.min(), secs[0]))
    return recs


def dataset(recs):
    X = np.concatenate([f for f, _, _ in recs]).astype(np.float32)
    t = np.concatenate([np.log2(s) for _, s, _ in recs]).astype(np.float32)
    return X, t


def init_params(seed=0):
    """He-style random initial parameters, seeded (float32, OOC_MLP_PARAMS values)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / 16), 64 * 16), np.zeros(64), rng.normal(0, np.sqrt(2.0 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, np.sqrt(1.0 / 64), 64), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == OOC_MLP_PARAMS
    return p


def train(recs, epochs=500, batch=64, lr=2e-3, weight_decay=1e-3, seed=1):
    """Train the cost model on the GPU with the library's kernels; returns (params, final loss)."""
    X, t = dataset(recs)
    return ooc_mlp_train(init_params(seed), X, t, epochs=epochs, batch=batch, lr=lr, seed=seed,
                         weight_decay=weight_decay)


DEFAULT_DATA = os.path.join(HERE, "costmodel_data_gb300.npz")


def save_records(recs, path):
    X, t = dataset(recs)
    np.savez(path, X=X, t=t, sizes=np.array([len(s) for _, s, _ in recs]),
             problems=np.array([p for _, _, p in recs], dtype=np.float64))


def load_records(path=DEFAULT_DATA):
    """Records saved by save_records: (features, seconds, problem) per problem."""
    d = np.load(path)
    offs = np.concatenate([[0], np.cumsum(d["sizes"])])
    return [(d["X"][a:b], np.exp2(d["t"][a:b].astype(np.float64)), tuple(d["problems"][i]))
            for i, (a, b) in enumerate(zip(offs[:-1], offs[1:]))]


def split(recs, seed):
    """Held-out quarter of the problems (seeded)."""
    idx = np.random.default_rng(seed).permutation(len(recs))
    n_test = max(1, len(recs) // 4)
    return [recs[i] for i in idx[n_test:]], [recs[i] for i in idx[:n_test]]


def regret(recs, params):
    """Per problem: measured time of the model's pick / best measured time - 1."""
    out = []
    for feats, secs, _ in recs:
        pred = ooc_mlp_forward(params, feats)
        out.append(float(secs[int(np.argmin(pred))] / secs.min() - 1.0))
    return np.array(out)


def heuristic_regret(recs):
    """Same for the planner's analytic choice (candidate 0)."""
    return np.array([float(secs[0] / secs.min() - 1.0) for _, secs, _ in recs])


def save(params, path=DEFAULT_MODEL):
    np.asarray(params, dtype=np.float32).tofile(path)


def load(path=DEFAULT_MODEL):
    p = np.fromfile(path, dtype=np.float32)
    if p.size != OOC_MLP_PARAMS:
        raise ValueError("%s holds %d values, expected %d" % (path, p.size, OOC_MLP_PARAMS))
    return p


def install(path=DEFAULT_MODEL):
    """Load a model file and install it for OOC_PLAN_MODEL."""
    p = load(path)
    ooc_costmodel_set(p)
    return p
