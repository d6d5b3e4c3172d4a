"""Train the schedule cost model on this GPU and write the model file.

    python -m paper_1808_05056_gb300.train_costmodel [--problems 96] [--out PATH] [--report PATH]

Autotunes a seeded set of out-of-core problems (FP64, BF16x3 and Ozaki forms,
mixed shapes and budgets) with ooc_autotune, trains the MLP on 3/4 of them with
the library's GPU kernels, and reports the regret of the model's picks and of
the analytic planner on the held-out quarter (time of the pick over the best
autotuned time, minus one).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1808_05056_gb300 as P  # noqa: E402
from paper_1808_05056_gb300 import tune  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=96)
    ap.add_argument("--candidates", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=500)
    ap.add_argument("--weight-decay", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--from-data", default=None, help="reuse autotuner timings saved by --data (no autotuning)")
    ap.add_argument("--out", default=tune.DEFAULT_MODEL)
    ap.add_argument("--report", default=None)
    ap.add_argument("--data", default=None, help="save the collected autotuner timings (.npz)")
    a = ap.parse_args()
    P.load()
    t0 = time.time()
    if a.from_data:
        recs = tune.load_records(a.from_data)
    else:
        probs = tune.training_problems(a.seed, a.problems)
        recs = tune.collect(probs, max_candidates=a.candidates, log=lambda s: print(s, flush=True))
    t_collect = time.time() - t0
    if a.data:
        tune.save_records(recs, a.data)
    # held-out regret over three seeded splits (model trained on the other three quarters)
    folds = []
    for k in range(3):
        train, test = tune.split(recs, a.seed + k)
        params, _ = tune.train(train, epochs=a.epochs, weight_decay=a.weight_decay, seed=a.seed + k)
        folds.append((tune.regret(test, params), tune.heuristic_regret(test)))
    rm = np.concatenate([m for m, _ in folds])
    rh = np.concatenate([h for _, h in folds])
    t0 = time.time()
    params, loss = tune.train(recs, epochs=a.epochs, weight_decay=a.weight_decay, seed=a.seed)
    t_train = time.time() - t0
    tune.save(params, a.out)

    def summ(r):
        return {"mean": float(r.mean()), "median": float(np.median(r)), "max": float(r.max()),
                "within_5pct": float(np.mean(r <= 0.05))}
    rep = {"problems": len(recs), "candidates_per_problem": int(np.median([len(s) for _, s, _ in recs])),
           "collect_seconds": t_collect, "train_seconds_final": t_train, "final_train_loss": loss,
           "epochs": a.epochs, "weight_decay": a.weight_decay,
           "heldout_regret_model": summ(rm), "heldout_regret_analytic_planner": summ(rh),
           "heldout_problems": int(rm.size), "model_file": os.path.basename(a.out)}
    print(json.dumps(rep), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
