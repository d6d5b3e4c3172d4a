"""One full-size configuration, run in a fresh process by test_gpu_fullsize.py.

    python tests/fullsize_check.py <config>

Builds the configuration's operands exactly as bench.py does (seeded Philox,
pinned host memory), runs one out-of-core call through the C ABI in the plan
bench.py times, recomputes sampled 64 x 64 blocks of C with the CPU oracle
(the old C blocks saved before the call) and prints one JSON line.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import bench  # noqa: E402
import bounds  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402
import paper_1808_05056_gb300 as P  # noqa: E402


def main(name):
    P.load()
    form, M, N, K, alpha, beta, budget, dist = bench.CONFIGS[name]
    out = {"config": name}
    if form == "batched":
        shapes = bench.batch_shapes(1234, M, N, K)
        ops = []
        for q, (m, n, k) in enumerate(shapes):
            A = torch.empty((m, k), dtype=torch.float64, pin_memory=True)
            B = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
            C = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
            synth.fill(A, 100 + q, 0, dist)
            synth.fill(B, 100 + q, 1, dist)
            ops.append((A, B, C))
        descs = [P.gemm_desc("N", "N", A, B, C, alpha, beta) for A, B, C in ops]
        from paper_1808_05056_gb300 import tune
        flags = 0
        if os.path.exists(tune.DEFAULT_MODEL):  # the learned-model plans the benchmark times
            tune.install()
            flags = P.OOC_PLAN_MODEL
        st = P.ooc_stats()
        rc = P.ooc_dgemm_batched(descs, budget, P.make_opts(form=P.OOC_FORM_FP64, flags=flags), st)
        out["rc"] = rc
        errs = []
        for q in range(0, len(shapes), max(1, len(shapes) // 16)):
            m, n, k = shapes[q]
            A, B, C = ops[q]
            i, j = bench.sample_blocks(dict(M=m, N=n), 1, 32, seed=q)[0]
            ref, _ = oracle.gemm_block("N", "N", i, j, 32, 32, k, alpha, A.numpy(), B.numpy(), 0.0, None)
            errs.append(oracle.rel_fro(C.numpy()[i:i + 32, j:j + 32], ref))
        out.update(max_rel_fro=max(errs), tol=1e-13, samples=len(errs), problems=len(shapes))
    else:
        dtname, tol, _, _ = bench.FORMS[form]
        dt = getattr(torch, dtname)
        A = torch.empty((M, K), dtype=dt, pin_memory=True)
        B = torch.empty((K, N), dtype=dt, pin_memory=True)
        C = torch.empty((M, N), dtype=dt, pin_memory=True)
        for t, s in ((A, 0), (B, 1), (C, 2)):
            synth.fill(t, 1, s, dist)
        w = dict(M=M, N=N, K=K)
        blocks = bench.sample_blocks(w, 24, 64)
        blocks += [(0, 0), (M - 64, N - 64), (M - 64, 0), (0, N - 64)]  # the corners: ragged edges
        cold = [C[i:i + 64, j:j + 64].numpy().astype(np.float64) for i, j in blocks]
        form_id = {"fp64": P.OOC_FORM_FP64, "ozaki": P.OOC_FORM_OZAKI, "bf16x3": P.OOC_FORM_BF16X3}[form]
        call = P.ooc_sgemm if form == "bf16x3" else P.ooc_dgemm
        st = P.ooc_stats()
        rc = call("N", "N", M, N, K, alpha, A, K, B, N, beta, C, N, budget, P.make_opts(form=form_id), st)
        out["rc"] = rc
        errs, ratios = [], []
        kchunks = max(1, -(-K // st.kb)) if st.kb else 1
        for (i, j), c0 in zip(blocks, cold):
            ref, _ = oracle.gemm_block("N", "N", i, j, 64, 64, K, alpha, A.numpy(), B.numpy(), beta,
                                       c0 if beta != 0 else None)
            got = C.numpy()[i:i + 64, j:j + 64]
            errs.append(oracle.rel_fro(got, ref))
            # elementwise: each form's own componentwise bound (tests/bounds.py)
            Ab = A.numpy()[i:i + 64, :].astype(np.float64)
            Bb = B.numpy()[:, j:j + 64].astype(np.float64)
            c0b = c0 if beta != 0 else None
            if form == "ozaki":
                bd = bounds.ozaki_bound(Ab, Bb, alpha, beta, c0b, st.slices, kchunks)
            elif form == "bf16x3":
                bd = bounds.bf16x3_bound(Ab, Bb, alpha, beta, c0b, kchunks)
            else:
                bd = None
            if bd is not None:
                ratios.append(bounds.worst_ratio(got, ref, bd))
        out.update(max_rel_fro=max(errs), tol=tol, samples=len(errs), blocks=st.blocks,
                   device_bytes=st.device_bytes, budget=budget)
        if ratios:
            out["max_elementwise_ratio"] = max(ratios)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main(sys.argv[1])
