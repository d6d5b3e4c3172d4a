"""Parity at the benchmark configurations' full sizes, in the plans bench.py times.

Each configuration runs in a fresh process (tests/fullsize_check.py): tens of
GiB of pinned host operands per configuration, freed when the process exits.
Outputs are checked on sampled 64 x 64 blocks (and the four corner blocks,
where tiles are ragged) against the CPU oracle, within each form's tolerance,
and for the split forms element by element within each form's componentwise
bound (tests/bounds.py).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("config", ["fp64-32768", "ozaki-65536", "bf16x3-65536", "batched-256"])
def test_full_size_sampled_parity(ooc, config):
    r = subprocess.run([sys.executable, os.path.join(HERE, "fullsize_check.py"), config], capture_output=True,
                       text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps(res))
    assert res["rc"] == 0, res
    assert res["max_rel_fro"] <= res["tol"], res
    # the split forms: every sampled element inside its form's componentwise bound
    assert res.get("max_elementwise_ratio", 0.0) <= 1.0, res
    if "device_bytes" in res:
        assert res["device_bytes"] <= res["budget"]
