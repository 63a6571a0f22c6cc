"""The autotuner's choices persist in the JSON file named by GF2_TUNE_CACHE
and are reused by a later process (batched variant and single-product plan).
Each run is a fresh process so the in-memory cache starts empty."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json
sys.path.insert(0, %(root)r)
import torch
import paper_0811_1714_gb300 as g
import synth
g.build()
dims = synth.batch_dims(40, seed=9, lo=32, hi=700)
MA, MB, MC, keep = [], [], [], []
for i, (m, l, n) in enumerate(dims):
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    MA.append(g.mat(A, l)); MB.append(g.mat(B, n)); MC.append(g.mat(C, n))
    g.gf2_random(MA[-1], 5 * i + 1); g.gf2_random(MB[-1], 5 * i + 2)
    keep.append((A, B, C))
v = g.gf2_mul_batched_ex(g.MatArrays(MC, MA, MB))
n = 4096
A, B, C = g.empty(n, n), g.empty(n, n), g.empty(n, n)
g.gf2_random(g.mat(A, n), 1); g.gf2_random(g.mat(B, n), 2)
g.gf2_mul(g.mat(C, n), g.mat(A, n), g.mat(B, n))          # automatic base and depth
bad = g.gf2_freivalds(g.mat(C, n), g.mat(A, n), g.mat(B, n), 7)
torch.cuda.synchronize()
print(json.dumps({"variant": v, "plan": g.gf2_describe_plan(n, n, n), "bad": bad}))
"""


def run_child(cache):
    env = dict(os.environ, GF2_TUNE_CACHE=cache)
    out = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_tune_cache_persists_across_processes(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = str(tmp_path / "tune.json")
    first = run_child(cache)
    saved = json.load(open(cache))
    assert any(k.startswith("batched-") for k in saved)
    assert any(k.startswith("mul-") for k in saved)
    second = run_child(cache)
    assert second["variant"] == first["variant"]
    assert second["plan"] == first["plan"]
    assert first["bad"] == 0 and second["bad"] == 0
