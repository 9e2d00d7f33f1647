"""Two host threads making their first library calls at the same moment.

The one-time set-up of a kernel instance (its shared-memory limit, a
per-device attribute, and its blocks per SM) is done once per (device,
instance) under a lock.  A fresh process starts two threads behind a barrier;
each calls hk_cross_section_batched on its own stream with its own workspace
(the batched entry point takes the caller's scratch, so nothing on the GPU is
shared), one with 501-bin lines (short-line instance) and one with 1601-bin
lines (wide-line instance), three times; then each result is compared with
the same call made again from one thread.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, threading
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
from paper_2101_02005_gb300 import build
build.build()
from paper_2101_02005_gb300 import hk, synth

torch.cuda.set_device(0)
Q = synth.partition_function
w = synth.config(0)
D = hk.DeviceLines.from_host(w.species[0])
grid = hk.make_grid(*w.grid.astuple())
states = [hk.make_state(1000.0, 1.0, float(Q(1000.0))), hk.make_state(600.0, 0.1, float(Q(600.0)))]
opts = [hk.make_opts(float(Q(296.0)), c, hk.HK_FP32C, flags=hk.HK_SIGMA_F64) for c in (25.0, 80.0)]
ws = [torch.empty(hk.hk_workspace_size(0, [D], len(states), grid, o), dtype=torch.uint8,
                  device="cuda") for o in opts]
outs = [[torch.empty((1, len(states), grid.nbins), dtype=torch.float64, device="cuda")
         for _ in range(3)] for _ in opts]
gate = threading.Barrier(2)
errors = []

def run(t):
    try:
        s = torch.cuda.Stream()
        gate.wait()
        for r in range(3):
            hk.hk_cross_section_batched([D], states, grid, opts[t], outs[t][r], ws[t], stream=s)
        s.synchronize()
    except Exception as e:
        errors.append(repr(e))

th = [threading.Thread(target=run, args=(t,)) for t in range(2)]
for x in th:
    x.start()
for x in th:
    x.join()
assert not errors, errors
hk.hk_sync_status()
for t in range(2):
    ref = hk.hk_cross_section_batched([D], states, grid, opts[t])
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.abs(r).max() > 0
    for k in range(3):
        g = outs[t][k].cpu().numpy()
        assert np.allclose(g, r, rtol=1e-12, atol=1e-300), (t, k, float(np.abs(g - r).max()))
print("ok")
"""


def test_two_threads_first_calls():
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.stdout[-2000:],
                                                                    r.stderr[-4000:])
