"""Two host threads making their first library calls at the same time, in a fresh process (so
the per-device launch settings — shared-memory limits, occupancies, the SM count — are set up
by whichever thread gets there first while the other waits): both solves succeed and equal the
same frames solved afterwards one at a time."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, threading
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2007_08576_gb300 import defsolve as d
from synth import CONFIGS, make_scene
sys.path.insert(0, sys.argv[1] + "/tests")
from gpu_common import MID
d.lib()
scenes = [make_scene(CONFIGS["frame_80x60_n32"], 1000), make_scene(MID, 4242)]
p = d.default_params(precision=2)
out = [None, None]
err = []
barrier = threading.Barrier(2)

def run(k):
    try:
        sc = scenes[k]
        fr = sc.frames[0]
        barrier.wait()
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        s.solve(10, stats=True)
        out[k] = s.deformation64()[1]
        s.close()
    except Exception as e:
        err.append(repr(e))

th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
for t in th: t.start()
for t in th: t.join()
assert not err, err
for k, sc in enumerate(scenes):
    fr = sc.frames[0]
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    s.solve(10, stats=True)
    t = s.deformation64()[1]
    s.close()
    dev = float(np.abs(t - out[k]).max())
    assert dev <= 1e-4, (k, dev)
print("ok")
"""


def test_concurrent_first_calls_from_two_threads():
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().endswith("ok")
