"""The tensor-core join launches in a fresh process before any many-jobs call.

The join kernel needs more than the default 48 KB of dynamic shared memory;
its launcher must raise the limit itself rather than rely on an earlier call
of another launcher having done so.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, %r)
import numpy as np, torch, synth
from paper_1809_09930_gb300 import gj
X = torch.from_numpy(synth.uniform(20000, 16, 7)).cuda()
with gj.Index(X, 0.9, k=0, flags=gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER) as ix:
    n = ix.count()
with gj.Index(X, 0.9, k=0) as ip:
    m = ip.count()
assert n == m, (n, m)
print("ok", n)
""" % ROOT


@pytest.mark.gpu
def test_tc_join_first_in_process():
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
