"""The checked build (-DPIC_CHECKED): every stored cell index is validated before use.  On valid
states it must change nothing: the same steps through the checked library and the ordinary one end
in byte-identical snapshots, with no device error raised."""
import hashlib
import os
import subprocess
import sys

import pytest

from paper_2606_28534_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = """
import hashlib, sys
sys.path.insert(0, {root!r})
from paper_2606_28534_gb300 import pic, workloads as W
out = []
for name in ("SMALL_C2", "SMALL_C3", "SMALL_C6"):
    g = pic.Simulation(W.variant(getattr(W, name), sort_interval=3, capacity_factor=2.0, neutral_capacity=2.0))
    g.step(17)
    g.sync()
    out.append(hashlib.sha256(g.snapshot()).hexdigest())
    g.close()
b = pic.Batch(W.small_ensemble(4))
b.step(7)
b.sync()
out.append(hashlib.sha256(b"".join(b.snapshot(k) for k in range(4))).hexdigest())
print(" ".join(out))
"""


def _hashes(lib):
    env = dict(os.environ, PIC_LIB=lib)
    r = subprocess.run([sys.executable, "-c", RUN.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return r.stdout.split()


def test_checked_build_changes_nothing_on_valid_states():
    plain = build.build()
    checked = build.build(checked=True)
    assert _hashes(checked) == _hashes(plain)
