"""Programmatic dependent launch (off by default, HLBM_PDL=1 turns it on) does
not change results: the same runs in child processes with and without it
give bitwise-equal fields.  The setting is read once per process, hence the
children.  Covers the launches that call griddepcontrol: the TMA collide
(one-tile and persistent), the cp.async collide, the wavefront and block FD
kernels, and the tiled batch path."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import hashlib, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_0902_3921_gb300 import build as B, inputs as I, lbm
B.build(); lbm.load_library()
CFG = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
h = hashlib.sha256()
for tuning in ("2,42,4,7,1", "4,54,4,5,1", "4,96,4,0,128"):
    os.environ["HLBM_TUNING"] = tuning
    lat = lbm.Lattice(lbm.LbmParams(Lx=256, Ly=192, fd_substeps=4, precision=lbm.LBM_F32DEV, **CFG))
    n, u = I.rest(2, 256, 192)
    u = u + 0.004 * np.sin(np.arange(256) / 7.0)[None, None, :]
    lat.init_fields(n, I.spinodal(2, 256, 192, seed=3), u).step(7).step(64)
    for a in lat.moments():
        h.update(np.ascontiguousarray(a).tobytes())
    lat.close()
del os.environ["HLBM_TUNING"]
os.environ["HLBM_BATCH_PATH"] = "tiled"
insts = [(64, 80, (1e-5, 0.0), 5), (36, 20, (0.0, 0.0), 0), (128, 64, (0.0, 2e-5), 100)]
b = lbm.Batch(lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG), insts)
for k, (Lx, Ly, g, fs) in enumerate(insts):
    n, u = I.rest(2, Lx, Ly)
    b.init_fields(k, n, I.spinodal(2, Lx, Ly, seed=10 + k), u)
b.step(3).step(20)
for k in range(len(insts)):
    for a in b.moments(k):
        h.update(np.ascontiguousarray(a).tobytes())
b.close()
print("DIGEST", h.hexdigest())
"""


def _digest(pdl):
    env = dict(os.environ, HLBM_PDL=pdl)
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("DIGEST")]
    assert line, out.stdout[-2000:]
    return line[0].split()[1]


def test_pdl_on_and_off_give_the_same_bits():
    assert _digest("1") == _digest("0")
