"""GPU check of the checked build (libdgwave_checked.so, DGW_DEVICE_CHECKS):
its stage kernels test every face connection code and block-table entry
they read before using it.  On valid input the checks must change nothing:
the same solves (tensor cores, node-thread and element-thread CUDA cores,
FP32 and FP64, a batch with media and a point source, a partition) give bit
for bit the results of the
normal library, and every status check stays DG_OK.  The checked library
runs in a child process (DGWAVE_CHECKED=1 selects it at import)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
import paper_1304_5546_gb300 as P
from synth import gaussian_pulse, jittered_delaunay_mesh, random_permittivity

out = {"lib": P._lib.LIB_PATH}
mesh = jittered_delaunay_mesh(12, seed=3)
for name, N, prec in (("tc5", 5, "fp32"), ("tc3", 3, "fp32"), ("simt4", 4, "fp32simt"),
                      ("fp64", 3, "fp64"), ("ept2", 2, "fp32"), ("ept1", 1, "fp32")):
    s = P.Solver(*mesh, N=N, precision=prec)
    x, y = s.nodes()
    q = s.from_numpy(np.stack(gaussian_pulse(x, y, 0.4, 0.6, 0.15)))
    res = s.new_fields()
    s.step(q, res, 0.9 * s.cfl_dt(), 3)
    P.dg_sync_check(s.op)
    out[name] = s.to_numpy(q)
    if name == "tc5":
        part = P.Partition(s, 3)
        q0 = s.from_numpy(np.stack(gaussian_pulse(x, y, 0.4, 0.6, 0.15)))
        part.set_fields(q0)
        part.step(0.9 * s.cfl_dt(), 3)
        got = s.new_fields()
        part.get_fields(got)
        part.sync_check()
        out["part"] = s.to_numpy(got)
m = jittered_delaunay_mesh(7, seed=8)
s = P.Solver(*m, N=5, precision="fp32", eps=random_permittivity(2 * 49, seed=8), host_only=True)
b = P.Batch({5: 128})
dt = 0.8 * s.cfl_dt()
slot = b.add(s, dt, source=(0.45, 0.55, 0.15 / dt, 0.3 * dt, 1.0))
x, y = s.nodes()
b.set_fields(slot, np.stack(gaussian_pulse(x, y, 0.5, 0.5, 0.2)).astype(np.float32))
b.step(3)
b.sync_check()
out["batch"] = b.get_fields(slot)
np.savez(sys.argv[1], **out)
"""


def _run(path, checked):
    env = dict(os.environ)
    env["DGWAVE_CHECKED"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, "-c", RUN % {"root": ROOT}, path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


def test_checked_build_matches_normal_build(tmp_path):
    from paper_1304_5546_gb300 import build as B
    B.build()
    B.build(checked=True)
    normal = _run(str(tmp_path / "normal.npz"), False)
    checked = _run(str(tmp_path / "checked.npz"), True)
    assert str(checked["lib"]).endswith("libdgwave_checked.so")
    assert str(normal["lib"]).endswith("libdgwave.so")
    for key in ("tc5", "tc3", "simt4", "fp64", "ept2", "ept1", "part", "batch"):
        assert np.array_equal(normal[key], checked[key]), key
    assert np.array_equal(normal["part"], normal["tc5"])
