"""GPU: the checked build (build.py --checked: every index the traversal gathers through is
checked, a bad one is reported instead of read) runs the parity cases cleanly -- no index
fault is latched on 2-D and 3-D cases with cyclic blocks, FP32 and FP64, J and J^T, the
persistent schedule (both item kernels) and the level schedule -- and gives the same
results as the normal build bit for bit.  An upstream position planted out of range (a
hook only the checked build has) is reported by tangent_status; the normal build refuses
the hook."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import build as B
from paper_2609_14982_b300 import eik

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import sys
import numpy as np
import torch
from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W
assert eik.LIB_PATH == sys.argv[1], eik.LIB_PATH
out = {}
cases = {"config1": W.config1(), "steep": W.config5_grid(0)}
for name, wl in cases.items():
    src = wl.src[:3]
    dg = eik.DeviceGrid(wl.grid)
    s = torch.tensor(wl.s, device="cuda")
    T, _ = eik.eik_forward(dg, s, src)
    for chunk, sched in ((0, eik.SCHED_PERSISTENT), (256, eik.SCHED_PERSISTENT), (0, eik.SCHED_LEVELS)):
        tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(chunk=chunk, schedule=sched))
        for dtype, R in ((torch.float64, 2), (torch.float32, 8)):
            rng = np.random.default_rng(R)
            p = torch.tensor(rng.standard_normal((wl.grid.N, R)), device="cuda", dtype=dtype)
            y = torch.tensor(rng.standard_normal((len(src), len(wl.rec), R)), device="cuda", dtype=dtype)
            _, d = tan.apply(p, shared_model=True)
            g, _ = tan.apply_T(y, sum_sources=True)
            tan.status()
            key = f"{name}-{chunk}-{sched}-{R}"
            out[key + "-d"] = d.double().cpu().numpy()
            out[key + "-g"] = g.double().cpu().numpy()
        tan.free()
np.savez(sys.argv[2], **out)
print("ok")
"""


def _run(lib, path):
    env = dict(os.environ, EIK_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, lib, path], env=env, capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))), timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
    return np.load(path)


def test_checked_build_runs_clean_and_equals_normal_build(tmp_path):
    checked = B.build(checked=True)
    normal = B.build()
    a = _run(checked, str(tmp_path / "checked.npz"))
    b = _run(normal, str(tmp_path / "normal.npz"))
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k


POKE = r"""
import sys
import numpy as np
import torch
from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W
wl = W.config1()
dg = eik.DeviceGrid(wl.grid)
s = torch.tensor(wl.s, device="cuda")
T, _ = eik.eik_forward(dg, s, wl.src[:1])
tan = eik.Tangent(dg, T, s, wl.src[:1], rec=wl.rec)
if sys.argv[1] == "normal":
    try:
        tan.debug_poke_edge(0, 10, wl.grid.N + 5)
    except eik.EikError as e:
        print("refused", e.code)
    sys.exit(0)
tan.debug_poke_edge(0, 10, wl.grid.N + 5)
p = torch.ones((wl.grid.N, 2), device="cuda", dtype=torch.float64)
tan.apply(p, shared_model=True)
try:
    tan.status()
    print("not reported")
except eik.EikError as e:
    print("reported", e.code, str(e))
"""


def test_checked_build_reports_a_planted_bad_index():
    checked = B.build(checked=True)
    normal = B.build()
    cwd = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", POKE, "checked"], env=dict(os.environ, EIK_LIB=checked),
                       capture_output=True, text=True, cwd=cwd, timeout=600)
    assert r.returncode == 0, r.stderr
    assert "reported -6" in r.stdout and "index out of range" in r.stdout, r.stdout
    r = subprocess.run([sys.executable, "-c", POKE, "normal"], env=dict(os.environ, EIK_LIB=normal),
                       capture_output=True, text=True, cwd=cwd, timeout=600)
    assert r.returncode == 0 and "refused -1" in r.stdout, r.stdout + r.stderr
