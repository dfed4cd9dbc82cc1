"""The bounds-checked build (-DIGG_BOUNDS_CHECK) on the default step's
kernels: hidden steps on 2x2x2 subdomains of a TMA size, on a field that
sends many points to the fix-up launch and through the one-launch halo
update, give the release build's bits with no index test failing. Each
build runs in its own process (the binding loads one library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import synth
import paper_2211_15716_gb300 as igg
from paper_2211_15716_gb300 import workloads as wl
n, dims, periods, o = (70, 21, 19), (2, 2, 2), (1, 0, 0), (2, 2, 2)
with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
    ng = g.global_size()
    T0 = np.empty(g.shape)
    Ci = np.empty(g.shape)
    for s in range(g.nsub):
        gi = g.global_indices(s)
        T0[s] = synth.sine_modes(1, *gi, ng, base=0.0)
        Ci[s] = synth.ci_uniform_c0(0, *gi, ng)
    T = torch.from_numpy(T0).cuda()
    Cd = torch.from_numpy(Ci).cuda()
    dx, dy, dz, dt = wl.setup(wl.Workload("b", n, dims, periods, o), g, Cd)
    g.fixup_stats(clear=True)
    res = g.run(7, T, T.clone(), Cd, 1.0, dt, dx, dy, dz, widths=(16, 2, 2))
    out = res.cpu().numpy()
    segs, pts = g.fixup_stats()
    assert g.device_status() == 0
assert pts > 0
np.save({out!r}, out)
print(igg.lib().igg_bounds_checked(), igg.bounds_status())
"""


def _run(tmp_path, checked):
    out = str(tmp_path / f"out{int(checked)}.npy")
    env = dict(os.environ)
    env.pop("IGG_BOUNDS_CHECK", None)
    if checked:
        env["IGG_BOUNDS_CHECK"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, out=out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    flag, status = map(int, r.stdout.split()[-2:])
    return np.load(out), flag, status


def test_checked_build_same_bits_no_failed_test(tmp_path):
    from paper_2211_15716_gb300 import build
    build.build()
    build.build(checked=True)
    rel, f0, s0 = _run(tmp_path, False)
    chk, f1, s1 = _run(tmp_path, True)
    assert (f0, f1) == (0, 1)
    assert s0 == 0 and s1 == 0
    assert np.array_equal(rel.view(np.uint64), chk.view(np.uint64))
