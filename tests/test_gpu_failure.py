"""Failure detection of the pipelined kernels, tested without a GPU fault: a
kernel's bounded wait on an mbarrier that never completes runs out, the
warps agree on stopping, the device error word reports it, and the context
stays usable (a step afterwards matches the oracle)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def test_bounded_wait_runs_out_and_reports():
    from paper_2211_15716_gb300 import igg as igg_mod
    status = igg_mod.selftest_bounded_wait()
    assert status == 1  # IGG_DEV_ERR_TIMEOUT, and no DRAIN bit
    # the context is still usable: a TMA step afterwards matches the oracle
    n = (64, 12, 10)
    g1 = [np.arange(k) for k in n]
    T0 = np.ascontiguousarray(np.broadcast_to(synth.gaussian_bump(*g1, n), (n[2], n[1], n[0])))
    Ci = np.full(T0.shape, 0.5)
    dd = [oracle.spacing(1.0, k) for k in n]
    dt = oracle.cfl_dt(*dd, 1.0, 0.5)
    ref = oracle.run(T0, Ci, 3, 1.0, dt, *dd)
    with igg.Grid(n) as g:
        T = torch.from_numpy(T0).cuda().reshape(g.shape)
        C = torch.from_numpy(Ci).cuda().reshape(g.shape)
        out = g.run(3, T.clone(), T.clone(), C, 1.0, dt, *dd)
        assert g.device_status() == 0
        gpu = out.cpu().numpy()[0]
    assert np.abs(gpu - ref).max() <= 1e-12 * np.abs(ref).max()
