"""GPU parity on 2-D and 1-D grids (a dimension of size 1 is absent) against
the oracle: plain and hidden runs, FP64 (both cells) and FP32, vector and
scalar kernels, decomposed topologies; invalid absent-dimension settings are
rejected."""
import numpy as np
import pytest
import torch

import oracle
from _inputs import grid_fields, oracle_fields

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")
from paper_2211_15716_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


CASES = [
    ((64, 37, 1), (2, 2, 1), (1, 0, 0), (2, 2, 2)),   # 2-D, vector kernel
    ((37, 21, 1), (2, 2, 1), (0, 1, 0), (2, 2, 2)),   # 2-D, scalar kernel (odd nx)
    ((130, 1, 1), (3, 1, 1), (1, 0, 0), (2, 2, 2)),   # 1-D, vector kernel
    ((41, 1, 1), (2, 1, 1), (0, 0, 0), (3, 2, 2)),    # 1-D, scalar kernel, overlap 3
    ((48, 1, 30), (2, 1, 2), (0, 0, 1), (2, 2, 2)),   # x-z plane
]


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
@pytest.mark.parametrize("hidden", [False, True])
@pytest.mark.parametrize("emu", [1, 0])
def test_low_dimensional_fp64_matches_oracle(n, dims, periods, overlap, hidden, emu):
    nt = 7
    T0o, Cio, dd, _ = oracle_fields(n, dims, periods, overlap, 4)
    dt = oracle.cfl_dt(*dd, 1.0, Cio.max())
    widths = tuple(max(2, o) for o in overlap) if hidden else None
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt, *dd, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 4)
        assert np.array_equal(T0, T0o)
        T, Cd = torch.from_numpy(T0).cuda(), torch.from_numpy(Ci).cuda()
        dx, dy, dz, dt2 = wl.setup(wl.Workload("t", n, dims, periods, overlap), g, Cd)
        assert (dx, dy, dz, dt2) == (*dd, dt)
        g.set_option(g.OPT_F64_EMU, emu)
        R = g.run(nt, T, T.clone(), Cd, 1.0, dt, dx, dy, dz, widths=widths)
        torch.cuda.synchronize()
        gpu = R.cpu().numpy()
    assert np.abs(gpu - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,dims,periods,overlap", CASES[:3])
def test_low_dimensional_fp32_within_bound(n, dims, periods, overlap):
    nt = 7
    T0o, Cio, dd, _ = oracle_fields(n, dims, periods, overlap, 5)
    dt = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt, *dd, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 5)
        T = torch.from_numpy(T0).float().cuda()
        Cd = torch.from_numpy(Ci).float().cuda()
        R = g.run(nt, T, T.clone(), Cd, 1.0, dt, *dd, widths=(2, 2, 2))
        torch.cuda.synchronize()
        gpu = R.double().cpu().numpy()
    assert np.abs(gpu - ref).max() <= (1 + nt) * 2 * 2.0 ** -24 * np.abs(ref).max()


def test_absent_dimension_errors():
    with pytest.raises(igg.IggError):
        igg.Grid((16, 8, 1), dims=(1, 1, 2))
    with pytest.raises(igg.IggError):
        igg.Grid((16, 8, 1), dims=(2, 1, 1), periods=(0, 0, 1))
    with igg.Grid((16, 8, 1), dims=(0, 0, 0), nsub=4) as g:
        assert g.dims[2] == 1 and g.global_size()[2] == 1
