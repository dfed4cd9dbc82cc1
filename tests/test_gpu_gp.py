"""GPU parity of the Gross-Pitaevskii step (igg_gp_step) against the
oracle's decomposed runs (FP64 within 1e-12, FP32 within its bound, 2-D
grids included) and conservation of the linear invariant on the GPU."""
import math

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


def inputs(n, dims, periods, o, seed):
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, o, periods)
    lin = np.arange(ng[0] * ng[1] * ng[2], dtype=np.uint64)
    G = [(synth.uniform(seed, k, lin) - (0.5 if k < 3 else 0.0)).reshape(ng[2], ng[1], ng[0])
         for k in (1, 2, 3)]
    out = [np.empty((nsub, n[2], n[1], n[0])) for _ in range(3)]
    for s in range(nsub):
        gi = oracle.global_indices(n, dims, o, periods, s)
        for A, B in zip(out, G):
            A[s] = B[np.ix_(gi[2], gi[1], gi[0])]
    return out


CASES = [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0)),
    ((40, 21, 19), (2, 1, 2), (1, 0, 1)),
    ((33, 17, 9), (1, 2, 2), (1, 1, 1)),
    ((64, 30, 1), (2, 2, 1), (1, 0, 0)),   # 2-D
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,dims,periods", CASES)
def test_gp_matches_oracle(n, dims, periods, dtype):
    o = (2, 2, 2)
    g, nt = 0.9, 8
    dd = (0.1, 0.12, math.inf if n[2] == 1 else 0.09)
    dt = 0.3 / (2 * sum(1 / h ** 2 for h in dd) + 1.0 + 2 * g)
    U, Vv, Pot = inputs(n, dims, periods, o, 7)
    ru, rv = U.copy(), Vv.copy()
    oracle.gp_run_decomposed(ru, rv, Pot, nt, g, dt, *dd, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as gr:
        u, v, P = (torch.from_numpy(a).to(dtype).cuda() for a in (U, Vv, Pot))
        for _ in range(nt):
            gr.gp_step(u, v, P, g, dt, *dd)
        torch.cuda.synchronize()
        gu, gv = u.double().cpu().numpy(), v.double().cpu().numpy()
    tol = 1e-12 if dtype == torch.float64 else 4e-6 * nt
    for a, r in ((gu, ru), (gv, rv)):
        assert np.abs(a - r).max() <= tol * np.abs(r).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,dims,periods", [
    ((40, 12, 10), (2, 1, 2), (1, 0, 0)),   # a periodic ring of two in x
    ((24, 12, 10), (1, 2, 1), (1, 0, 0)),   # its own x neighbour
    ((32, 10, 12), (3, 1, 1), (0, 0, 1)),   # a middle subdomain with both x neighbours
])
def test_gp_overlap3_x_matches_oracle(n, dims, periods, dtype):
    """Overlap 3 in x on the TMA kernel, whose half steps store the x
    exchange's planes (n - 3 and 2) into the neighbours' halo columns
    themselves: halo cells included, the run matches the oracle's decomposed
    run."""
    o = (3, 2, 2)
    g, nt = 0.9, 6
    dd = (0.1, 0.12, 0.09)
    dt = 0.3 / (2 * sum(1 / h ** 2 for h in dd) + 1.0 + 2 * g)
    U, Vv, Pot = inputs(n, dims, periods, o, 9)
    ru, rv = U.copy(), Vv.copy()
    oracle.gp_run_decomposed(ru, rv, Pot, nt, g, dt, *dd, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as gr:
        u, v, P = (torch.from_numpy(a).to(dtype).cuda() for a in (U, Vv, Pot))
        for _ in range(nt):
            gr.gp_step(u, v, P, g, dt, *dd)
        torch.cuda.synchronize()
        gu, gv = u.double().cpu().numpy(), v.double().cpu().numpy()
    tol = 1e-12 if dtype == torch.float64 else 4e-6 * nt
    for a, r in ((gu, ru), (gv, rv)):
        assert np.abs(a - r).max() <= tol * np.abs(r).max()


def test_gp_linear_invariant_gpu():
    """g = 0, zero boundary values: ||u^n||^2 + <v^{n+1/2}, v^{n-1/2}> stays
    the same after every step (u^n, v^{n+1/2} after step n)."""
    n = (48, 40, 36)
    dd = (0.1, 0.12, 0.09)
    g1 = [np.arange(k) for k in n]
    bump = np.broadcast_to(synth.gaussian_bump(*g1, n, sigma=0.2) - 1.7, (n[2], n[1], n[0]))
    inner = np.zeros((n[2], n[1], n[0]))
    inner[1:-1, 1:-1, 1:-1] = 1.0
    U = np.ascontiguousarray(bump * inner)[None]
    Vv = np.ascontiguousarray(0.3 * bump * inner * np.cos(np.arange(n[0]) * 0.7))[None]
    Pot = np.zeros_like(U)
    dt = 0.2 / (2 * sum(1 / h ** 2 for h in dd))
    with igg.Grid(n) as gr:
        u, v, P = (torch.from_numpy(a).cuda() for a in (U, Vv, Pot))
        vprev = Vv[0]
        vals = []
        for _ in range(100):
            gr.gp_step(u, v, P, 0.0, dt, *dd, halo=False)
            torch.cuda.synchronize()
            vn = v.cpu().numpy()[0]
            vals.append(oracle.gp_invariant(u.cpu().numpy()[0], vprev, vn))
            vprev = vn
    assert np.abs(np.array(vals) - vals[0]).max() <= 1e-11 * vals[0]


def _gp_run(n, dims, periods, U, Vv, Pot, g, dt, dd, nt, dtype, tma):
    o = (2, 2, 2)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as gr:
        gr.set_option(igg.Grid.OPT_TMA, 1 if tma else 0)
        u, v, P = (torch.from_numpy(a).to(dtype).cuda() for a in (U, Vv, Pot))
        for _ in range(nt):
            gr.gp_step(u, v, P, g, dt, *dd)
        torch.cuda.synchronize()
        assert gr.device_status() == 0
        return u.double().cpu().numpy(), v.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gp_tma_and_tiled_kernels_same_bits(dtype):
    """The TMA kernel (several x tiles with a ragged one, two subdomains) and
    the tiled kernel share the per-point arithmetic: identical bits."""
    n, dims, periods = (132, 37, 29), (2, 1, 1), (1, 0, 0)
    g, nt = 0.9, 4
    dd = (0.1, 0.12, 0.09)
    dt = 0.3 / (2 * sum(1 / h ** 2 for h in dd) + 1.0 + 2 * g)
    U, Vv, Pot = inputs(n, dims, periods, (2, 2, 2), 11)
    a = _gp_run(n, dims, periods, U, Vv, Pot, g, dt, dd, nt, dtype, True)
    b = _gp_run(n, dims, periods, U, Vv, Pot, g, dt, dd, nt, dtype, False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("tma", [True, False])
def test_gp_fp64_values_outside_pair_ranges(tma):
    """Fields holding tiny, huge and zero values (FP64 sum at those points)
    still meet the oracle within 1e-12 of the largest value."""
    n, dims, periods = (66, 21, 19), (1, 1, 1), (0, 0, 0)
    g, nt = 0.9, 3
    dd = (0.1, 0.12, 0.09)
    dt = 0.3 / (2 * sum(1 / h ** 2 for h in dd) + 1.0 + 2 * g)
    U, Vv, Pot = inputs(n, dims, periods, (2, 2, 2), 12)
    rng = np.random.default_rng(3)
    pick = rng.random(U.shape)
    U = np.where(pick < 0.03, U * 1e-20, U)
    U = np.where((pick >= 0.03) & (pick < 0.05), 0.0, U)
    Vv = np.where(pick > 0.98, Vv * 1e-30, Vv)
    ru, rv = U.copy(), Vv.copy()
    oracle.gp_run_decomposed(ru, rv, Pot, nt, g, dt, *dd, dims, periods, (2, 2, 2))
    gu, gv = _gp_run(n, dims, periods, U, Vv, Pot, g, dt, dd, nt, torch.float64, tma)
    for a, r in ((gu, ru), (gv, rv)):
        assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max()
