"""GPU parity of the library (through the C ABI) against the FP64 oracle.

Bars: halo updates bit exact; FP64 steps within 1e-12 of max|T| of the
oracle; split and unsplit steps bit-identical to each other on the GPU;
FP32 within (1 + nt) * 2 * 2^-24 * max|T| (input rounding plus at most about
two FP32 ulps per step, the scheme being non-expansive in the max norm under
the 6.1 CFL rule); BF16 storage within one BF16 ulp of the oracle's one-step
result on the same BF16 inputs, rounded to BF16."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _inputs import grid_fields, oracle_fields

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")
from paper_2211_15716_gb300 import workloads as wl  # noqa: E402

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def dev(a, dtype=torch.float64):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype == torch.bfloat16:
        bits = synth.to_bf16_bits(np.asarray(a))
        return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    return t.to(dtype).cuda()


def rel_err(gpu, ref):
    return float(np.abs(gpu - ref).max() / np.abs(ref).max())


CASES = [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2)),
    ((8, 7, 6), (2, 2, 2), (1, 0, 0), (2, 2, 2)),
    ((9, 6, 11), (3, 1, 2), (0, 1, 1), (2, 2, 2)),
    ((13, 7, 9), (3, 1, 2), (1, 1, 1), (2, 3, 2)),
    ((10, 9, 8), (1, 1, 1), (1, 1, 1), (2, 2, 2)),
    ((7, 7, 7), (2, 1, 1), (1, 0, 1), (3, 2, 2)),
    ((37, 21, 19), (2, 2, 1), (1, 1, 0), (2, 2, 2)),   # several tiles and ragged tails
    ((70, 18, 12), (1, 2, 2), (0, 0, 1), (2, 2, 2)),
]


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
def test_grid_bookkeeping_matches_oracle(n, dims, periods, overlap):
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        assert g.global_size() == oracle.global_size(n, dims, overlap, periods)
        left, right = oracle.neighbours(dims, periods)
        for s in range(g.nsub):
            info = g.subdomain_info(s)
            assert info["coords"] == oracle.coords(s, dims)
            assert info["left"] == tuple(left[s]) and info["right"] == tuple(right[s])
            for a, b in zip(g.global_indices(s), oracle.global_indices(n, dims, overlap, periods, s)):
                assert np.array_equal(a, b)


def test_dims_create_matches_oracle():
    for nsub in (1, 2, 6, 8, 12, 16, 30):
        with igg.Grid((6, 6, 6), nsub=nsub) as g:
            assert g.dims == oracle.dims_create(nsub)


@pytest.mark.parametrize("es,npdt,tdt", [(8, np.uint64, torch.float64), (4, np.uint32, torch.float32),
                                         (2, np.uint16, torch.bfloat16)])
@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
def test_halo_bit_exact(n, dims, periods, overlap, es, npdt, tdt):
    """update_halo! on random bit patterns: every point equal bit for bit."""
    rng = np.random.default_rng(7)
    nsub = dims[0] * dims[1] * dims[2]
    bits = rng.integers(0, np.iinfo(npdt).max, size=(nsub, n[2], n[1], n[0]), dtype=npdt, endpoint=True)
    ref = bits.copy()
    oracle.update_halo(ref, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        itype = {8: torch.int64, 4: torch.int32, 2: torch.int16}[es]
        t = torch.from_numpy(bits.view({8: np.int64, 4: np.int32, 2: np.int16}[es])).cuda()
        f = t.view(tdt)
        g.update_halo(f)
        out = f.view(itype).cpu().numpy().view(npdt)
    assert np.array_equal(out, ref)


def test_halo_several_fields_one_call():
    n, dims, periods, o = (9, 8, 7), (2, 2, 1), (1, 0, 0), (2, 2, 2)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((4, n[2], n[1], n[0]))
    b = rng.standard_normal(a.shape)
    ra, rb = a.copy(), b.copy()
    oracle.update_halo(ra, dims, periods, o)
    oracle.update_halo(rb, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        ta, tb = dev(a), dev(b)
        g.update_halo(ta, tb)
        assert np.array_equal(ta.cpu().numpy(), ra) and np.array_equal(tb.cpu().numpy(), rb)


def _run_both(n, dims, periods, overlap, nt, widths, seed=0, tkind="gaussian_rough", f64_emu=1):
    T0o, Cio, dd, ng = oracle_fields(n, dims, periods, overlap, seed, tkind)
    dt_o = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt_o, *dd, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, seed, tkind)
        assert np.array_equal(T0, T0o) and np.array_equal(Ci, Cio)
        T, Cd = dev(T0), dev(Ci)
        T2 = T.clone()
        w = wl.Workload("t", n, dims, periods, overlap)
        dx, dy, dz, dt = wl.setup(w, g, Cd)
        assert (dx, dy, dz, dt) == (*dd, dt_o)
        g.set_option(g.OPT_F64_EMU, f64_emu)
        res = g.run(nt, T, T2, Cd, 1.0, dt, dx, dy, dz, widths=widths)
        torch.cuda.synchronize()
        return res.cpu().numpy(), ref


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
@pytest.mark.parametrize("hidden", [False, True])
@pytest.mark.parametrize("emu", [1, 0])
def test_fp64_run_matches_oracle(n, dims, periods, overlap, hidden, emu):
    widths = tuple(max(2, o) for o in overlap) if hidden else None
    gpu, ref = _run_both(n, dims, periods, overlap, nt=7, widths=widths, f64_emu=emu)
    assert rel_err(gpu, ref) <= FP64_TOL
    # halo points are copies of computed points: compare them too (all points)
    assert np.isfinite(gpu).all()


@pytest.mark.parametrize("n,dims,periods,overlap", CASES[:4] + CASES[6:])
@pytest.mark.parametrize("widths", [(2, 2, 2), (16, 2, 2), (3, 4, 5)])
def test_split_bit_identical_to_unsplit(n, dims, periods, overlap, widths):
    """igg_step_hidden == igg_step + igg_update_halo, bit for bit."""
    widths = tuple(max(w, o) for w, o in zip(widths, overlap))
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 5)
        T, Cd = dev(T0), dev(Ci)
        dx, dy, dz, dt = wl.setup(wl.Workload("t", n), g, Cd)
        A, B = T.clone(), T.clone()
        g.step(A, T, Cd, 1.0, dt, dx, dy, dz)
        g.update_halo(A)
        g.step_hidden(widths, B, T, Cd, 1.0, dt, dx, dy, dz)
        torch.cuda.synchronize()
        assert torch.equal(A.view(torch.int64), B.view(torch.int64))


def test_single64_nt100_matches_oracle():
    """64^3 single grid, Gaussian bump, c0 ~ U[1.5,2.5], nt = 100."""
    w = wl.WORKLOADS["single64"]
    n = w.n
    g1 = [np.arange(k) for k in n]
    T0o = synth.gaussian_bump(*g1, n) * np.ones((n[2], n[1], n[0]))
    Cio = np.ascontiguousarray(synth.ci_uniform_c0(w.seed, *g1, n))
    dd = [oracle.spacing(1.0, k) for k in n]
    dt_o = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = oracle.run(np.ascontiguousarray(T0o), Cio, w.nt, 1.0, dt_o, *dd)
    with igg.Grid(n) as g:
        T, T2, Ci = wl.make_fields(w, g)
        dx, dy, dz, dt = wl.setup(w, g, Ci)
        assert dt == dt_o
        res = g.run(w.nt, T, T2, Ci, w.lam, dt, dx, dy, dz)
        gpu = res.cpu().numpy()[0]
    assert rel_err(gpu, ref) <= FP64_TOL
    assert np.abs(ref - T0o).max() > 1e-3


@pytest.mark.parametrize("nt", [0, 1, 2, 3])
def test_run_parity_of_nt(nt):
    """nt = 0 leaves T; odd nt leaves the newest state in T2."""
    n, dims, periods, o = (12, 10, 9), (1, 1, 1), (0, 0, 0), (2, 2, 2)
    gpu, ref = _run_both(n, dims, periods, o, nt=nt, widths=None)
    assert rel_err(gpu, ref) <= FP64_TOL


@pytest.mark.parametrize("nt", [3, 4])
def test_run_host_matches_run_and_oracle(nt):
    """igg_run_host (host fields in, H2D, T2 = copy(T), nt hidden steps, D2H
    of the newest state) equals igg_run on device fields bit for bit, and the
    oracle within the FP64 bar."""
    n, dims, periods, o = (70, 18, 12), (2, 2, 1), (1, 0, 0), (2, 2, 2)
    T0o, Cio, dd, ng = oracle_fields(n, dims, periods, o, 4)
    dt = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt, *dd, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        T0, Ci = grid_fields(g, 4)
        Th = torch.from_numpy(T0.copy()).pin_memory()
        Ch = torch.from_numpy(Ci.copy()).pin_memory()
        T, T2, Cd = (torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(3))
        g.run_host(nt, Th, Ch, T, T2, Cd, 1.0, dt, *dd, widths=(16, 2, 2))
        torch.cuda.synchronize()
        A = dev(T0)
        r = g.run(nt, A, A.clone(), dev(Ci), 1.0, dt, *dd, widths=(16, 2, 2))
        assert torch.equal(Th.view(torch.int64), r.cpu().view(torch.int64))
    assert rel_err(Th.numpy(), ref) <= FP64_TOL


def test_minimum_size_one_inner_point():
    n = (3, 3, 3)
    gpu, ref = _run_both(n, (1, 1, 1), (0, 0, 0), (2, 2, 2), nt=3, widths=(2, 2, 2))
    assert rel_err(gpu, ref) <= FP64_TOL


def test_widths_larger_than_array():
    n, dims, periods, o = (9, 8, 7), (2, 1, 1), (0, 0, 0), (2, 2, 2)
    gpu, ref = _run_both(n, dims, periods, o, nt=4, widths=(20, 20, 20))
    assert rel_err(gpu, ref) <= FP64_TOL


def test_fp32_matches_oracle_within_bound():
    n, dims, periods, o = (40, 24, 18), (2, 1, 2), (1, 0, 0), (2, 2, 2)
    nt = 50
    T0o, Cio, dd, ng = oracle_fields(n, dims, periods, o, 3, "gaussian")
    dt = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt, *dd, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        T, Cd = dev(T0o, torch.float32), dev(Cio, torch.float32)
        T2 = T.clone()
        res = g.run(nt, T, T2, Cd, 1.0, dt, *dd, widths=(16, 2, 2))
        gpu = res.double().cpu().numpy()
    err = np.abs(gpu - ref).max()
    bound = (1 + nt) * 2 * 2.0 ** -24 * np.abs(ref).max()
    assert err <= bound, (err, bound)


def test_bf16_one_step_within_one_ulp():
    """One BF16-storage step vs the oracle's FP64 step on the same BF16
    inputs, rounded to BF16: at most one BF16 ulp apart everywhere."""
    n, dims, periods, o = (40, 20, 16), (2, 1, 1), (0, 0, 0), (2, 2, 2)
    T0o, Cio, dd, ng = oracle_fields(n, dims, periods, o, 4, "gaussian_rough")
    Tb = synth.bf16_bits_to_f64(synth.to_bf16_bits(T0o))
    Cb = synth.bf16_bits_to_f64(synth.to_bf16_bits(Cio))
    dt = oracle.cfl_dt(*dd, 1.0, Cio.max())
    ref = Tb.copy()
    for s in range(ref.shape[0]):
        oracle.step(ref[s], np.ascontiguousarray(Tb[s]), np.ascontiguousarray(Cb[s]), 1.0, dt, *dd)
    ref_b = oracle.round_to_bf16(ref)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        T, Cd = dev(T0o, torch.bfloat16), dev(Cio, torch.bfloat16)
        T2 = T.clone()
        g.step(T2, T, Cd, 1.0, dt, *dd)
        gpu = T2.double().cpu().numpy()
    diff = np.abs(gpu - ref_b)
    assert (diff <= oracle.bf16_ulp(ref_b)).all()
    assert (diff == 0).mean() > 0.99


def test_reductions_match_oracle():
    rng = np.random.default_rng(11)
    a = rng.uniform(1.0, 3.0, 1_000_003)
    b = rng.uniform(0.4, 0.7, a.size)
    ta, tb = dev(a), dev(b)
    assert igg.reduce(igg.RED_MAX, ta).item() == a.max()
    assert igg.reduce(igg.RED_SUM, ta).item() == pytest.approx(oracle.fsum(a), rel=1e-13)
    assert igg.reduce(igg.RED_SUM_DIV, ta, tb).item() == pytest.approx(oracle.fsum(a / b), rel=1e-13)
    assert igg.reduce(igg.RED_SUM_SQDIFF, ta, tb).item() == pytest.approx(oracle.fsum((a - b) ** 2), rel=1e-13)
    # deterministic: same bits on a second call
    x1 = igg.reduce(igg.RED_SUM, ta).item()
    assert igg.reduce(igg.RED_SUM, ta).item() == x1
    # empty input
    assert igg.reduce(igg.RED_SUM, ta[:0]).item() == 0.0


def test_misaligned_pointer_rejected():
    with igg.Grid((8, 8, 8)) as g:
        buf = torch.zeros(8 * 8 * 8 + 1, dtype=torch.float64, device="cuda")
        T = buf[1:]
        with pytest.raises(igg.IggError) as e:
            g.step(T.clone(), T, T.clone(), 1.0, 1e-3, 1.0, 1.0, 1.0)
        assert e.value.code == -1


def test_widths_below_overlap_rejected():
    with igg.Grid((8, 8, 8), overlap=(3, 2, 2)) as g:
        T = g.empty()
        with pytest.raises(igg.IggError):
            g.step_hidden((2, 2, 2), T.clone(), T, T.clone(), 1.0, 1e-3, 1.0, 1.0, 1.0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,dims,periods,overlap,widths", [
    ((64, 37, 29), (2, 1, 2), (1, 0, 0), (2, 2, 2), (16, 2, 2)),
    ((144, 40, 70), (1, 2, 1), (0, 1, 0), (2, 2, 2), (3, 4, 5)),
    ((256, 33, 18), (2, 2, 2), (1, 0, 1), (2, 3, 2), (16, 3, 2)),
    ((64, 37, 29), (1, 1, 2), (0, 0, 0), (2, 2, 2), (40, 20, 20)),  # empty inner block
])
def test_tma_and_vector_kernels_same_bits(dtype, n, dims, periods, overlap, widths):
    """The TMA-pipelined kernel and the register-pipelined vector kernel give
    identical bits for the full step and the hidden step, and the device
    error word stays clear."""
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 8)
        T, Cd = dev(T0, dtype), dev(Ci, dtype)
        dx, dy, dz, dt = wl.setup(wl.Workload("t", n), g, dev(Ci))
        outs = []
        for tma in (1, 0):
            g.set_option(g.OPT_TMA, tma)
            A, B = T.clone(), T.clone()
            g.step(A, T, Cd, 1.0, dt, dx, dy, dz)
            g.step_hidden(widths, B, T, Cd, 1.0, dt, dx, dy, dz)
            R = g.run(5, T.clone(), T.clone(), Cd, 1.0, dt, dx, dy, dz, widths=widths)
            torch.cuda.synchronize()
            outs.append((A, B, R))
        assert g.device_status() == 0
        iv = {torch.float64: torch.int64, torch.float32: torch.int32, torch.bfloat16: torch.int16}[dtype]
        for a, b in zip(outs[0], outs[1]):
            assert torch.equal(a.view(iv), b.view(iv))


def test_tma_full_size_decomposed_matches_oracle():
    """The benchmark's launch configuration (2x2x2 x 512x256x256 FP64,
    widths (16,2,2), graph loop) at full size: 2 hidden steps through the
    TMA path, every point compared with the oracle."""
    w = wl.WORKLOADS["decomposed_2x2x2_512x256x256"]
    with igg.Grid(w.n, dims=w.dims, overlap=w.overlap, periods=w.periods) as g:
        T, T2, Ci = wl.make_fields(w, g)
        dx, dy, dz, dt = wl.setup(w, g, Ci)
        T0 = T.cpu().numpy()
        Cih = Ci.cpu().numpy()
        res = g.run(2, T, T2, Ci, w.lam, dt, dx, dy, dz, widths=w.widths)
        gpu = res.cpu().numpy()
        assert g.device_status() == 0
    oracle.set_threads(0)
    ref = oracle.run_decomposed(T0, Cih, 2, w.lam, dt, dx, dy, dz, w.dims, w.periods, w.overlap,
                                widths=w.widths)
    assert rel_err(gpu, ref) <= FP64_TOL


@pytest.mark.parametrize("emu", [1, 0])
def test_fp64_stationarity_bit_exact(emu):
    """A constant field is a fixed point bit for bit, in both FP64 cells."""
    n = (64, 20, 18)
    with igg.Grid(n) as g:
        g.set_option(g.OPT_F64_EMU, emu)
        T = torch.full(g.shape, 1.7, dtype=torch.float64, device="cuda")
        Ci = dev(grid_fields(g, 3)[1])
        T2 = g.run(5, T, T.clone(), Ci, 1.0, 1e-5, 0.01, 0.01, 0.01)
        assert torch.equal(T2, torch.full_like(T2, 1.7))


@pytest.mark.parametrize("kind", ["sign_changes", "wide_exponents", "binade_crossing"])
def test_fp64_emulation_hard_fields(kind):
    """Fields that send many points to the FP64 fallback of the emulated cell
    (values of both signs, near zero, exponents spanning 10^-30..10^30, values
    straddling powers of two) still match the oracle within 1e-12, and the
    emulated and FP64 cells agree to a few FP64 roundings."""
    n = (64, 24, 20)
    g1 = [np.arange(k) for k in n]
    rng = np.random.default_rng(12)
    base = np.ascontiguousarray(synth.gaussian_bump(*g1, n, sigma=0.2) * np.ones((n[2], n[1], n[0])))
    if kind == "sign_changes":
        T0 = base - 2.2 + 1e-3 * rng.standard_normal(base.shape)
    elif kind == "wide_exponents":
        T0 = np.exp(rng.uniform(-69, 69, base.shape)) * (1 + 0.01 * base)
    else:
        T0 = 2.0 + 0.05 * rng.standard_normal(base.shape)
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(1, *g1, n))
    dd = [oracle.spacing(1.0, k) for k in n]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    nt = 6
    ref = oracle.run(np.ascontiguousarray(T0), Ci, nt, 1.0, dt, *dd)
    outs = []
    with igg.Grid(n) as g:
        for emu in (1, 0):
            g.set_option(g.OPT_F64_EMU, emu)
            T = torch.from_numpy(T0).cuda().view(g.shape)
            outs.append(g.run(nt, T.clone(), T.clone(), dev(Ci).view(g.shape), 1.0, dt, *dd).cpu().numpy()[0])
    for o in outs:
        assert np.abs(o - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(outs[0] - outs[1]).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("spacing", [(0.01, 0.01, 0.01), (0.006, 0.01, 0.01), (0.006, 0.01, 0.013),
                                     (0.01, 0.01, 0.006)])
def test_fp64_weight_groups_match_oracle(spacing):
    """The emulated FP64 cell adds the second differences of equal weights
    exactly before its products (all three weights equal, wy == wz, or none
    grouped when only wx == wy): each grouping matches the oracle within
    1e-12, and the TMA and vector kernels, full and hidden steps, give the
    same bits."""
    n, dims, periods, overlap = (70, 21, 19), (2, 1, 2), (1, 0, 0), (2, 2, 2)
    widths = (16, 2, 2)
    T0o, Cio, _, _ = oracle_fields(n, dims, periods, overlap, 4)
    dt = oracle.cfl_dt(*spacing, 1.0, Cio.max())
    nt = 7
    ref = oracle.run_decomposed(T0o, Cio, nt, 1.0, dt, *spacing, dims, periods, overlap)
    outs = []
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 4)
        T, Cd = dev(T0), dev(Ci)
        for tma in (1, 0):
            g.set_option(g.OPT_TMA, tma)
            for wd in (None, widths):
                R = g.run(nt, T.clone(), T.clone(), Cd, 1.0, dt, *spacing, widths=wd)
                torch.cuda.synchronize()
                outs.append(R)
        assert g.device_status() == 0
    for R in outs:
        assert rel_err(R.cpu().numpy(), ref) <= FP64_TOL
        assert torch.equal(R.view(torch.int64), outs[0].view(torch.int64))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,dims,periods,overlap", [
    ((64, 21, 19), (2, 2, 2), (0, 0, 0), (2, 2, 2)),   # faces, edges and corners
    ((64, 21, 19), (2, 2, 2), (1, 1, 1), (2, 2, 2)),   # periodic
    ((64, 37, 29), (1, 1, 1), (1, 1, 1), (2, 2, 2)),   # its own neighbour
    ((128, 20, 18), (2, 3, 1), (1, 0, 1), (3, 2, 3)),  # overlap 3
])
def test_fused_halo_same_bits_as_split(dtype, n, dims, periods, overlap):
    """The hidden step with the halo update fused into the step launch gives
    the same bits, halo cells included, as the boundary/inner split with
    plane copies, and matches the oracle (FP64)."""
    widths = tuple(max(2, o) for o in overlap)
    T0o, Cio, dd, _ = oracle_fields(n, dims, periods, overlap, 6)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 6)
        T, Cd = dev(T0, dtype), dev(Ci, dtype)
        dx, dy, dz, dt = wl.setup(wl.Workload("t", n), g, dev(Ci))
        outs = []
        for fused in (1, 0):
            g.set_option(g.OPT_FUSED_HALO, fused)
            R = g.run(5, T.clone(), T.clone(), Cd, 1.0, dt, dx, dy, dz, widths=widths)
            torch.cuda.synchronize()
            outs.append(R)
        assert g.device_status() == 0
    iv = {torch.float64: torch.int64, torch.float32: torch.int32, torch.bfloat16: torch.int16}[dtype]
    assert torch.equal(outs[0].view(iv), outs[1].view(iv))
    if dtype == torch.float64:
        ref = oracle.run_decomposed(T0o, Cio, 5, 1.0, dt, *dd, dims, periods, overlap)
        assert rel_err(outs[0].cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,dims,periods,overlap", [
    ((70, 21, 19), (2, 2, 2), (1, 0, 0), (2, 2, 2)),   # faces, edges, corners; periodic in x
    ((72, 18, 12), (2, 1, 1), (1, 0, 0), (2, 2, 2)),   # exchange in x only
    ((70, 20, 14), (1, 2, 2), (0, 1, 0), (2, 3, 2)),   # overlap 3: sent planes off the halo
    ((70, 20, 12), (1, 1, 1), (1, 1, 1), (2, 2, 2)),   # periodic self-neighbours
    ((200, 40, 36), (2, 2, 2), (0, 0, 1), (2, 2, 2)),  # several tiles per row, inner tiles
])
def test_hidden_halo_beside_inner_tiles_same_bits(dtype, n, dims, periods, overlap):
    """The hidden step with the face tiles first and the halo update beside
    the inner tiles (IGG_OPT_HIDE_HALO) gives the bits of the full step
    followed by the halo update, over several steps."""
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0, Ci = grid_fields(g, 5, "gaussian_rough")
        w = wl.Workload("h", n, dims, periods, overlap)
        Cd = dev(Ci, dtype)
        dx, dy, dz, dt = wl.setup(w, g, dev(Ci))
        outs = []
        for hide in (1, 0):
            g.set_option(g.OPT_HIDE_HALO, hide)
            T = dev(T0, dtype)
            r = g.run(5, T, T.clone(), Cd, 1.0, dt, dx, dy, dz, widths=(16, 4, 4))
            r2 = T.clone()
            g.step_hidden((16, 4, 4), r2, r, Cd, 1.0, dt, dx, dy, dz)
            torch.cuda.synchronize()
            outs.append((r.view(torch.uint8).cpu().numpy(), r2.view(torch.uint8).cpu().numpy()))
        assert g.device_status() == 0
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
