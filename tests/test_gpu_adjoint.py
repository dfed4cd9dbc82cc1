"""GPU parity of the adjoint form (hand-written adjoint kernel, checkpointed
drivers, torch.autograd.Function) against the FP64 oracle's adjoint, finite
differences and dot-product identities."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")
from paper_2211_15716_gb300 import autograd as ag  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def case(n, seed=4):
    g = [np.arange(k) for k in n]
    Ci_star = np.ascontiguousarray(synth.ci_smooth(seed, *g, n))
    Ci = np.full(Ci_star.shape, 0.53)
    T0 = np.ascontiguousarray(np.broadcast_to(synth.gaussian_bump(*g, n, sigma=0.15), Ci.shape))
    dd = [oracle.spacing(1.0, k) for k in n]
    dt = oracle.cfl_dt(*dd, 1.0, max(Ci.max(), Ci_star.max()))
    return T0, Ci, Ci_star, dd, dt


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.array(a)).to(dtype).cuda().reshape(1, *a.shape)


def test_adjoint_step_matches_oracle():
    n = (21, 13, 17)
    T0, Ci, Ci_star, dd, dt = case(n)
    rng = np.random.default_rng(0)
    lam_in = rng.standard_normal(T0.shape)
    ref_out = np.empty_like(lam_in)
    ref_g = np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, T0, Ci_star, ref_g, 1.0, dt, *dd)
    with igg.Grid(n) as g:
        out = torch.empty((1, *T0.shape), dtype=torch.float64, device="cuda")
        gci = torch.zeros_like(out)
        ag.adjoint_step(g, out, dev(lam_in), dev(T0), dev(Ci_star), gci, 1.0, dt, *dd)
        torch.cuda.synchronize()
        o, gg = out.cpu().numpy()[0], gci.cpu().numpy()[0]
    assert np.abs(o - ref_out).max() <= 1e-12 * np.abs(ref_out).max()
    assert np.abs(gg - ref_g).max() <= 1e-12 * np.abs(ref_g).max()


def test_dot_product_identity_gpu():
    """<A x, y> = <x, A^T y> with the GPU forward step and GPU adjoint step."""
    n = (24, 19, 16)
    _, _, Ci_star, dd, dt = case(n)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(Ci_star.shape)
    y = rng.standard_normal(Ci_star.shape)
    with igg.Grid(n) as g:
        X, Y, C = dev(x), dev(y), dev(Ci_star)
        AX = X.clone()
        g.step(AX, X, C, 1.0, dt, *dd)
        ATY = torch.empty_like(Y)
        gci = torch.zeros_like(Y)
        ag.adjoint_step(g, ATY, Y, X, C, gci, 1.0, dt, *dd)
        lhs = float((AX * Y).sum())
        rhs = float((X * ATY).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(np.abs(x).sum() + np.abs(y).sum())


@pytest.mark.parametrize("nt,every", [(12, 4), (13, 5), (7, 1), (9, 16)])
def test_checkpointed_gradient_matches_oracle(nt, every):
    n = (14, 12, 11)
    T0, Ci, Ci_star, dd, dt = case(n)
    T_obs = oracle.forward_states(T0, Ci_star, nt, 1.0, dt, *dd)[-1]
    J, gT0, gCi = oracle.gradient(T0, np.ascontiguousarray(Ci), T_obs, nt, 1.0, dt, *dd)
    with igg.Grid(n) as g:
        T0d, Cd, Od = dev(T0), dev(Ci), dev(T_obs)
        T_nt, ckpt = ag.forward_checkpointed(g, nt, every, T0d, Cd, 1.0, dt, *dd)
        lam_nt = ag.residual(T_nt, Od)
        J_gpu = 0.5 * igg.reduce(igg.RED_SUM_SQDIFF, T_nt, Od).item()
        gT, gC = ag.adjoint_checkpointed(g, nt, every, ckpt, Cd, lam_nt, 1.0, dt, *dd)
        torch.cuda.synchronize()
        gT, gC = gT.cpu().numpy()[0], gC.cpu().numpy()[0]
    assert J_gpu == pytest.approx(J, rel=1e-10)
    assert np.linalg.norm(gT - gT0) <= 1e-10 * np.linalg.norm(gT0)
    assert np.linalg.norm(gC - gCi) <= 1e-10 * np.linalg.norm(gCi)


def test_autograd_finite_differences_32():
    """torch.autograd through the library, central differences on 32^3."""
    n = (32, 32, 32)
    nt = 20
    T0, Ci, Ci_star, dd, dt = case(n)
    with igg.Grid(n) as g:
        Cs = dev(Ci_star)
        T0d = dev(T0)
        T_obs = ag.solve(T0d, Cs, g, nt, 1.0, dt, *dd).detach()
        rng = np.random.default_rng(3)
        T_obs = T_obs + 1e-3 * torch.from_numpy(rng.standard_normal(T_obs.shape)).cuda()
        C = dev(Ci).requires_grad_(True)
        T = T0d.clone().requires_grad_(True)

        def J(Tin, Cin):
            return 0.5 * ((ag.solve(Tin, Cin, g, nt, 1.0, dt, *dd) - T_obs) ** 2).sum()

        loss = J(T, C)
        loss.backward()
        with torch.no_grad():
            for which in ("Ci", "T0"):
                v = torch.from_numpy(rng.standard_normal(C.shape)).cuda()
                base = C if which == "Ci" else T
                h = 1e-6 * base.norm() / v.norm()
                if which == "Ci":
                    fd = (J(T, C + h * v) - J(T, C - h * v)) / (2 * h)
                    ad = (C.grad * v).sum()
                else:
                    fd = (J(T + h * v, C) - J(T - h * v, C)) / (2 * h)
                    ad = (T.grad * v).sum()
                assert abs(float(fd - ad)) <= 1e-6 * abs(float(ad)), (which, float(fd), float(ad))


def test_fp32_gradient_vs_fp64_oracle():
    """FP32 fields, FP64 gradient accumulation: relative L2 error against the
    FP64 oracle's gradient stays below 1e-3 (stated accuracy of the form)."""
    n = (20, 18, 16)
    nt, every = 16, 4
    T0, Ci, Ci_star, dd, dt = case(n)
    T_obs = oracle.forward_states(T0, Ci_star, nt, 1.0, dt, *dd)[-1]
    J, gT0, gCi = oracle.gradient(T0, np.ascontiguousarray(Ci), T_obs, nt, 1.0, dt, *dd)
    with igg.Grid(n) as g:
        T0d, Cd, Od = (dev(a, torch.float32) for a in (T0, Ci, T_obs))
        T_nt, ckpt = ag.forward_checkpointed(g, nt, every, T0d, Cd, 1.0, dt, *dd)
        gT, gC = ag.adjoint_checkpointed(g, nt, every, ckpt, Cd, ag.residual(T_nt, Od), 1.0, dt, *dd)
        gT, gC = gT.double().cpu().numpy()[0], gC.cpu().numpy()[0]
    assert np.linalg.norm(gC - gCi) <= 1e-3 * np.linalg.norm(gCi)
    assert np.linalg.norm(gT - gT0) <= 1e-3 * np.linalg.norm(gT0)


def test_adjoint_rejects_low_dimensional_grid():
    with igg.Grid((8, 8, 1), dims=(2, 1, 1)) as g:
        t = g.empty()
        with pytest.raises(igg.IggError):
            ag.adjoint_step(g, t.clone(), t, t, t, torch.zeros_like(t), 1.0, 1e-3, 1.0, 1.0, 1.0)


def _adjoint_inputs(n, seed):
    T0, Ci, Ci_star, dd, dt = case(n, seed)
    rng = np.random.default_rng(seed)
    return rng.standard_normal(T0.shape), T0, Ci_star, dd, dt


def _gpu_adjoint(n, lam_in, Tn, Ci, g0, dd, dt, dtype, tma=True):
    with igg.Grid(n) as g:
        g.set_option(igg.Grid.OPT_TMA, 1 if tma else 0)
        out = torch.empty((1, *Tn.shape), dtype=dtype, device="cuda")
        gci = dev(g0)
        ag.adjoint_step(g, out, dev(lam_in, dtype), dev(Tn, dtype), dev(Ci, dtype), gci, 1.0, dt, *dd)
        torch.cuda.synchronize()
        status = g.device_status()
        return out.double().cpu().numpy()[0], gci.cpu().numpy()[0], status


def _stencil_magnitude(lam_in, Ci, dd, dt):
    """|lam_in| + |wc v| + sum_d w_d (|v-| + |v+|) per point, v = Ci lam_in on
    inner points (the scale the adjoint's rounding errors are measured on)."""
    w = [dt / (d * d) for d in dd]
    av = np.zeros_like(lam_in)
    av[1:-1, 1:-1, 1:-1] = np.abs(Ci * lam_in)[1:-1, 1:-1, 1:-1]
    p = np.pad(av, 1)
    m = np.abs(lam_in) + 2 * sum(w) * av
    m += w[0] * (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:])
    m += w[1] * (p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1])
    m += w[2] * (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1])
    return m


@pytest.mark.parametrize("n", [(130, 37, 29), (64, 8, 5), (66, 17, 40), (128, 9, 70)])
def test_adjoint_step_tma_sizes_match_oracle(n):
    """FP64 adjoint step on sizes the TMA kernel takes (rows of a multiple of
    16 bytes): several x tiles with a ragged one, single-row-block and
    multi-chunk z extents; lam_out and gCi against the oracle."""
    lam_in, T0, Ci_star, dd, dt = _adjoint_inputs(n, 5)
    ref_out, ref_g = np.empty_like(lam_in), np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, T0, Ci_star, ref_g, 1.0, dt, *dd)
    g0 = np.zeros_like(lam_in)
    o, gg, status = _gpu_adjoint(n, lam_in, T0, Ci_star, g0, dd, dt, torch.float64)
    assert status == 0
    assert np.abs(o - ref_out).max() <= 1e-12 * np.abs(ref_out).max()
    assert np.abs(gg - ref_g).max() <= 1e-12 * np.abs(ref_g).max()
    # a nonzero gCi on entry is accumulated into, boundary entries untouched
    g1 = np.random.default_rng(7).standard_normal(lam_in.shape)
    _, gg1, _ = _gpu_adjoint(n, lam_in, T0, Ci_star, g1, dd, dt, torch.float64)
    inner = np.zeros(lam_in.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.array_equal(gg1[~inner], g1[~inner])
    assert np.abs(gg1 - (g1 + ref_g)).max() <= 1e-12 * (np.abs(g1).max() + np.abs(ref_g).max())


@pytest.mark.parametrize("dtype,n", [(torch.float64, (130, 37, 29)), (torch.float64, (66, 17, 40)),
                                     (torch.float32, (132, 37, 29)), (torch.float32, (128, 9, 70))])
def test_adjoint_tma_and_tiled_kernels_same_bits(dtype, n):
    """The TMA kernel and the tiled kernel share the per-point arithmetic:
    identical lam_out and gCi bits (FP64 and FP32 fields)."""
    lam_in, T0, Ci_star, dd, dt = _adjoint_inputs(n, 6)
    # a few stencils outside the float-pair ranges (FP64 sum for those points)
    lam_in[3, 4, 5] = 1e-30
    lam_in[7, 2, 9] = 3e20
    lam_in[10, 5, 60 % n[0]] = 0.0
    g0 = np.random.default_rng(8).standard_normal(lam_in.shape)
    a = _gpu_adjoint(n, lam_in, T0, Ci_star, g0, dd, dt, dtype, tma=True)
    b = _gpu_adjoint(n, lam_in, T0, Ci_star, g0, dd, dt, dtype, tma=False)
    assert a[2] == 0 and b[2] == 0
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("tma", [True, False])
def test_adjoint_fp64_sum_for_values_outside_pair_ranges(tma):
    """Stencils holding lam_in or Ci outside the float-pair ranges (tiny,
    huge, zero, subnormal) take the FP64 sum; every point stays within 1e-13
    of its own stencil magnitude of the oracle's result."""
    n = (66, 19, 23)
    lam_in, T0, Ci_star, dd, dt = _adjoint_inputs(n, 9)
    rng = np.random.default_rng(10)
    pick = rng.random(lam_in.shape)
    lam_in = np.where(pick < 0.05, lam_in * 1e-30, lam_in)
    lam_in = np.where((pick >= 0.05) & (pick < 0.1), lam_in * 1e25, lam_in)
    lam_in = np.where((pick >= 0.1) & (pick < 0.12), 0.0, lam_in)
    lam_in = np.where((pick >= 0.12) & (pick < 0.13), 1e-310, lam_in)
    Ci = np.where(rng.random(lam_in.shape) < 0.05, Ci_star * 1e-9, Ci_star)
    ref_out, ref_g = np.empty_like(lam_in), np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, T0, Ci, ref_g, 1.0, dt, *dd)
    o, gg, status = _gpu_adjoint(n, lam_in, T0, Ci, np.zeros_like(lam_in), dd, dt, torch.float64, tma)
    assert status == 0
    mag = _stencil_magnitude(lam_in, Ci, dd, dt)
    assert np.all(np.abs(o - ref_out) <= 1e-13 * mag)


def test_adjoint_weights_outside_pair_range():
    """Weights below 2^-18 (tiny dt): every point takes the FP64 sum."""
    n = (64, 12, 10)
    lam_in, T0, Ci_star, dd, _ = _adjoint_inputs(n, 11)
    dt = 1e-12
    ref_out, ref_g = np.empty_like(lam_in), np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, T0, Ci_star, ref_g, 1.0, dt, *dd)
    o, gg, status = _gpu_adjoint(n, lam_in, T0, Ci_star, np.zeros_like(lam_in), dd, dt, torch.float64)
    assert status == 0
    mag = _stencil_magnitude(lam_in, Ci_star, dd, dt)
    assert np.all(np.abs(o - ref_out) <= 1e-14 * mag)
    assert np.abs(gg - ref_g).max() <= 1e-12 * np.abs(ref_g).max()


@pytest.mark.parametrize("n", [(132, 37, 29), (128, 9, 70)])
def test_adjoint_step_fp32_tma_sizes(n):
    """FP32 fields on TMA sizes: lam_out within FP32 rounding of the oracle's
    adjoint of the same (FP32-representable) inputs, gCi likewise."""
    lam_in, T0, Ci_star, dd, dt = _adjoint_inputs(n, 12)
    lam_in, T0, Ci_star = (a.astype(np.float32).astype(np.float64) for a in (lam_in, T0, Ci_star))
    ref_out, ref_g = np.empty_like(lam_in), np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, T0, Ci_star, ref_g, 1.0, dt, *dd)
    o, gg, status = _gpu_adjoint(n, lam_in, T0, Ci_star, np.zeros_like(lam_in), dd, dt, torch.float32)
    assert status == 0
    mag = _stencil_magnitude(lam_in, Ci_star, dd, dt)
    assert np.all(np.abs(o - ref_out) <= 1e-6 * mag)
    assert np.abs(gg - ref_g).max() <= 1e-5 * np.abs(ref_g).max()


@pytest.mark.parametrize("tma", [True, False])
def test_adjoint_gci_paths_crossing_powers_of_two_and_zero(tma):
    """T_n smooth but crossing zero and several powers of two: stencils of one
    exponent (bit-pattern differences), of two neighbouring exponents
    (shifted significands) and with a sign change (FP64 sum) all meet the
    oracle's gCi within 1e-12 of its largest entry."""
    n = (66, 21, 19)
    lam_in, _, Ci_star, dd, dt = _adjoint_inputs(n, 13)
    g = [np.arange(k) for k in n]
    Tn = np.ascontiguousarray(synth.sine_modes(21, *g, n, base=0.3, amp=1.5))
    assert (Tn < 0).any() and (np.abs(Tn) > 2).any()
    ref_out, ref_g = np.empty_like(lam_in), np.zeros_like(lam_in)
    oracle.adjoint_step(ref_out, lam_in, Tn, Ci_star, ref_g, 1.0, dt, *dd)
    o, gg, status = _gpu_adjoint(n, lam_in, Tn, Ci_star, np.zeros_like(lam_in), dd, dt,
                                 torch.float64, tma)
    assert status == 0
    assert np.abs(gg - ref_g).max() <= 1e-12 * np.abs(ref_g).max()
    assert np.abs(o - ref_out).max() <= 1e-12 * np.abs(ref_out).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_checkpointed_gradient_tma_and_tiled_same_bits(dtype):
    """The checkpointed run on the TMA kernel (FP64: Ci split into pairs once
    per run) and on the tiled kernel give the same bits; some Ci lie outside
    the pair range (their points take the FP64 sum, Ci read from memory)."""
    n = (66, 17, 12)
    nt, every = 9, 4
    T0, Ci, Ci_star, dd, dt = case(n)
    Cm = np.where(np.random.default_rng(5).random(Ci.shape) < 0.05, 1e-9, Ci)
    T_obs = oracle.forward_states(T0, Ci_star, nt, 1.0, dt, *dd)[-1]
    res = []
    for tma in (True, False):
        with igg.Grid(n) as g:
            g.set_option(igg.Grid.OPT_TMA, 1 if tma else 0)
            T0d, Cd, Od = (dev(a, dtype) for a in (T0, Cm, T_obs))
            T_nt, ckpt = ag.forward_checkpointed(g, nt, every, T0d, Cd, 1.0, dt, *dd)
            gT, gC = ag.adjoint_checkpointed(g, nt, every, ckpt, Cd, ag.residual(T_nt, Od), 1.0, dt, *dd)
            torch.cuda.synchronize()
            assert g.device_status() == 0
            res.append((gT.double().cpu().numpy(), gC.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    if dtype == torch.float64:
        J, gT0, gCi = oracle.gradient(T0, np.ascontiguousarray(Cm), T_obs, nt, 1.0, dt, *dd)
        assert np.linalg.norm(res[0][0][0] - gT0) <= 1e-10 * np.linalg.norm(gT0)
        assert np.linalg.norm(res[0][1][0] - gCi) <= 1e-10 * np.linalg.norm(gCi)
