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
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda().reshape(1, *a.shape)


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


def test_adjoint_rejects_decomposed_grid():
    with igg.Grid((8, 8, 8), dims=(2, 1, 1)) as g:
        t = g.empty()
        with pytest.raises(igg.IggError):
            ag.adjoint_step(g, t.clone(), t, t, t, torch.zeros_like(t), 1.0, 1e-3, 1.0, 1.0, 1.0)
