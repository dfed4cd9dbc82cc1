"""GPU parity of the adjoint on grids of subdomains (the differentiated form
of Fig. 1's solver on the implicit global grid) against the oracle: the
transpose of the halo update bit for bit, checkpointed gradients against
oracle.gradient_decomposed, torch.autograd against central differences."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")
from paper_2211_15716_gb300 import autograd as ag  # noqa: E402

CASES = [
    ((24, 14, 12), (2, 2, 2), (1, 0, 0), (2, 2, 2)),   # TMA adjoint kernel per subdomain
    ((21, 13, 11), (3, 1, 2), (0, 1, 1), (2, 2, 2)),   # tiled kernel (odd rows)
    ((24, 12, 10), (1, 1, 1), (1, 1, 1), (2, 2, 2)),   # periodic self-neighbours
    ((26, 14, 12), (2, 2, 1), (0, 0, 0), (3, 2, 2)),   # overlap 3
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    oracle.build()


def _fields(n, dims, periods, overlap, seed=4):
    left, _ = oracle.neighbours(dims, periods)
    nsub = left.shape[0]
    ng = oracle.global_size(n, dims, overlap, periods)
    T0 = np.empty((nsub, n[2], n[1], n[0]))
    Ci = np.empty_like(T0)
    for s in range(nsub):
        g = oracle.global_indices(n, dims, overlap, periods, s)
        T0[s] = synth.gaussian_bump(*g, ng, sigma=0.2)
        Ci[s] = synth.ci_uniform_c0(seed, *g, ng)
    dd = [oracle.spacing(1.0, ng[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    return np.ascontiguousarray(T0), np.ascontiguousarray(Ci), dd, dt


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
def test_halo_adjoint_bit_exact(n, dims, periods, overlap):
    rng = np.random.default_rng(7)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        lam = rng.standard_normal(g.shape)
        ref = lam.copy()
        oracle.update_halo_adjoint(ref, dims, periods, overlap)
        t = torch.from_numpy(lam).cuda()
        ag.update_halo_adjoint(g, t)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), ref)
        # FP32: the same adds in FP32
        t32 = torch.from_numpy(lam.astype(np.float32)).cuda()
        ag.update_halo_adjoint(g, t32)
        r32 = lam.astype(np.float32).astype(np.float64)
        oracle.update_halo_adjoint(r32, dims, periods, overlap)
        assert np.allclose(t32.double().cpu().numpy(), r32, rtol=2e-7, atol=1e-6)


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
@pytest.mark.parametrize("nt,every", [(9, 4), (6, 1)])
def test_decomposed_checkpointed_gradient_matches_oracle(n, dims, periods, overlap, nt, every):
    T0, Ci, dd, dt = _fields(n, dims, periods, overlap)
    T_obs = oracle.run_decomposed(T0, Ci * 1.05, nt, 1.0, dt, *dd, dims, periods, overlap)
    J, gT0, gCi = oracle.gradient_decomposed(T0, Ci, T_obs, nt, 1.0, dt, *dd, dims, periods,
                                             overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0d, Cd, Od = (torch.from_numpy(a).cuda() for a in (T0, Ci, T_obs))
        T_nt, ckpt = ag.forward_checkpointed(g, nt, every, T0d, Cd, 1.0, dt, *dd)
        ref_nt = oracle.run_decomposed(T0, Ci, nt, 1.0, dt, *dd, dims, periods, overlap)
        assert np.abs(T_nt.cpu().numpy() - ref_nt).max() <= 1e-12 * np.abs(ref_nt).max()
        gT, gC = ag.adjoint_checkpointed(g, nt, every, ckpt, Cd, ag.residual(T_nt, Od), 1.0, dt,
                                         *dd)
        torch.cuda.synchronize()
        assert g.device_status() == 0
        gT, gC = gT.cpu().numpy(), gC.cpu().numpy()
    assert np.linalg.norm(gT - gT0) <= 1e-10 * np.linalg.norm(gT0)
    assert np.linalg.norm(gC - gCi) <= 1e-10 * np.linalg.norm(gCi)


def test_decomposed_fp32_gradient_vs_fp64_oracle():
    n, dims, periods, overlap = CASES[0]
    nt = 8
    T0, Ci, dd, dt = _fields(n, dims, periods, overlap)
    T_obs = oracle.run_decomposed(T0, Ci * 1.05, nt, 1.0, dt, *dd, dims, periods, overlap)
    _, gT0, gCi = oracle.gradient_decomposed(T0, Ci, T_obs, nt, 1.0, dt, *dd, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        T0d, Cd, Od = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (T0, Ci, T_obs))
        T_nt, ckpt = ag.forward_checkpointed(g, nt, 3, T0d, Cd, 1.0, dt, *dd)
        gT, gC = ag.adjoint_checkpointed(g, nt, 3, ckpt, Cd, ag.residual(T_nt, Od), 1.0, dt, *dd)
        gT, gC = gT.double().cpu().numpy(), gC.cpu().numpy()
    assert np.linalg.norm(gC - gCi) <= 1e-3 * np.linalg.norm(gCi)
    assert np.linalg.norm(gT - gT0) <= 1e-3 * np.linalg.norm(gT0)


def test_decomposed_autograd_finite_differences():
    """torch.autograd through the library on 2x2x2 subdomains (periodic in x),
    central differences of a misfit along random directions of Ci and T0."""
    n, dims, periods, overlap = (32, 18, 16), (2, 2, 2), (1, 0, 0), (2, 2, 2)
    nt = 12
    T0, Ci, dd, dt = _fields(n, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        Cs = torch.from_numpy(Ci * 1.05).cuda()
        T0d = torch.from_numpy(T0).cuda()
        T_obs = ag.solve(T0d, Cs, g, nt, 1.0, dt, *dd).detach()
        rng = np.random.default_rng(9)
        C = torch.from_numpy(Ci).cuda().requires_grad_(True)
        T = T0d.clone().requires_grad_(True)

        def J(Tin, Cin):
            return 0.5 * ((ag.solve(Tin, Cin, g, nt, 1.0, dt, *dd) - T_obs) ** 2).sum()

        J(T, C).backward()
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
