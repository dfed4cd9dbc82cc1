"""Pins of the oracle's Gross-Pitaevskii solver (complex field psi = u + i v,
u at whole and v at half time steps): a closed-form linear standing mode,
exact conservation of ||u^n||^2 + <v^{n+1/2}, v^{n-1/2}> in the linear case,
the nonlinear phase rotation of a uniform field, and decomposed ==
undecomposed bit for bit."""
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_halo import compare_to_undecomposed


def sine_mode(n, m, dd):
    out = np.ones((n[2], n[1], n[0]))
    for d in range(3):
        x = np.arange(n[d]) * dd[d]
        shp = [1, 1, 1]
        shp[2 - d] = n[d]
        out = out * np.sin(np.pi * m[d] * x).reshape(shp)
    return out


@pytest.mark.parametrize("m", [(1, 1, 1), (2, 3, 1)])
def test_linear_mode_closed_form(m):
    """g = 0, V = V0: a Dirichlet sine mode is an eigenvector of H with
    omega = mu/2 + V0, mu = sum_d 4/dd^2 sin^2(pi m_d dd/2). From u^0 = A mode,
    v^{1/2} = 0, the staggered steps give u^k = A (cos k theta +
    (1 - cos theta)/sin theta sin k theta) mode, cos theta = 1 - (dt omega)^2/2."""
    n = (17, 13, 11)
    dd = [1.0 / (n[d] - 1) for d in range(3)]
    V0, A = 0.7, 0.4
    mu = sum(4 / dd[d] ** 2 * math.sin(math.pi * m[d] * dd[d] / 2) ** 2 for d in range(3))
    om = 0.5 * mu + V0
    # stable for every mode: dt below 2 / (largest eigenvalue of H)
    dt = 0.5 / (0.5 * sum(4 / h ** 2 for h in dd) + V0)
    mode = sine_mode(n, m, dd)
    u = np.ascontiguousarray(A * mode)
    v = np.zeros_like(u)
    V = np.full(u.shape, V0)
    th = math.acos(1 - (dt * om) ** 2 / 2)
    for k in range(1, 401):
        oracle.gp_run(u, v, V, 1, 0.0, dt, *dd)
        amp = A * (math.cos(k * th) + (1 - math.cos(th)) / math.sin(th) * math.sin(k * th))
        assert np.abs(u - amp * mode).max() <= 1e-13 * k
    assert 400 * th > 2.0  # the mode went through a large part of a period


def test_linear_invariant_conserved():
    n = (14, 12, 10)
    dd = [0.1, 0.12, 0.09]
    g = [np.arange(k) for k in n]
    r2 = sum(((np.arange(n[d]) - (n[d] - 1) / 2) * dd[d]).reshape([-1 if k == 2 - d else 1 for k in range(3)]) ** 2
             for d in range(3))
    V = np.ascontiguousarray(np.broadcast_to(2.0 * r2, (n[2], n[1], n[0])))
    bump = np.broadcast_to(synth.gaussian_bump(*g, n, sigma=0.2) - 1.7, (n[2], n[1], n[0]))
    inner = np.zeros((n[2], n[1], n[0]))
    inner[1:-1, 1:-1, 1:-1] = 1.0
    u = np.ascontiguousarray(bump * inner)
    v = np.ascontiguousarray(0.3 * bump * inner * np.cos(np.arange(n[0]) * 0.7))
    dt = 0.2 / (0.5 * sum(4 / h ** 2 for h in dd) + V.max())
    C = []
    for _ in range(120):
        oracle.gp_half(0, u, v, V, 0.0, dt, *dd)
        vp = v.copy()
        oracle.gp_half(1, u, v, V, 0.0, dt, *dd)
        C.append(oracle.gp_invariant(u, vp, v))
    assert np.abs(np.array(C[1:]) - C[0]).max() <= 1e-12 * C[0]


def test_uniform_field_rotates_at_g_rho():
    """A uniform field on a periodic grid (zero Laplacian) rotates in the
    complex plane at the frequency g*rho: u^n ~ sqrt(rho) cos(g rho n dt)."""
    n, dims, per, o = (6, 6, 6), (1, 1, 1), (1, 1, 1), (2, 2, 2)
    rho, gg, dt, nt = 0.8, 1.5, 0.005, 200
    u = np.full((1, n[2], n[1], n[0]), math.sqrt(rho))
    v = np.zeros_like(u)
    V = np.zeros_like(u)
    oracle.gp_run_decomposed(u, v, V, nt, gg, dt, 0.1, 0.1, 0.1, dims, per, o)
    assert np.ptp(u) == 0.0 and np.ptp(v) == 0.0
    # continuous solution sqrt(rho) exp(-i g rho t); the staggered start
    # (v^{1/2} = 0) offsets the phase by O(g rho dt), far below the O(0.3)
    # that a wrong density (u^2 - v^2) or a flipped g would give here
    t = nt * dt
    assert abs(u.flat[0] - math.sqrt(rho) * math.cos(gg * rho * t)) <= 1e-2
    assert abs(v.flat[0] + math.sqrt(rho) * math.sin(gg * rho * t)) <= 1e-2
    assert abs(u.flat[0] ** 2 + v.flat[0] ** 2 - rho) <= 1e-2


@pytest.mark.parametrize("n,dims,periods", [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0)),
    ((9, 6, 7), (3, 1, 2), (1, 0, 1)),
    ((7, 7, 7), (2, 2, 1), (1, 1, 1)),
])
def test_decomposed_equals_undecomposed(n, dims, periods):
    o = (2, 2, 2)
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, o, periods)
    lin = np.arange(ng[0] * ng[1] * ng[2], dtype=np.uint64)
    UG = (synth.uniform(11, 1, lin) - 0.5).reshape(ng[2], ng[1], ng[0])
    VG = (synth.uniform(11, 2, lin) - 0.5).reshape(ng[2], ng[1], ng[0])
    PotG = synth.uniform(11, 3, lin).reshape(ng[2], ng[1], ng[0])
    nu = tuple(ng[d] + (o[d] if periods[d] else 0) for d in range(3))
    gu = [np.arange(nu[d]) % ng[d] for d in range(3)]
    u1, v1, P1 = (np.ascontiguousarray(A[np.ix_(gu[2], gu[1], gu[0])]) for A in (UG, VG, PotG))
    U, Vv, Pot = (np.empty((nsub, n[2], n[1], n[0])) for _ in range(3))
    for s in range(nsub):
        gi = oracle.global_indices(n, dims, o, periods, s)
        for A, B in ((U, UG), (Vv, VG), (Pot, PotG)):
            A[s] = B[np.ix_(gi[2], gi[1], gi[0])]
    g, dt, dd = 0.9, 2e-3, (0.1, 0.1, 0.1)
    nt = 6
    oracle.gp_run_decomposed(U, Vv, Pot, nt, g, dt, *dd, dims, periods, o)
    one = (1, 1, 1)
    uu, vv, pp = u1[None].copy(), v1[None].copy(), P1[None].copy()
    oracle.gp_run_decomposed(uu, vv, pp, nt, g, dt, *dd, one, periods, o)
    compare_to_undecomposed(U, uu[0], n, dims, o)
    compare_to_undecomposed(Vv, vv[0], n, dims, o)
