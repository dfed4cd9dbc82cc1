"""Pins of the oracle's adjoint on a grid of subdomains (the differentiated
form of Fig. 1's solver on the implicit global grid): one step is
T_{n+1} = H(S(T_n)), S the step on every subdomain and H the halo update, so
the adjoint step is S^T H^T. Checked against what fixes it independently:
dot-product identities of H and of the whole step, central finite
differences of the loss, and the single-array gradient when the grid has
one subdomain and no halo. A planted mistake in H^T (the halo entry not set
to 0 after it is added to its source) fails the identity."""
import numpy as np
import pytest

import oracle
import synth

TOPOLOGIES = [
    ((9, 8, 7), (2, 2, 2), (1, 0, 0), (2, 2, 2)),
    ((8, 9, 7), (3, 1, 2), (0, 1, 1), (2, 2, 2)),
    ((9, 7, 8), (1, 1, 1), (1, 1, 1), (2, 2, 2)),   # periodic self-neighbours
    ((10, 9, 8), (2, 2, 1), (0, 0, 0), (3, 2, 2)),  # overlap 3
]


def _fields(n, dims, periods, overlap, seed=4):
    left, _ = oracle.neighbours(dims, periods)
    nsub = left.shape[0]
    ng = oracle.global_size(n, dims, overlap, periods)
    T0 = np.empty((nsub, n[2], n[1], n[0]))
    Ci = np.empty_like(T0)
    for s in range(nsub):
        g = oracle.global_indices(n, dims, overlap, periods, s)
        T0[s] = synth.gaussian_bump(*g, ng, sigma=0.2) + 0.1 * synth.uniform(
            seed, 1, synth.global_linear_index(*g, ng))
        Ci[s] = synth.ci_uniform_c0(seed, *g, ng)
    dd = [oracle.spacing(1.0, ng[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    return np.ascontiguousarray(T0), np.ascontiguousarray(Ci), dd, dt


def _dot(a, b):
    return oracle.fsum(a * b)


def _halo_adjoint_without_zeroing(lam, dims, periods, overlap):
    """The planted mistake: H^T that adds each halo entry into its source but
    leaves the halo entry in place."""
    nsub, nz, ny, nx = lam.shape
    n = (nx, ny, nz)
    left, right = oracle.neighbours(dims, periods)
    for d in (2, 1, 0):
        o = overlap[d]
        if o < 2 or n[d] < 2:
            continue
        for s in range(nsub):
            for side, nb in ((0, left[s, d]), (1, right[s, d])):
                if nb < 0:
                    continue
                dst = 0 if side == 0 else n[d] - 1
                src = n[d] - o if side == 0 else o - 1
                ix = [slice(None)] * 3
                ix[2 - d] = dst
                jx = [slice(None)] * 3
                jx[2 - d] = src
                lam[nb][tuple(jx)] += lam[s][tuple(ix)]


@pytest.mark.parametrize("n,dims,periods,overlap", TOPOLOGIES)
def test_halo_adjoint_dot_product(n, dims, periods, overlap):
    """<H x, y> = <x, H^T y> for random x, y over every entry."""
    nsub = int(np.prod(dims))
    rng = np.random.default_rng(1)
    x = rng.standard_normal((nsub, n[2], n[1], n[0]))
    y = rng.standard_normal(x.shape)
    Hx = x.copy()
    oracle.update_halo(Hx, dims, periods, overlap)
    HTy = y.copy()
    oracle.update_halo_adjoint(HTy, dims, periods, overlap)
    lhs, rhs = _dot(Hx, y), _dot(x, HTy)
    assert abs(lhs - rhs) <= 1e-13 * oracle.fsum(np.abs(Hx * y))
    # the planted mistake fails it
    bad = y.copy()
    _halo_adjoint_without_zeroing(bad, dims, periods, overlap)
    assert abs(lhs - _dot(x, bad)) > 1e-6 * oracle.fsum(np.abs(Hx * y))


@pytest.mark.parametrize("n,dims,periods,overlap", TOPOLOGIES)
def test_decomposed_step_dot_product(n, dims, periods, overlap):
    """<A x, y> = <x, A^T y> with A = H S the decomposed step (linear in T)
    and A^T = S^T H^T."""
    _, Ci, dd, dt = _fields(n, dims, periods, overlap)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(Ci.shape)
    y = rng.standard_normal(Ci.shape)
    Ax = x.copy()
    for s in range(x.shape[0]):
        oracle.step(Ax[s], x[s], Ci[s], 1.0, dt, *dd)
    oracle.update_halo(Ax, dims, periods, overlap)
    yy = y.copy()
    oracle.update_halo_adjoint(yy, dims, periods, overlap)
    ATy = np.empty_like(y)
    gCi = np.zeros_like(y)
    for s in range(y.shape[0]):
        oracle.adjoint_step(ATy[s], yy[s], x[s], Ci[s], gCi[s], 1.0, dt, *dd)
    lhs, rhs = _dot(Ax, y), _dot(x, ATy)
    assert abs(lhs - rhs) <= 1e-13 * oracle.fsum(np.abs(Ax * y))


@pytest.mark.parametrize("n,dims,periods,overlap", TOPOLOGIES[:2] + TOPOLOGIES[3:])
def test_decomposed_gradient_finite_differences(n, dims, periods, overlap):
    """Central differences of J(T0, Ci) = 0.5 sum((T_nt - T_obs)^2) over the
    decomposed run, along random directions of Ci and of T0."""
    T0, Ci, dd, dt = _fields(n, dims, periods, overlap)
    nt = 6
    rng = np.random.default_rng(3)
    T_obs = oracle.run_decomposed(T0, Ci * 1.05, nt, 1.0, dt, *dd, dims, periods, overlap)
    J, gT, gC = oracle.gradient_decomposed(T0, Ci, T_obs, nt, 1.0, dt, *dd, dims, periods, overlap)

    def Jof(T, C):
        return oracle.loss(oracle.run_decomposed(T, C, nt, 1.0, dt, *dd, dims, periods, overlap), T_obs)

    assert J == Jof(T0, Ci)
    for which in ("Ci", "T0"):
        v = rng.standard_normal(Ci.shape)
        h = 1e-6 * (np.linalg.norm(Ci if which == "Ci" else T0) / np.linalg.norm(v))
        if which == "Ci":
            fd = (Jof(T0, Ci + h * v) - Jof(T0, Ci - h * v)) / (2 * h)
            ad = _dot(gC, v)
        else:
            fd = (Jof(T0 + h * v, Ci) - Jof(T0 - h * v, Ci)) / (2 * h)
            ad = _dot(gT, v)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (which, fd, ad)


def test_single_subdomain_equals_single_array_gradient():
    """One subdomain without neighbours: H is the identity and the gradient is
    the single-array one, bit for bit."""
    n = (11, 9, 8)
    T0, Ci, dd, dt = _fields(n, (1, 1, 1), (0, 0, 0), (2, 2, 2))
    T_obs = oracle.run(T0[0], Ci[0] * 1.05, 5, 1.0, dt, *dd)
    J1, gT1, gC1 = oracle.gradient(T0[0], Ci[0], T_obs, 5, 1.0, dt, *dd)
    J2, gT2, gC2 = oracle.gradient_decomposed(T0, Ci, T_obs[None], 5, 1.0, dt, *dd, (1, 1, 1),
                                              (0, 0, 0), (2, 2, 2))
    assert J1 == J2
    assert np.array_equal(gT1, gT2[0]) and np.array_equal(gC1, gC2[0])
