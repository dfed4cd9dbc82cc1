"""Pins of the oracle's step (Fig. 1 step!) against what the mathematics
fixes: a hand-computed golden case, the discrete Fourier-mode decay factor,
stationarity, conservation with periodic boundaries, mirror symmetry, and an
independent Kronecker-sum sparse Laplacian."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if line:
            vals[line[0]] = float(line[1])
    return vals


def test_golden_3x3x3_hand_computed():
    g = _golden("step_3x3x3.txt")
    T = np.full((3, 3, 3), g["other"])
    T[1, 1, 1] = g["centre"]
    T[1, 1, 0], T[1, 1, 2] = g["xm"], g["xp"]
    T[1, 0, 1], T[1, 2, 1] = g["ym"], g["yp"]
    T[0, 1, 1], T[2, 1, 1] = g["zm"], g["zp"]
    Ci = np.full((3, 3, 3), 99.0)
    Ci[1, 1, 1] = g["ci"]
    T2 = T.copy()
    oracle.step(T2, T, Ci, g["lam"], g["dt"], g["dx"], g["dy"], g["dz"])
    assert T2[1, 1, 1] == g["expected"]
    mask = np.ones_like(T, dtype=bool)
    mask[1, 1, 1] = False
    assert (T2[mask] == T[mask]).all()


def _sine_field(n, m, base, amp, periodic=False):
    """base + amp * prod_d sin(pi m_d x_d), x_d = i*dd, dd = 1/(n_d - 1)."""
    ax = [np.sin(np.pi * m[d] * np.arange(n[d]) / (n[d] - 1)) for d in range(3)]
    return base + amp * (ax[2][:, None, None] * ax[1][None, :, None] * ax[0][None, None, :])


@pytest.mark.parametrize("m", [(1, 1, 1), (2, 3, 1), (5, 1, 4)])
def test_fourier_mode_decay_dirichlet(m):
    """A product of sines vanishing on the boundary is a discrete eigenvector
    of the 7-point operator: one step multiplies its amplitude by
    g = 1 - dt*lam*c*sum_d 4/dd^2 sin^2(pi m_d dd/2) (constant Ci = c)."""
    n = (17, 13, 11)  # distinct sizes and spacings catch transposed axes
    dd = [1.0 / (n[d] - 1) for d in range(3)]
    lam, c, nt, A, base = 1.3, 0.55, 40, 0.25, 1.7
    dt = oracle.cfl_dt(dd[0], dd[1], dd[2], lam, c)
    T0 = _sine_field(n, m, base, A)
    Ci = np.full(T0.shape, c)
    T = oracle.run(T0, Ci, nt, lam, dt, *dd)
    g = 1 - dt * lam * c * sum(4 / dd[d] ** 2 * np.sin(np.pi * m[d] * dd[d] / 2) ** 2 for d in range(3))
    expected = base + A * g ** nt * (T0 - base) / A
    inner = (slice(1, -1),) * 3
    err = np.abs(T[inner] - expected[inner]).max()
    assert err <= 1e-13 * nt
    # the decay is real: the amplitude changed by far more than the tolerance
    assert abs(A * (1 - g ** nt)) > 1e-3


@pytest.mark.parametrize("m", [(1, 2, 3), (4, 1, 2)])
def test_fourier_mode_decay_periodic(m):
    """Periodic grid (one subdomain, self halo): cos(2 pi m i / n_g) decays by
    g = 1 - dt*lam*c*sum_d 4/dd^2 sin^2(pi m_d / n_g,d) per step."""
    n_g = (12, 10, 14)
    o = (2, 2, 2)
    n = tuple(n_g[d] + o[d] for d in range(3))
    dd = [oracle.spacing(1.0, n_g[d]) for d in range(3)]
    lam, c, nt, A, base = 0.9, 0.6, 30, 0.3, 1.7
    dt = oracle.cfl_dt(dd[0], dd[1], dd[2], lam, c)
    idx = [np.arange(n[d]) % n_g[d] for d in range(3)]
    ax = [np.cos(2 * np.pi * m[d] * idx[d] / n_g[d]) for d in range(3)]
    mode = ax[2][:, None, None] * ax[1][None, :, None] * ax[0][None, None, :]
    T0 = base + A * mode
    Ci = np.full(T0.shape, c)
    T = oracle.run(T0, Ci, nt, lam, dt, *dd, periodic_self_halo=(1, 1, 1), overlap=o)
    g = 1 - dt * lam * c * sum(4 / dd[d] ** 2 * np.sin(np.pi * m[d] / n_g[d]) ** 2 for d in range(3))
    expected = base + A * g ** nt * mode
    assert np.abs(T - expected).max() <= 1e-13 * nt
    assert abs(A * (1 - g ** nt)) > 1e-3


def test_stationarity_bit_exact():
    n = (9, 8, 7)
    gx, gy, gz = (np.arange(k) for k in n)
    Ci = synth.ci_uniform_c0(5, gx, gy, gz, n)
    T = np.full(Ci.shape, 1.7)
    T2 = np.full(Ci.shape, -1.0)
    oracle.step(T2, T, np.ascontiguousarray(Ci), 1.0, 1e-3, 0.1, 0.2, 0.3)
    assert (T2[1:-1, 1:-1, 1:-1] == 1.7).all()


def test_conservation_periodic():
    """All dims periodic: sum over unique points of T/Ci is conserved, since
    (T2 - T)/Ci = dt*lam*(discrete Laplacian), whose periodic sum telescopes."""
    n_g = (10, 12, 9)
    o = (2, 2, 2)
    n = tuple(n_g[d] + o[d] for d in range(3))
    idx = [np.arange(n[d]) % n_g[d] for d in range(3)]
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(3, *idx, n_g))
    T0 = synth.gaussian_bump(*idx, n_g, sigma=0.2)
    dd = [oracle.spacing(1.0, n_g[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    T = oracle.run(T0, Ci, 100, 1.0, dt, *dd, periodic_self_halo=(1, 1, 1), overlap=o)
    u = (slice(0, n_g[2]), slice(0, n_g[1]), slice(0, n_g[0]))
    H0 = oracle.fsum(T0[u] / Ci[u])
    H1 = oracle.fsum(T[u] / Ci[u])
    assert abs(H1 - H0) / H0 <= 1e-12
    # and the field did change
    assert np.abs(T - T0).max() > 1e-2


def test_mirror_symmetry_bit_exact():
    n = (11, 9, 8)
    g = [np.arange(k) for k in n]
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(9, *g, n))
    T0 = np.ascontiguousarray(synth.gaussian_bump(*g, n, sigma=0.15)
                              + 0.1 * synth.uniform(9, 3, synth.global_linear_index(*g, n)))
    dd = (0.1, 0.12, 0.09)
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    A = oracle.run(T0, Ci, 7, 1.0, dt, *dd)
    B = oracle.run(np.ascontiguousarray(T0[:, :, ::-1]), np.ascontiguousarray(Ci[:, :, ::-1]), 7, 1.0, dt, *dd)
    assert (A[:, :, ::-1] == B).all()


def _kron_laplacian(n, dd):
    def d2(k, h):
        return sp.diags([np.ones(k - 1), -2 * np.ones(k), np.ones(k - 1)], [-1, 0, 1]) / (h * h)
    I = [sp.identity(n[d]) for d in range(3)]
    Lx, Ly, Lz = d2(n[0], dd[0]), d2(n[1], dd[1]), d2(n[2], dd[2])
    # flattened order z, y, x (x fastest)
    return (sp.kron(I[2], sp.kron(I[1], Lx)) + sp.kron(I[2], sp.kron(Ly, I[0]))
            + sp.kron(Lz, sp.kron(I[1], I[0]))).tocsr()


def test_kronecker_sum_laplacian():
    """An independent formulation: T2 = T + dt*lam*Ci*(L T) on inner points,
    L the Kronecker sum of 1-D second-difference matrices."""
    n = (7, 9, 11)
    dd = (0.11, 0.07, 0.05)
    g = [np.arange(k) for k in n]
    T = np.ascontiguousarray(1 + synth.uniform(1, 0, synth.global_linear_index(*g, n)))  # rough field
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(1, *g, n))
    lam, dt = 1.7, 1e-4
    T2 = T.copy()
    oracle.step(T2, T, Ci, lam, dt, *dd)
    L = _kron_laplacian(n, dd)
    ref = (T.ravel() + dt * lam * Ci.ravel() * (L @ T.ravel())).reshape(T.shape)
    inner = (slice(1, -1),) * 3
    scale = np.abs(dt * lam * Ci * (L @ T.ravel()).reshape(T.shape))[inner].max()
    assert np.abs(T2[inner] - ref[inner]).max() <= 1e-13 * max(scale, 1.0)
    # the update is not trivially small
    assert scale > 1e-3
