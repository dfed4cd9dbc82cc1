"""Pins of the oracle's staggered-grid acoustic step (the multi-field
staggered stencil that uses update_halo! on fields of different sizes): a
closed-form standing wave in each dimension, conservation of the leapfrog
energy, and a decomposed run with staggered halo updates bit-identical to the
undecomposed run."""
import math

import numpy as np
import pytest

import oracle
import synth


def fields(n, P0=None):
    nx, ny, nz = n
    P = np.zeros((nz, ny, nx)) if P0 is None else np.ascontiguousarray(P0, dtype=np.float64)
    return P, np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_standing_wave_closed_form(d):
    """P0 = cos(pi m (i + 1/2) / n) along dimension d, V = 0: an eigenvector of
    -div grad with eigenvalue (4/h^2) sin^2(pi m/(2n)) under zero wall
    velocities. With s = c^2 dt^2 lambda / 2 and cos(theta) = 1 - s the
    leapfrog amplitude after k steps is cos(k theta) - s/sin(theta) sin(k theta)."""
    n = [3, 3, 3]
    n[d] = 24
    m, rho, K = 3, 1.3, 2.1
    h = [0.1, 0.07, 0.05]
    c2 = K / rho
    lam = 4.0 / h[d] ** 2 * math.sin(math.pi * m / (2 * n[d])) ** 2
    dt = 0.4 * h[d] / math.sqrt(c2)
    shape = (n[2], n[1], n[0])
    i = np.arange(n[d])
    prof = np.cos(math.pi * m * (i + 0.5) / n[d])
    P0 = np.broadcast_to(prof.reshape([-1 if k == 2 - d else 1 for k in range(3)]), shape)
    P, Vx, Vy, Vz = fields(n, P0)
    s = c2 * dt * dt * lam / 2.0
    th = math.acos(1.0 - s)
    for k in range(1, 61):
        oracle.acoustic_step(P, Vx, Vy, Vz, rho, K, dt, *h)
        amp = math.cos(k * th) - s / math.sin(th) * math.sin(k * th)
        assert np.abs(P - amp * P0).max() <= 1e-12 * k
    other = [v for q, v in enumerate((Vx, Vy, Vz)) if q != d]
    assert all(np.abs(v).max() == 0.0 for v in other)


def test_energy_conserved():
    n = (14, 12, 10)
    g = [np.arange(k) for k in n]
    P0 = np.broadcast_to(synth.gaussian_bump(*g, n, sigma=0.2), (n[2], n[1], n[0]))
    P, Vx, Vy, Vz = fields(n, P0 - 1.7)
    rho, K, h = 1.1, 2.5, (0.1, 0.12, 0.09)
    dt = 0.3 * min(h) / math.sqrt(K / rho)
    E = []
    for _ in range(150):
        Pp = P.copy()
        oracle.acoustic_step(P, Vx, Vy, Vz, rho, K, dt, *h)
        E.append(oracle.acoustic_energy(Pp, P, Vx, Vy, Vz, rho, K, *h))
    assert np.abs(np.array(E) - E[0]).max() <= 1e-12 * abs(E[0])


@pytest.mark.parametrize("n,dims,periods", [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0)),
    ((9, 6, 7), (3, 1, 2), (0, 0, 0)),
    ((7, 8, 6), (2, 2, 1), (0, 0, 0)),
])
def test_decomposed_equals_undecomposed(n, dims, periods):
    """Cells and faces of every subdomain equal the undecomposed run's at
    their global indices after nt steps with staggered halo updates."""
    o = (2, 2, 2)
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, o, periods)
    rho, K, h = 1.0, 1.7, (0.1, 0.1, 0.1)
    dt = 0.3 * 0.1 / math.sqrt(K / rho)
    lin = np.arange(ng[0] * ng[1] * ng[2], dtype=np.uint64)
    PG = (synth.uniform(8, 1, lin) - 0.5).reshape(ng[2], ng[1], ng[0])
    PGu, VxG, VyG, VzG = fields(ng, PG)
    P, Vx, Vy, Vz = (np.zeros((nsub,) + a.shape) for a in fields(n))
    idx = []
    for sub in range(nsub):
        c = oracle.coords(sub, dims)
        ii = [c[d] * (n[d] - o[d]) + np.arange(n[d] + 1) for d in range(3)]
        idx.append(ii)
        P[sub] = PG[np.ix_(ii[2][:-1], ii[1][:-1], ii[0][:-1])]
    nt = 9
    for _ in range(nt):
        oracle.acoustic_step(PGu, VxG, VyG, VzG, rho, K, dt, *h)
    oracle.acoustic_run_decomposed(P, Vx, Vy, Vz, nt, rho, K, dt, *h, n, dims, periods, o)
    for sub in range(nsub):
        ix, iy, iz = idx[sub]
        assert np.array_equal(P[sub], PGu[np.ix_(iz[:-1], iy[:-1], ix[:-1])])
        assert np.array_equal(Vx[sub], VxG[np.ix_(iz[:-1], iy[:-1], ix)])
        assert np.array_equal(Vy[sub], VyG[np.ix_(iz[:-1], iy, ix[:-1])])
        assert np.array_equal(Vz[sub], VzG[np.ix_(iz, iy[:-1], ix[:-1])])
