"""Pins of the oracle on 2-D and 1-D grids (a dimension of size 1 is absent:
no neighbours, no second difference, no halo, infinite spacing): closed-form
mode decay, the 3-D step reduced exactly, decomposed == undecomposed and
split == unsplit bit for bit."""
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_halo import make_case, compare_to_undecomposed


@pytest.mark.parametrize("n,m", [((17, 13, 1), (2, 3, 0)), ((23, 1, 1), (3, 0, 0)), ((19, 1, 1), (5, 0, 0))])
def test_mode_decay_low_dimensional(n, m):
    """A product of sines over the present dimensions vanishing on their
    boundaries decays by g = 1 - dt*lam*c*sum_d 4/dd^2 sin^2(pi m_d dd/2),
    the sum over the present dimensions only."""
    act = [d for d in range(3) if n[d] > 1]
    dd = [oracle.spacing(1.0, n[d]) for d in range(3)]
    assert all(math.isinf(dd[d]) for d in range(3) if n[d] == 1)
    lam, c, nt, A, base = 1.1, 0.6, 40, 0.25, 1.7
    dt = oracle.cfl_dt(*dd, lam, c)
    prof = np.ones((n[2], n[1], n[0]))
    for d in act:
        x = np.arange(n[d]) * dd[d]
        shp = [1, 1, 1]
        shp[2 - d] = n[d]
        prof = prof * np.sin(np.pi * m[d] * x).reshape(shp)
    T0 = base + A * prof
    T = oracle.run(T0, np.full(T0.shape, c), nt, lam, dt, *dd)
    g = 1 - dt * lam * c * sum(4 / dd[d] ** 2 * math.sin(math.pi * m[d] * dd[d] / 2) ** 2 for d in act)
    inner = tuple(slice(1, -1) if n[d] > 1 else slice(None) for d in (2, 1, 0))
    assert np.abs(T[inner] - (base + A * g ** nt * prof)[inner]).max() <= 1e-13 * nt
    assert abs(A * (1 - g ** nt)) > 1e-3


def test_two_d_is_the_three_d_step_on_a_z_invariant_field():
    """A 2-D grid gives, bit for bit, the middle plane of a 3-D run whose
    field does not change along z (its z differences are exactly 0 too) with
    an infinite dz."""
    n2 = (15, 12, 1)
    g = [np.arange(k) for k in n2]
    P = synth.gaussian_bump(*g, n2, sigma=0.2)
    T2d = np.ascontiguousarray(np.broadcast_to(P, (1, 12, 15)))
    C2d = np.ascontiguousarray(np.broadcast_to(synth.ci_uniform_c0(3, *g, n2), (1, 12, 15)))
    T3d = np.ascontiguousarray(np.broadcast_to(T2d, (3, 12, 15)))
    C3d = np.ascontiguousarray(np.broadcast_to(C2d, (3, 12, 15)))
    dd = (0.07, 0.09, math.inf)
    dt = oracle.cfl_dt(*dd, 1.0, C2d.max())
    a = oracle.run(T2d, C2d, 7, 1.0, dt, *dd)
    b = oracle.run(T3d, C3d, 7, 1.0, dt, *dd)
    assert np.array_equal(a[0], b[1])


@pytest.mark.parametrize("n,dims,periods,overlap", [
    ((8, 7, 1), (2, 2, 1), (0, 0, 0), (2, 2, 2)),
    ((9, 6, 1), (3, 1, 1), (1, 0, 0), (2, 2, 2)),
    ((10, 1, 1), (3, 1, 1), (0, 0, 0), (2, 2, 2)),
    ((7, 1, 1), (2, 1, 1), (1, 0, 0), (3, 2, 2)),
])
def test_low_dimensional_decomposed_equals_undecomposed(n, dims, periods, overlap):
    T, Ci, Tu, Ciu, dd, dt = make_case(n, dims, periods, overlap, seed=2)
    nt = 6
    Td = oracle.run_decomposed(T, Ci, nt, 1.0, dt, *dd, dims, periods, overlap)
    Ts = oracle.run_decomposed(T, Ci, nt, 1.0, dt, *dd, dims, periods, overlap,
                               widths=tuple(max(2, o) for o in overlap))
    assert np.array_equal(Td, Ts)
    Tr = oracle.run(Tu, Ciu, nt, 1.0, dt, *dd,
                    periodic_self_halo=periods if any(periods) else None, overlap=overlap)
    compare_to_undecomposed(Td, Tr, n, dims, overlap)


def test_absent_dimension_rules():
    with pytest.raises(ValueError):
        oracle.global_size((8, 8, 1), (1, 1, 2), (2, 2, 2), (0, 0, 0))
    with pytest.raises(ValueError):
        oracle.global_size((8, 8, 1), (1, 1, 1), (2, 2, 2), (0, 0, 1))
    assert oracle.global_size((8, 7, 1), (2, 2, 1), (2, 2, 2), (0, 0, 0)) == (14, 12, 1)
