"""Pins of the oracle's implicit-global-grid bookkeeping (Sec. Approach;
Fig. 1 init_global_grid and nx_g()/ny_g()/nz_g())."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dims_cases():
    out = []
    for line in open(os.path.join(GOLDEN, "mpi_dims_create.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        nn, din = int(line[0]), tuple(int(v) for v in line[1:4])
        exp = None if line[4] == "error" else tuple(int(v) for v in line[4:7])
        out.append((nn, din, exp))
    return out


@pytest.mark.parametrize("nn,din,exp", _dims_cases())
def test_dims_create_mpi_standard_examples(nn, din, exp):
    if exp is None:
        with pytest.raises(ValueError):
            oracle.dims_create(nn, din)
    else:
        assert oracle.dims_create(nn, din) == exp


@pytest.mark.parametrize("nsub", [1, 2, 3, 4, 6, 8, 12, 16, 27, 30, 64, 97])
def test_dims_create_properties(nsub):
    d = oracle.dims_create(nsub)
    assert d[0] * d[1] * d[2] == nsub
    assert d[0] >= d[1] >= d[2] >= 1
    # no other non-increasing factorisation has a smaller largest factor
    best = min(max(a, b, nsub // (a * b)) for a in range(1, nsub + 1) for b in range(1, nsub + 1)
               if nsub % (a * b) == 0)
    assert max(d) == best


def test_dims_create_cubes():
    for p in (2, 3, 4, 5):
        assert oracle.dims_create(p ** 3) == (p, p, p)


@pytest.mark.parametrize("dims,periods", [((2, 2, 2), (1, 0, 0)), ((3, 1, 2), (0, 1, 1)),
                                          ((1, 1, 1), (1, 1, 1)), ((4, 2, 1), (0, 0, 0))])
def test_global_indices_cover_global_grid(dims, periods):
    """Union of every subdomain's global indices is exactly range(n_g) per
    axis, consecutive subdomains share exactly `overlap` planes."""
    n, o = (9, 7, 8), (2, 3, 2)
    ng = oracle.global_size(n, dims, o, periods)
    nsub = dims[0] * dims[1] * dims[2]
    for d in range(3):
        seen = set()
        for s in range(nsub):
            seen.update(oracle.global_indices(n, dims, o, periods, s)[d].tolist())
        assert seen == set(range(ng[d]))
    # overlap: the last o planes of coord c are the first o planes of coord c+1
    for d in range(3):
        for s in range(nsub):
            c = oracle.coords(s, dims)
            if c[d] + 1 < dims[d]:
                cc = list(c)
                cc[d] += 1
                t = oracle.sub_index(cc, dims)
                a = oracle.global_indices(n, dims, o, periods, s)[d]
                b = oracle.global_indices(n, dims, o, periods, t)[d]
                assert list(a[n[d] - o[d]:]) == list(b[:o[d]])


def test_global_size_single_subdomain():
    assert oracle.global_size((10, 11, 12), (1, 1, 1), (2, 2, 2), (0, 0, 0)) == (10, 11, 12)
    assert oracle.global_size((10, 11, 12), (1, 1, 1), (2, 2, 2), (1, 1, 1)) == (8, 9, 10)
    # the large decomposed workload: 2x2x2 of 512x256x256, overlap 2, periodic in x
    assert oracle.global_size((512, 256, 256), (2, 2, 2), (2, 2, 2), (1, 0, 0)) == (1020, 510, 510)


def test_neighbours():
    left, right = oracle.neighbours((2, 1, 1), (1, 0, 0))
    assert left[0, 0] == 1 and right[0, 0] == 1 and left[1, 0] == 0 and right[1, 0] == 0
    assert (left[:, 1:] == -1).all() and (right[:, 1:] == -1).all()
    left, right = oracle.neighbours((3, 1, 1), (0, 0, 0))
    assert left[0, 0] == -1 and right[0, 0] == 1 and right[2, 0] == -1 and left[2, 0] == 1
    left, right = oracle.neighbours((1, 1, 1), (1, 1, 1))
    assert (left == 0).all() and (right == 0).all()


def test_coords_roundtrip():
    dims = (3, 4, 5)
    for s in range(60):
        assert oracle.sub_index(oracle.coords(s, dims), dims) == s
    assert oracle.coords(1, dims) == (1, 0, 0)  # x fastest


def test_cfl_dt_properties():
    dt = oracle.cfl_dt(0.1, 0.2, 0.05, 1.0, 0.5)
    assert dt == pytest.approx(0.05 ** 2 / 0.5 / 6.1, rel=1e-15)
    assert oracle.cfl_dt(0.1, 0.1, 0.1, 2.0, 0.5) == pytest.approx(0.5 * oracle.cfl_dt(0.1, 0.1, 0.1, 1.0, 0.5), rel=1e-15)
    # stability: the largest discrete eigenvalue gives |g| <= 1
    dx, dy, dz, lam, c = 0.1, 0.07, 0.13, 1.3, 0.61
    dt = oracle.cfl_dt(dx, dy, dz, lam, c)
    g_min = 1 - dt * lam * c * sum(4 / h ** 2 for h in (dx, dy, dz))
    assert -1 <= g_min <= 1
