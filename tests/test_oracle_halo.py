"""Pins of the oracle's halo update and split (update_halo! and
@hide_communication, Sec. Approach and Fig. 1): a decomposed run with halo
updates is bit-identical to the undecomposed run, the boundary/inner split is
bit-identical to the plain step, and every halo point is written."""
import numpy as np
import pytest

import oracle
import synth


def make_case(n, dims, periods, overlap, seed=0, sigma=0.15):
    """Inputs of the decomposed grid [nsub][nz][ny][nx] and of the
    undecomposed array (extent n_g, or n_g + o when periodic), all drawn on
    global indices."""
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, overlap, periods)
    T = np.empty((nsub, n[2], n[1], n[0]))
    Ci = np.empty_like(T)
    for s in range(nsub):
        g = oracle.global_indices(n, dims, overlap, periods, s)
        T[s] = synth.gaussian_bump(*g, ng, sigma=sigma) + 0.05 * synth.uniform(seed, 5, synth.global_linear_index(*g, ng))
        Ci[s] = synth.ci_uniform_c0(seed, *g, ng)
    nu = tuple(ng[d] + (overlap[d] if periods[d] else 0) for d in range(3))
    gu = [np.arange(nu[d]) % ng[d] for d in range(3)]
    Tu = synth.gaussian_bump(*gu, ng, sigma=sigma) + 0.05 * synth.uniform(seed, 5, synth.global_linear_index(*gu, ng))
    Ciu = synth.ci_uniform_c0(seed, *gu, ng)
    dd = [oracle.spacing(1.0, ng[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ciu.max())
    return T, Ci, np.ascontiguousarray(Tu), np.ascontiguousarray(Ciu), dd, dt


def compare_to_undecomposed(Td, Tu, n, dims, overlap):
    nsub = Td.shape[0]
    for s in range(nsub):
        ix, iy, iz = oracle.undecomposed_index(n, dims, overlap, s)
        assert np.array_equal(Td[s], Tu[np.ix_(iz, iy, ix)]), f"subdomain {s} differs"


CASES = [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2)),
    ((8, 7, 6), (2, 2, 2), (1, 0, 0), (2, 2, 2)),
    ((9, 6, 11), (3, 1, 2), (0, 1, 1), (2, 2, 2)),
    ((13, 7, 9), (3, 1, 2), (1, 1, 1), (2, 3, 2)),
    ((10, 9, 8), (1, 1, 1), (1, 1, 1), (2, 2, 2)),
    ((7, 7, 7), (2, 1, 1), (1, 0, 1), (3, 2, 2)),
    ((6, 6, 6), (2, 2, 1), (1, 1, 0), (2, 2, 2)),
]


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
def test_decomposed_equals_undecomposed(n, dims, periods, overlap):
    T, Ci, Tu, Ciu, dd, dt = make_case(n, dims, periods, overlap)
    # identical inputs by construction
    compare_to_undecomposed(T, Tu, n, dims, overlap)
    nt = 6
    Td = oracle.run_decomposed(T, Ci, nt, 1.0, dt, *dd, dims, periods, overlap)
    Tr = oracle.run(Tu, Ciu, nt, 1.0, dt, *dd, periodic_self_halo=periods, overlap=overlap)
    compare_to_undecomposed(Td, Tr, n, dims, overlap)
    assert np.abs(Tr - Tu).max() > 1e-6  # the run did something


@pytest.mark.parametrize("widths", [(2, 2, 2), (16, 2, 2), (3, 4, 5)])
@pytest.mark.parametrize("n,dims,periods,overlap", CASES[:4])
def test_split_equals_unsplit(n, dims, periods, overlap, widths):
    widths = tuple(max(w, o) for w, o in zip(widths, overlap))
    T, Ci, _, _, dd, dt = make_case(n, dims, periods, overlap, seed=2)
    A = oracle.run_decomposed(T, Ci, 5, 1.0, dt, *dd, dims, periods, overlap)
    B = oracle.run_decomposed(T, Ci, 5, 1.0, dt, *dd, dims, periods, overlap, widths=widths)
    assert np.array_equal(A, B)


def test_split_sets_partition_inner_points():
    n = (20, 9, 8)
    T = np.random.default_rng(0).random((n[2], n[1], n[0]))
    Ci = np.ones_like(T)
    Ta = np.full_like(T, np.nan)
    Tb = np.full_like(T, np.nan)
    w = (3, 2, 2)
    oracle.step_part(Ta, T, Ci, 1.0, 1e-3, 1, 1, 1, w, 1)
    oracle.step_part(Tb, T, Ci, 1.0, 1e-3, 1, 1, 1, w, 0)
    a, b = ~np.isnan(Ta), ~np.isnan(Tb)
    assert not (a & b).any()
    inner = np.zeros_like(a)
    inner[1:-1, 1:-1, 1:-1] = True
    assert ((a | b) == inner).all()
    # inner block: 1-based indices w+1 .. n-w in every dimension
    assert b.sum() == (20 - 2 * 3) * (9 - 2 * 2) * (8 - 2 * 2)


@pytest.mark.parametrize("n,dims,periods,overlap", CASES)
def test_poisoned_halo_is_overwritten(n, dims, periods, overlap):
    """Fill every halo plane with NaN; after update_halo! none is left."""
    T, _, _, _, _, _ = make_case(n, dims, periods, overlap)
    left, right = oracle.neighbours(dims, periods)
    P = T.copy()
    for s in range(T.shape[0]):
        for d, sl0, sl1 in ((0, np.s_[:, :, 0], np.s_[:, :, -1]), (1, np.s_[:, 0, :], np.s_[:, -1, :]),
                            (2, np.s_[0, :, :], np.s_[-1, :, :])):
            if left[s, d] >= 0:
                P[s][sl0] = np.nan
            if right[s, d] >= 0:
                P[s][sl1] = np.nan
    oracle.update_halo(P, dims, periods, overlap)
    assert not np.isnan(P).any()
    # and the consistent field is a fixed point of the halo update
    Q = T.copy()
    oracle.update_halo(Q, dims, periods, overlap)
    assert np.array_equal(Q, T)
    assert np.array_equal(P, T)


def test_halo_bytes_generic():
    """The halo update is a bit copy: a uint16 field (BF16 storage) gets the
    same pattern of copies as a float64 field."""
    n, dims, periods, o = (8, 7, 6), (2, 2, 1), (1, 0, 0), (2, 2, 2)
    rng = np.random.default_rng(1)
    F = rng.integers(0, 65535, size=(4, n[2], n[1], n[0]), dtype=np.uint16)
    D = F.astype(np.float64)
    oracle.update_halo(F, dims, periods, o)
    oracle.update_halo(D, dims, periods, o)
    assert np.array_equal(F.astype(np.float64), D)


def test_planted_mistake_is_caught(monkeypatch):
    """A halo update that skips the z dimension must break decomposed ==
    undecomposed (the bit-exact check has teeth)."""
    n, dims, periods, o = (8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2)
    T, Ci, Tu, Ciu, dd, dt = make_case(n, dims, periods, o)
    real = oracle.neighbours

    def broken(dims_, periods_):
        left, right = real(dims_, periods_)
        left[:, 2] = -1
        right[:, 2] = -1
        return left, right

    monkeypatch.setattr(oracle, "neighbours", broken)
    Td = oracle.run_decomposed(T, Ci, 3, 1.0, dt, *dd, dims, periods, o)
    monkeypatch.undo()
    Tr = oracle.run(Tu, Ciu, 3, 1.0, dt, *dd)
    with pytest.raises(AssertionError):
        compare_to_undecomposed(Td, Tr, n, dims, o)


STAGGERED = [
    # n, dims, periods, overlap, delta (field size n + delta)
    ((8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2), (1, 0, 0)),
    ((8, 7, 6), (2, 2, 2), (1, 1, 0), (2, 2, 2), (1, 1, 1)),
    ((9, 8, 7), (3, 1, 2), (0, 1, 1), (3, 2, 3), (-1, 1, -1)),
    ((7, 7, 7), (2, 2, 1), (1, 0, 1), (2, 2, 2), (-1, 0, 1)),   # overlap 1 in x: no x exchange
    ((6, 6, 6), (1, 1, 1), (1, 1, 1), (2, 2, 2), (1, 1, 1)),    # its own neighbour
]


@pytest.mark.parametrize("n,dims,periods,overlap,delta", STAGGERED)
def test_staggered_halo_restores_global_field(n, dims, periods, overlap, delta):
    """A staggered field (local size n + delta, overlap o + delta) cut from one
    global field (extent dims*(n-o) + o + delta, or dims*(n-o) periodic) with
    every exchanged halo plane poisoned: after the halo update every point of
    every subdomain equals the global field at its global index."""
    nf = tuple(n[d] + delta[d] for d in range(3))
    of = oracle.staggered_overlap(n, nf, overlap)
    nsub = dims[0] * dims[1] * dims[2]
    ng = tuple(dims[d] * (n[d] - overlap[d]) + (0 if periods[d] else overlap[d] + delta[d])
               for d in range(3))
    G = synth.uniform(21, 3, np.arange(ng[0] * ng[1] * ng[2], dtype=np.uint64)).reshape(ng[2], ng[1], ng[0])
    left, right = oracle.neighbours(dims, periods)
    F = np.empty((nsub, nf[2], nf[1], nf[0]))
    idx = []
    for s in range(nsub):
        c = oracle.coords(s, dims)
        ii = [(c[d] * (n[d] - overlap[d]) + np.arange(nf[d])) % ng[d] for d in range(3)]
        idx.append(ii)
        F[s] = G[np.ix_(ii[2], ii[1], ii[0])]
        for d in range(3):
            if of[d] < 2:
                continue
            sl = [slice(None)] * 3
            if left[s][d] >= 0:
                sl[2 - d] = 0
                F[s][tuple(sl)] = np.nan
            if right[s][d] >= 0:
                sl[2 - d] = nf[d] - 1
                F[s][tuple(sl)] = np.nan
    oracle.update_halo_staggered(F, n, dims, periods, overlap)
    for s in range(nsub):
        ii = idx[s]
        assert np.array_equal(F[s], G[np.ix_(ii[2], ii[1], ii[0])]), f"subdomain {s}"


def test_staggered_overlap_rule():
    assert oracle.staggered_overlap((8, 7, 6), (9, 6, 6), (2, 2, 2)) == (3, 1, 2)
    with pytest.raises(ValueError):
        oracle.update_halo_staggered(np.zeros((1, 6, 6, 10)), (8, 6, 6), (1, 1, 1), (0, 0, 0), (2, 2, 2))
