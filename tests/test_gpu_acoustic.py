"""GPU parity of the staggered-grid acoustic step (igg_acoustic_step: cell
and face fields of different sizes, halo update of all four in one launch
per dimension) against the oracle's decomposed run, and conservation of the
leapfrog energy on the GPU."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def decomposed_inputs(n, dims, periods, o, seed):
    """P cut from one global random field (cell indices), V = 0."""
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, o, periods)
    lin = np.arange(ng[0] * ng[1] * ng[2], dtype=np.uint64)
    PG = (synth.uniform(seed, 1, lin) - 0.5).reshape(ng[2], ng[1], ng[0])
    P = np.zeros((nsub, n[2], n[1], n[0]))
    for s in range(nsub):
        c = oracle.coords(s, dims)
        ii = [(c[d] * (n[d] - o[d]) + np.arange(n[d])) % ng[d] for d in range(3)]
        P[s] = PG[np.ix_(ii[2], ii[1], ii[0])]
    Vx = np.zeros((nsub, n[2], n[1], n[0] + 1))
    Vy = np.zeros((nsub, n[2], n[1] + 1, n[0]))
    Vz = np.zeros((nsub, n[2] + 1, n[1], n[0]))
    return P, Vx, Vy, Vz


CASES = [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0)),
    ((9, 6, 7), (3, 1, 2), (0, 0, 0)),
    ((40, 20, 18), (2, 2, 1), (1, 0, 1)),
    ((33, 17, 9), (1, 2, 2), (1, 1, 1)),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,dims,periods", CASES)
def test_acoustic_matches_oracle(n, dims, periods, dtype):
    o = (2, 2, 2)
    rho, K, h = 1.2, 2.3, (0.1, 0.08, 0.12)
    dt = 0.3 * min(h) / math.sqrt(K / rho)
    nt = 9
    host = decomposed_inputs(n, dims, periods, o, 3)
    ref = [a.copy() for a in host]
    oracle.acoustic_run_decomposed(*ref, nt, rho, K, dt, *h, n, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        dev = [torch.from_numpy(a).to(dtype).cuda() for a in host]
        for _ in range(nt):
            g.acoustic_step(*dev, rho, K, dt, *h)
        torch.cuda.synchronize()
        got = [d.double().cpu().numpy() for d in dev]
    tol = 1e-12 if dtype == torch.float64 else 2e-6 * nt
    for name, a, r in zip(("P", "Vx", "Vy", "Vz"), got, ref):
        scale = max(np.abs(r).max(), 1e-300)
        assert np.abs(a - r).max() <= tol * scale, (name, np.abs(a - r).max() / scale)


@pytest.mark.parametrize("n,dims,periods,o", [
    ((20, 9, 8), (2, 1, 2), (1, 0, 0), (3, 2, 2)),   # overlap 3 in x, periodic ring of two
    ((21, 8, 9), (3, 2, 1), (0, 1, 0), (3, 2, 2)),   # a middle subdomain with both x neighbours
    ((19, 9, 8), (1, 2, 1), (1, 0, 0), (3, 2, 2)),   # its own x neighbour
])
def test_acoustic_overlap3_x_matches_oracle(n, dims, periods, o):
    """Overlap 3 in x: the launches store the x-exchange's planes (P, Vy,
    Vz: n - 3 and 2; Vx, overlap 4: n - 3 and 3) themselves; halo cells
    included, the run matches the oracle's decomposed run within 1e-12."""
    rho, K, h = 1.2, 2.3, (0.1, 0.08, 0.12)
    dt = 0.3 * min(h) / math.sqrt(K / rho)
    nt = 7
    host = decomposed_inputs(n, dims, periods, o, 5)
    ref = [a.copy() for a in host]
    oracle.acoustic_run_decomposed(*ref, nt, rho, K, dt, *h, n, dims, periods, o)
    with igg.Grid(n, dims=dims, overlap=o, periods=periods) as g:
        dev = [torch.from_numpy(a).cuda() for a in host]
        for _ in range(nt):
            g.acoustic_step(*dev, rho, K, dt, *h)
        torch.cuda.synchronize()
        got = [d.cpu().numpy() for d in dev]
    for name, a, r in zip(("P", "Vx", "Vy", "Vz"), got, ref):
        scale = max(np.abs(r).max(), 1e-300)
        assert np.abs(a - r).max() <= 1e-12 * scale, (name, np.abs(a - r).max() / scale)


def test_acoustic_energy_conserved_gpu():
    n = (48, 40, 36)
    rho, K, h = 1.1, 2.5, (0.1, 0.12, 0.09)
    dt = 0.3 * min(h) / math.sqrt(K / rho)
    g1 = [np.arange(k) for k in n]
    P0 = np.ascontiguousarray(np.broadcast_to(synth.gaussian_bump(*g1, n, sigma=0.2), (n[2], n[1], n[0]))) - 1.7
    with igg.Grid(n) as g:
        P, Vx, Vy, Vz = g.acoustic_fields()
        P.copy_(torch.from_numpy(P0).view(P.shape))
        E = []
        for _ in range(100):
            Pp = P.double().cpu().numpy()[0]
            g.acoustic_step(P, Vx, Vy, Vz, rho, K, dt, *h)
            torch.cuda.synchronize()
            E.append(oracle.acoustic_energy(Pp, *(t.cpu().numpy()[0] for t in (P, Vx, Vy, Vz)),
                                            rho, K, *h))
    assert np.abs(np.array(E) - E[0]).max() <= 1e-11 * abs(E[0])
