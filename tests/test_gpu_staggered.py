"""GPU parity of the staggered-field halo update (igg_update_halo_staggered)
against the oracle: bit exact on random bit patterns, several fields per
call, every element size; sizes off by more than one point are rejected."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")

CASES = [
    # n, dims, periods, overlap, delta (field size n + delta)
    ((8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2), (1, 0, 0)),
    ((8, 7, 6), (2, 2, 2), (1, 1, 0), (2, 2, 2), (1, 1, 1)),
    ((9, 8, 7), (3, 1, 2), (0, 1, 1), (3, 2, 3), (-1, 1, -1)),
    ((7, 7, 7), (2, 2, 1), (1, 0, 1), (2, 2, 2), (-1, 0, 1)),
    ((6, 6, 6), (1, 1, 1), (1, 1, 1), (2, 2, 2), (1, 1, 1)),
    ((33, 18, 12), (2, 3, 2), (1, 0, 1), (2, 2, 2), (1, -1, 1)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("es,npdt,tdt", [(8, np.uint64, torch.float64), (4, np.uint32, torch.float32),
                                         (2, np.uint16, torch.bfloat16)])
@pytest.mark.parametrize("n,dims,periods,overlap,delta", CASES)
def test_staggered_halo_bit_exact(n, dims, periods, overlap, delta, es, npdt, tdt):
    nf = tuple(n[d] + delta[d] for d in range(3))
    nsub = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(17)
    fields = [rng.integers(0, np.iinfo(npdt).max, size=(nsub, nf[2], nf[1], nf[0]), dtype=npdt,
                           endpoint=True) for _ in range(2)]
    refs = [f.copy() for f in fields]
    for r in refs:
        oracle.update_halo_staggered(r, n, dims, periods, overlap)
    ivt = {8: torch.int64, 4: torch.int32, 2: torch.int16}[es]
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        dev = [torch.from_numpy(f.view({8: np.int64, 4: np.int32, 2: np.int16}[es])).cuda().view(tdt)
               for f in fields]
        g.update_halo_staggered(nf, *dev)
        torch.cuda.synchronize()
        for d, r in zip(dev, refs):
            got = d.view(ivt).cpu().numpy().view(npdt)
            assert np.array_equal(got, r)


def test_staggered_sizes_rejected():
    with igg.Grid((8, 8, 8), dims=(2, 1, 1)) as g:
        for nf in [(10, 8, 8), (8, 6, 8), (2, 8, 8)]:
            t = torch.zeros(2 * nf[0] * nf[1] * nf[2], dtype=torch.float64, device="cuda")
            with pytest.raises(igg.IggError):
                g.update_halo_staggered(nf, t)


@pytest.mark.parametrize("n,dims,periods,overlap", [
    ((8, 7, 6), (2, 2, 2), (0, 0, 0), (2, 2, 2)),
    ((12, 9, 10), (2, 1, 3), (1, 1, 0), (2, 3, 2)),
    ((6, 6, 6), (1, 1, 1), (1, 1, 1), (2, 2, 2)),
])
def test_fields_of_mixed_sizes_one_call(n, dims, periods, overlap):
    """A staggered set (a cell field and the three face fields, sizes n and
    n + e_d) updated in one call equals the oracle's update of each field."""
    sizes = [tuple(n)] + [tuple(n[k] + (1 if k == d else 0) for k in range(3)) for d in range(3)]
    nsub = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(5)
    host = [rng.integers(0, 2**63, size=(nsub, s[2], s[1], s[0]), dtype=np.uint64) for s in sizes]
    refs = [h.copy() for h in host]
    for r in refs:
        oracle.update_halo_staggered(r, n, dims, periods, overlap)
    with igg.Grid(n, dims=dims, overlap=overlap, periods=periods) as g:
        dev = [torch.from_numpy(h.view(np.int64)).cuda().view(torch.float64) for h in host]
        g.update_halo_fields(dev, sizes)
        torch.cuda.synchronize()
        for d, r in zip(dev, refs):
            assert np.array_equal(d.view(torch.int64).cpu().numpy().view(np.uint64), r)
