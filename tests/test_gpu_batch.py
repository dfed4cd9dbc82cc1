"""GPU parity of the batched form: many uneven problems, one launch per step
(the vector kernel over per-problem tiles, or the persistent scalar
kernel), against the oracle run problem by problem; every kernel, tiling and
the single-grid kernel give the same bits."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

igg = pytest.importorskip("paper_2211_15716_gb300")
from paper_2211_15716_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def small_batch(count=13, nmin=3, nmax=41, seed=9):
    sizes, lam, ci = synth.batch_problems(seed, count, nmin, nmax)
    return [tuple(int(v) for v in s) for s in sizes], lam, ci


def oracle_run(sizes, lam, ci, nt):
    out = []
    for b, (nx, ny, nz) in enumerate(sizes):
        g = [np.arange(nx), np.arange(ny), np.arange(nz)]
        T0 = np.ascontiguousarray(np.broadcast_to(synth.gaussian_bump(*g, (nx, ny, nz)), (nz, ny, nx)))
        C = np.full(T0.shape, float(ci[b]))
        dd = [oracle.spacing(1.0, n) for n in (nx, ny, nz)]
        dt = oracle.cfl_dt(*dd, float(lam[b]), float(ci[b]))
        out.append((oracle.run(T0, C, nt, float(lam[b]), dt, *dd), dd, dt))
    return out


def gpu_batch(sizes, lam, ci, refs, dtype):
    B = igg.Batch(sizes, dtype)
    B.set_coefs(lam, [r[2] for r in refs], [r[1][0] for r in refs], [r[1][1] for r in refs],
                [r[1][2] for r in refs])
    T, T2, Ci = wl.make_batch_fields(B, ci, dtype)
    return B, T, T2, Ci


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_matches_oracle(dtype):
    sizes, lam, ci = small_batch()
    nt = 9
    refs = oracle_run(sizes, lam, ci, nt)
    B, T, T2, Ci = gpu_batch(sizes, lam, ci, refs, dtype)
    with B:
        res = B.run(nt, T, T2, Ci)
        torch.cuda.synchronize()
        for b in range(len(sizes)):
            gpu = B.view(res, b).double().cpu().numpy()
            ref = refs[b][0]
            err = np.abs(gpu - ref).max()
            if dtype == torch.float64:
                assert err <= 1e-12 * np.abs(ref).max(), (b, sizes[b], err)
            else:
                assert err <= (1 + nt) * 2 * 2.0 ** -24 * np.abs(ref).max(), (b, sizes[b], err)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_every_tiling_same_bits(dtype):
    sizes, lam, ci = small_batch(count=7, nmin=5, nmax=70, seed=4)
    refs = oracle_run(sizes, lam, ci, 0)
    B, T, T2, Ci = gpu_batch(sizes, lam, ci, refs, dtype)
    with B:
        outs = []
        for variant in range(5):
            for zb in (0, 1, 8, 32):
                B.configure(variant, zb, 0)
                R = T.clone()
                B.step(R, T, Ci)
                outs.append(R)
        torch.cuda.synchronize()
        bits = [o.view(torch.int16 if dtype == torch.bfloat16 else
                       (torch.int64 if dtype == torch.float64 else torch.int32)) for o in outs]
        for o in bits[1:]:
            assert torch.equal(o, bits[0])


def test_batch_equals_single_grid_kernel():
    """Problem b of the batch == the grid library's step on that problem
    alone, bit for bit (one arithmetic for all kernels)."""
    sizes, lam, ci = small_batch(count=5, nmin=10, nmax=50, seed=2)
    refs = oracle_run(sizes, lam, ci, 0)
    B, T, T2, Ci = gpu_batch(sizes, lam, ci, refs, torch.float32)
    with B:
        B.step(T2, T, Ci)
        for b, (nx, ny, nz) in enumerate(sizes):
            with igg.Grid((nx, ny, nz)) as g:
                t = B.view(T, b).contiguous().view(1, nz, ny, nx)
                c = B.view(Ci, b).contiguous().view(1, nz, ny, nx)
                r = t.clone()
                dd = refs[b][1]
                g.step(r, t, c, float(lam[b]), refs[b][2], *dd)
                torch.cuda.synchronize()
                assert torch.equal(r.view(-1).view(torch.int32), B.view(T2, b).reshape(-1).view(torch.int32))


def test_autotune_keeps_results():
    sizes, lam, ci = small_batch(count=20, nmin=8, nmax=64, seed=6)
    refs = oracle_run(sizes, lam, ci, 0)
    B, T, T2, Ci = gpu_batch(sizes, lam, ci, refs, torch.float32)
    with B:
        A = T.clone()
        B.step(A, T, Ci)
        best = B.autotune(T2, T, Ci, reps=2)
        assert 0 <= best["variant"] <= 4 and best["ms"] > 0
        cfg = B.config()
        assert (cfg["variant"], cfg["zb"], cfg["ctas_per_sm"]) == (best["variant"], best["zb"], best["ctas_per_sm"])
        R = T.clone()
        B.step(R, T, Ci)
        torch.cuda.synchronize()
        assert torch.equal(A.view(torch.int32), R.view(torch.int32))


def test_batch_gaps_untouched_and_layout():
    sizes = [(3, 3, 3), (5, 4, 3), (33, 9, 17)]
    B = igg.Batch(sizes, torch.float32)
    with B:
        assert B.offsets[0] == 0
        for b, (nx, ny, nz) in enumerate(sizes):
            assert B.pitches[b] >= nx and (B.pitches[b] * 4) % 16 == 0 and B.pitches[b] < nx + 4
        for b in range(1, 3):
            nx, ny, nz = sizes[b - 1]
            assert B.offsets[b] >= B.offsets[b - 1] + B.pitches[b - 1] * ny * nz
            assert (B.offsets[b] * 4) % 256 == 0
        B.set_coefs([1.0] * 3, [1e-3] * 3, [0.1] * 3, [0.1] * 3, [0.1] * 3)
        T = torch.full((B.total,), 7.0, device="cuda")
        Ci = torch.full((B.total,), 0.5, device="cuda")
        T2 = torch.full((B.total,), -3.0, device="cuda")
        B.step(T2, T, Ci)
        torch.cuda.synchronize()
        mask = torch.zeros(B.total, dtype=torch.bool, device="cuda")
        for b in range(len(sizes)):
            B.view(mask, b)[1:-1, 1:-1, 1:-1] = True
        assert (T2[mask] == 7.0).all()          # stationary field
        assert (T2[~mask] == -3.0).all()        # boundaries, row padding and gaps untouched


def test_batch_full_workload_every_problem():
    """256 problems, dims uniform on {32..192}, FP32, 200 steps through the
    graph (the autotuned tiling); every problem compared with the oracle in
    full, at the FP32 bound."""
    sizes, lam, ci, dd, dt = wl.batch_problems()
    B = igg.Batch(sizes, torch.float32)
    with B:
        B.set_coefs(lam, dt, [d[0] for d in dd], [d[1] for d in dd], [d[2] for d in dd])
        T, T2, Ci = wl.make_batch_fields(B, ci)
        B.autotune(T2, T, Ci, reps=1)
        T2.copy_(T)
        nt = 200
        res = B.run(nt, T, T2, Ci)
        torch.cuda.synchronize()
        oracle.set_threads(0)
        for b in range(len(sizes)):
            nx, ny, nz = sizes[b]
            g = [np.arange(nx), np.arange(ny), np.arange(nz)]
            T0 = np.ascontiguousarray(np.broadcast_to(synth.gaussian_bump(*g, (nx, ny, nz)), (nz, ny, nx)))
            ref = oracle.run(T0, np.full(T0.shape, float(ci[b])), nt, float(lam[b]), dt[b], *dd[b])
            gpu = B.view(res, b).double().cpu().numpy()
            assert np.abs(gpu - ref).max() <= (1 + nt) * 2 * 2.0 ** -24 * np.abs(ref).max()


_CACHE_SCRIPT = r"""
import sys, torch
sys.path.insert(0, {root!r})
import paper_2211_15716_gb300 as igg
sizes = [(8 + 3 * i, 9 + i, 7 + 2 * i) for i in range(12)]
B = igg.Batch(sizes, torch.float32)
n = len(sizes)
B.set_coefs([1.0] * n, [1e-4] * n, [0.1] * n, [0.1] * n, [0.1] * n)
T = B.empty().fill_(1.5)
C = B.empty().fill_(0.5)
T2 = B.empty().fill_(-7.0)
best = B.autotune(T2, T, C, reps=2)
untouched = bool((T2 == -7.0).all())
print(best["variant"], best["zb"], best["ctas_per_sm"], int(untouched))
B.destroy()
"""


def test_autotune_cache_in_process_and_file(tmp_path):
    """A second batch of the same shapes takes the cached tiling without
    timing (T2 untouched), in the same process and, through the file named
    by IGG_AUTOTUNE_CACHE, in a new one; reps < 0 times again."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, IGG_AUTOTUNE_CACHE=str(cache))
    outs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _CACHE_SCRIPT.format(root=root)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(list(map(int, r.stdout.split()[-4:])))
    assert outs[0][3] == 0  # tuned: T2 written
    assert outs[1][:3] == outs[0][:3] and outs[1][3] == 1  # from the file: nothing timed
    lines = cache.read_text().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1 and "|dt1|n12|" in lines[0]
    # in-process: the first call tunes, the second is cached, reps < 0 re-tunes
    sizes, lam, ci = small_batch(count=7, nmin=8, nmax=30, seed=11)
    refs = oracle_run(sizes, lam, ci, 0)
    B, T, T2, Ci = gpu_batch(sizes, lam, ci, refs, torch.float32)
    with B:
        a = B.autotune(T2, T, Ci, reps=1)
        T2.fill_(-3.0)
        b = B.autotune(T2, T, Ci, reps=1)
        assert bool((T2 == -3.0).all()) and (a["variant"], a["zb"]) == (b["variant"], b["zb"])
        B.autotune(T2, T, Ci, reps=-1)
        assert not bool((T2 == -3.0).all())
