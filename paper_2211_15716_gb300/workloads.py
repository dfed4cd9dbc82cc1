"""Synthetic workloads on a Grid: inputs from the seeded generators (synth),
drawn on global indices so that any decomposition holds the same global field,
and Fig. 1's set-up: dx = lx/(nx_g()-1) and
dt = min(dx^2, dy^2, dz^2)/lam/maximum(Ci)/6.1, with maximum(Ci) reduced on
the device in FP64.

Workloads (each the physics of Fig. 1 with seeded, randomised inputs):
  * single 64^3 FP64 grid, Gaussian bump, c0 ~ U[1.5, 2.5], nt = 100;
  * 2x2x2 subdomains of 512x256x256 FP64 (overlap 2, periodic in x),
    hidden communication with widths (16, 2, 2), same physics, nt = 100;
  * the same decomposed grid with T0 = 8 sine modes of amplitude 0.1 about 0
    (a field that changes sign);
  * a 1024^3 grid in FP32 / BF16 storage with Ci ~ U[0.4, 0.67] and 8 sine
    modes of amplitude 0.1 on 1.7 (error check at 128^3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

import synth

from .igg import RED_MAX, Grid, reduce


def spacing(l: float, n_g: int) -> float:
    """Fig. 1: dx = lx/(nx_g()-1); +inf for an absent dimension (n_g = 1) of a
    2-D or 1-D grid, whose weight dt*lam/dx^2 is then 0."""
    return float("inf") if n_g == 1 else l / (n_g - 1)


def cfl_dt(dx: float, dy: float, dz: float, lam: float, ci_max: float) -> float:
    """Fig. 1: dt = min(dx^2, dy^2, dz^2)/lam/maximum(Ci)/6.1."""
    return min(dx * dx, dy * dy, dz * dz) / lam / ci_max / 6.1


@dataclass
class Workload:
    name: str
    n: tuple
    dims: tuple = (1, 1, 1)
    periods: tuple = (0, 0, 0)
    overlap: tuple = (2, 2, 2)
    widths: tuple | None = None
    nt: int = 100
    lam: float = 1.0
    l: tuple = (1.0, 1.0, 1.0)
    seed: int = 0
    t0: str = "gaussian"       # "gaussian" | "sines"
    ci: str = "c0"             # "c0": Ci = 1/U[1.5,2.5]; "uniform": Ci ~ U[0.4, 0.67]
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "single64": Workload("single64", (64, 64, 64), seed=0),
    "decomposed_2x2x2_512x256x256": Workload(
        "decomposed_2x2x2_512x256x256", (512, 256, 256), dims=(2, 2, 2), periods=(1, 0, 0),
        widths=(16, 2, 2), seed=1),
    "decomposed_2x2x2_256x128x128": Workload(
        "decomposed_2x2x2_256x128x128", (256, 128, 128), dims=(2, 2, 2), periods=(1, 0, 0),
        widths=(16, 2, 2), seed=1),
    # the same grid and physics with a sign-changing T0 (the sine modes about
    # 0): the emulated FP64 cell's worst case (stencils across zero and across
    # powers of two)
    "decomposed_2x2x2_512x256x256_signed": Workload(
        "decomposed_2x2x2_512x256x256_signed", (512, 256, 256), dims=(2, 2, 2), periods=(1, 0, 0),
        widths=(16, 2, 2), seed=1, t0="sines0"),
    "decomposed_2x2x2_256x128x128_signed": Workload(
        "decomposed_2x2x2_256x128x128_signed", (256, 128, 128), dims=(2, 2, 2), periods=(1, 0, 0),
        widths=(16, 2, 2), seed=1, t0="sines0"),
    "precision_1024": Workload("precision_1024", (1024, 1024, 1024), nt=1000, seed=2, t0="sines",
                               ci="uniform"),
    "precision_128": Workload("precision_128", (128, 128, 128), nt=1000, seed=2, t0="sines",
                              ci="uniform"),
}


def host_fields(w: Workload, grid: Grid, sub: int):
    """(T0, Ci) of one subdomain as float64 numpy arrays [nz][ny][nx]."""
    ng = grid.global_size()
    g = grid.global_indices(sub)
    if w.t0 == "gaussian":
        T = synth.gaussian_bump(*g, ng, l=w.l)
    elif w.t0 == "sines0":
        T = synth.sine_modes(w.seed, *g, ng, l=w.l, base=0.0)
    else:
        T = synth.sine_modes(w.seed, *g, ng, l=w.l)
    if w.ci == "c0":
        Ci = synth.ci_uniform_c0(w.seed, *g, ng)
    else:
        Ci = synth.ci_uniform(w.seed, *g, ng)
    shape = (grid.n[2], grid.n[1], grid.n[0])
    return np.broadcast_to(T, shape), np.broadcast_to(Ci, shape)


def _to_device(a64: np.ndarray, dtype: torch.dtype, out: torch.Tensor):
    if dtype == torch.float64:
        out.copy_(torch.from_numpy(np.array(a64, dtype=np.float64, order="C", copy=True)))
    elif dtype == torch.float32:
        out.copy_(torch.from_numpy(synth.to_f32(a64)))
    else:
        bits = synth.to_bf16_bits(a64)
        out.view(torch.int16).copy_(torch.from_numpy(bits.view(np.int16)))


def make_fields(w: Workload, grid: Grid, dtype=torch.float64):
    """Device fields T, T2 (= copy(T), Fig. 1) and Ci of the workload."""
    T = grid.empty(dtype)
    Ci = grid.empty(dtype)
    for s in range(grid.nsub):
        T0, C = host_fields(w, grid, s)
        _to_device(T0, dtype, T[s])
        _to_device(C, dtype, Ci[s])
    T2 = T.clone()
    return T, T2, Ci


def setup(w: Workload, grid: Grid, Ci: torch.Tensor):
    """(dx, dy, dz, dt) of Fig. 1 for the workload on `grid`."""
    ng = grid.global_size()
    dx, dy, dz = (spacing(w.l[d], ng[d]) for d in range(3))
    ci_max = float(reduce(RED_MAX, Ci).item())
    return dx, dy, dz, cfl_dt(dx, dy, dz, w.lam, ci_max)


def batch_problems(seed=3, count=256, nmin=32, nmax=192):
    """The batched workload: `count` problems with each dimension uniform on
    {nmin..nmax}, lam ~ U[0.5, 2], constant Ci = 1/U[1.5, 2.5] per problem,
    Gaussian-bump T0, per-problem dx = 1/(n-1) and dt by Fig. 1's rule."""
    sizes, lam, ci = synth.batch_problems(seed, count, nmin, nmax)
    dd = [[spacing(1.0, int(n)) for n in s] for s in sizes]
    dt = [cfl_dt(*dd[b], float(lam[b]), float(ci[b])) for b in range(count)]
    return [tuple(int(v) for v in s) for s in sizes], lam, ci, dd, dt


def make_batch_fields(batch, ci, dtype=torch.float32):
    """T (Gaussian bump per problem), T2 = copy(T) and Ci (constant per
    problem) packed in the batch layout."""
    T = batch.empty()
    Ci = batch.empty()
    T.zero_()
    Ci.zero_()
    for b, (nx, ny, nz) in enumerate(batch.sizes):
        g = [np.arange(nx), np.arange(ny), np.arange(nz)]
        t0 = np.broadcast_to(synth.gaussian_bump(*g, (nx, ny, nz)), (nz, ny, nx))
        _to_device(t0, dtype, batch.view(T, b))
        _to_device(np.full((nz, ny, nx), float(ci[b])), dtype, batch.view(Ci, b))
    return T, T.clone(), Ci
