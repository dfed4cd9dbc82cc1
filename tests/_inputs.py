"""Input construction for parity tests. The oracle side maps local points to
global indices with the oracle's own grid bookkeeping; the GPU side with the
library's (igg_subdomain_info); both draw values from `synth`."""
import numpy as np

import oracle
import synth


def field_values(kind, seed, g, ng, l=(1.0, 1.0, 1.0)):
    if kind == "gaussian":
        return synth.gaussian_bump(*g, ng, l=l)
    if kind == "gaussian_rough":
        return synth.gaussian_bump(*g, ng, l=l, sigma=0.15) + 0.05 * synth.uniform(
            seed, 5, synth.global_linear_index(*g, ng))
    if kind == "sines":
        return synth.sine_modes(seed, *g, ng, l=l)
    if kind == "c0":
        return synth.ci_uniform_c0(seed, *g, ng)
    if kind == "uniform":
        return synth.ci_uniform(seed, *g, ng)
    raise ValueError(kind)


def oracle_fields(n, dims, periods, overlap, seed, tkind="gaussian_rough", ckind="c0"):
    """float64 [nsub][nz][ny][nx] T0 and Ci, oracle-side index mapping."""
    nsub = dims[0] * dims[1] * dims[2]
    ng = oracle.global_size(n, dims, overlap, periods)
    T = np.empty((nsub, n[2], n[1], n[0]))
    Ci = np.empty_like(T)
    for s in range(nsub):
        g = oracle.global_indices(n, dims, overlap, periods, s)
        T[s] = field_values(tkind, seed, g, ng)
        Ci[s] = field_values(ckind, seed, g, ng)
    dd = [oracle.spacing(1.0, ng[d]) for d in range(3)]
    return T, Ci, dd, ng


def grid_fields(grid, seed, tkind="gaussian_rough", ckind="c0"):
    """Same fields, GPU-side index mapping (numpy float64)."""
    ng = grid.global_size()
    T = np.empty(grid.shape)
    Ci = np.empty(grid.shape)
    for s in range(grid.nsub):
        g = grid.global_indices(s)
        T[s] = field_values(tkind, seed, g, ng)
        Ci[s] = field_values(ckind, seed, g, ng)
    return T, Ci
