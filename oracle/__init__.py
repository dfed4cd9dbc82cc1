"""Oracle: a plain, slow, FP64 CPU statement of the heat-diffusion hot path of
"Distributed Parallelization of xPU Stencil Computations in Julia"
(Omlin, Raess, Utkin; arXiv 2211.15716).

TEST INFRASTRUCTURE ONLY. The test-suite, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may use this package; the GPU library never
does, and this package imports nothing from it. The element loops are plain C
(`oracle.c`, built with -ffp-contract=off so that every operation rounds as
written); the grid bookkeeping and the time-loop drivers below are plain
Python/numpy.

What each function follows (section / figure of the paper):
  * dims_create, global_size, coords, neighbours, global_indices:
    the implicit global grid built from the number of processes and a
    process topology that is given or chosen automatically (Sec. Approach;
    Fig. 1 init_global_grid, nx_g()/ny_g()/nz_g()).
  * spacing, cfl_dt: Fig. 1's dx = lx/(nx_g()-1) and
    dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1.
  * step: Fig. 1's step! kernel on inner points.
  * step_part: the same update restricted to the boundary set or the inner
    block of @hide_communication (16, 2, 2) (Fig. 1; Sec. Approach).
  * update_halo: update_halo! (Sec. Approach; Fig. 1), dims in x, y, z order.
  * run / run_decomposed: Fig. 1's time loop, T2 = copy(T), step!, halo
    update of T2, swap T, T2 = T2, T.
  * adjoint_step / gradient: the transposed step run backward in time, for
    a misfit loss 0.5*sum((T_nt - T_obs)^2) (the differentiated form of the
    Fig. 1 solver).
  * update_halo_adjoint / gradient_decomposed: the same on a grid of
    subdomains: the transpose of the halo update (each halo entry added into
    its source and set to 0, dimensions z, y, x), then the transposed step on
    every subdomain.
Readings of points the paper leaves open (overlap 2 with halo width 1,
global size n_g = dims*(n-o) + o for non-periodic and dims*(n-o) for periodic
dimensions, subdomain numbering x fastest, the second difference as a
difference of one-sided differences, the boundary set of the split) are
stated where they are used.

Pins (tests/test_oracle_*.py): discrete Fourier-mode decay (closed form),
stationarity, conservation of sum(T/Ci) with periodic boundaries, mirror
symmetry, a Kronecker-sum sparse Laplacian, a hand-computed 3x3x3 golden
case, decomposed == undecomposed bit for bit, split == unsplit bit for bit,
MPI_Dims_create examples, adjoint dot-product identities and central finite
differences (single array and decomposed grids; the decomposed gradient
equals the single-array one on one subdomain, bit for bit).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from itertools import product

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


# --------------------------------------------------------------------------
# build / load
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP when present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L = ctypes.c_long
        D = ctypes.c_double
        lib.oracle_step.argtypes = [L, L, L, P, P, P, D, D, D, D, D]
        lib.oracle_step_part.argtypes = [L, L, L, P, P, P, D, D, D, D, D, L, L, L, ctypes.c_int]
        lib.oracle_update_halo.argtypes = [ctypes.c_int, P, P, L, L, L, P, P, L]
        lib.oracle_update_halo_adjoint.argtypes = [ctypes.c_int, P, P, L, L, L, P, P]
        lib.oracle_adjoint_step.argtypes = [L, L, L, P, P, P, P, P, D, D, D, D, D]
        lib.oracle_acoustic_step.argtypes = [L, L, L, P, P, P, P, D, D, D, D, D, D]
        lib.oracle_gp_half.argtypes = [L, L, L, ctypes.c_int, P, P, P, D, D, D, D, D]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the C loops; returns the count in use."""
    lib = _load()
    lib.oracle_set_threads(int(n))
    return lib.oracle_threads()


def threads() -> int:
    return _load().oracle_threads()


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check3(a: np.ndarray, dtype=np.float64):
    if a.dtype != dtype or not a.flags.c_contiguous:
        raise ValueError("oracle arrays must be C-contiguous " + np.dtype(dtype).name)


# --------------------------------------------------------------------------
# implicit global grid (Sec. Approach; Fig. 1 init_global_grid, nx_g())
# --------------------------------------------------------------------------
def dims_create(nsub: int, dims=(0, 0, 0)) -> tuple:
    """Balanced factorisation of nsub over the zero entries of dims, as
    MPI_Dims_create defines it: the free entries are as close to each other as
    possible and in non-increasing order. Brute force over all assignments:
    minimise the largest free factor, then the spread, then prefer the
    non-increasing order. Raises ValueError if impossible."""
    dims = list(int(d) for d in dims)
    fixed = 1
    for d in dims:
        if d < 0:
            raise ValueError("negative dims entry")
        if d > 0:
            fixed *= d
    if nsub <= 0 or nsub % fixed:
        raise ValueError("nsub is not a multiple of the fixed dims")
    rest = nsub // fixed
    free = [i for i, d in enumerate(dims) if d == 0]
    if not free:
        if rest != 1:
            raise ValueError("dims product differs from nsub")
        return tuple(dims)
    divisors = [k for k in range(1, rest + 1) if rest % k == 0]
    best = None
    for combo in product(divisors, repeat=len(free)):
        if math.prod(combo) != rest:
            continue
        if list(combo) != sorted(combo, reverse=True):
            continue
        key = (max(combo), max(combo) - min(combo))
        if best is None or key < best[0]:
            best = (key, combo)
    for i, v in zip(free, best[1]):
        dims[i] = v
    return tuple(dims)


def global_size(n, dims, overlap, periods) -> tuple:
    """n_g per dimension: dims*(n-o) + o for a non-periodic dimension and
    dims*(n-o) for a periodic one (reading of the implicit global grid: the
    last o planes of a subdomain coincide with the first o of the next). A
    dimension of size 1 is absent (2-D and 1-D grids): one subdomain, not
    periodic, n_g = 1."""
    for d in range(3):
        if n[d] == 1 and (dims[d] != 1 or periods[d]):
            raise ValueError("a dimension of size 1 needs dims 1 and no periodicity")
    return tuple(1 if n[d] == 1 else
                 dims[d] * (n[d] - overlap[d]) + (0 if periods[d] else overlap[d])
                 for d in range(3))


def coords(sub: int, dims) -> tuple:
    """Cartesian coordinates of subdomain `sub`, x fastest."""
    return (sub % dims[0], (sub // dims[0]) % dims[1], sub // (dims[0] * dims[1]))


def sub_index(c, dims) -> int:
    return c[0] + dims[0] * (c[1] + dims[1] * c[2])


def neighbours(dims, periods):
    """(left, right): int32 arrays [nsub][3] of neighbour subdomain numbers,
    -1 where the dimension ends at a physical boundary."""
    nsub = dims[0] * dims[1] * dims[2]
    left = np.full((nsub, 3), -1, dtype=np.int32)
    right = np.full((nsub, 3), -1, dtype=np.int32)
    for s in range(nsub):
        c = coords(s, dims)
        for d in range(3):
            for side, step in ((left, -1), (right, +1)):
                cc = list(c)
                cc[d] += step
                if cc[d] < 0 or cc[d] >= dims[d]:
                    if not periods[d]:
                        continue
                    cc[d] %= dims[d]
                side[s, d] = sub_index(cc, dims)
    return left, right


def global_indices(n, dims, overlap, periods, sub: int):
    """Per axis, the global index of each local point of subdomain `sub`:
    coord*(n-o) + i, wrapped modulo n_g in a periodic dimension."""
    c = coords(sub, dims)
    ng = global_size(n, dims, overlap, periods)
    out = []
    for d in range(3):
        g = c[d] * (n[d] - overlap[d]) + np.arange(n[d], dtype=np.int64)
        if n[d] == 1:
            g = np.zeros(1, dtype=np.int64)
        if periods[d]:
            g = g % ng[d]
        out.append(g)
    return out


def undecomposed_index(n, dims, overlap, sub: int):
    """Per axis, the index in the undecomposed array (extent n_g, or n_g + o
    for a periodic dimension) of each local point of subdomain `sub`."""
    c = coords(sub, dims)
    return [np.zeros(1, dtype=np.int64) if n[d] == 1 else
            c[d] * (n[d] - overlap[d]) + np.arange(n[d], dtype=np.int64) for d in range(3)]


def spacing(l: float, n_g: int) -> float:
    """Fig. 1: dx = lx/(nx_g()-1); +inf for an absent dimension (n_g = 1), whose
    term d2/dd^2 is then 0."""
    return math.inf if n_g == 1 else l / (n_g - 1)


def cfl_dt(dx: float, dy: float, dz: float, lam: float, ci_max: float) -> float:
    """Fig. 1: dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1, left to right."""
    return min(dx * dx, dy * dy, dz * dz) / lam / ci_max / 6.1


# --------------------------------------------------------------------------
# element loops (oracle.c)
# --------------------------------------------------------------------------
def step(T2: np.ndarray, T: np.ndarray, Ci: np.ndarray, lam, dt, dx, dy, dz):
    """Fig. 1 step! on one local array [nz][ny][nx] (inner points of T2)."""
    for a in (T2, T, Ci):
        _check3(a)
    nz, ny, nx = T.shape
    _load().oracle_step(nx, ny, nz, _ptr(T2), _ptr(T), _ptr(Ci), lam, dt, dx, dy, dz)


def step_part(T2, T, Ci, lam, dt, dx, dy, dz, widths, select: int):
    """Boundary set (select=1) or inner block (select=0) of the split."""
    for a in (T2, T, Ci):
        _check3(a)
    nz, ny, nx = T.shape
    _load().oracle_step_part(nx, ny, nz, _ptr(T2), _ptr(T), _ptr(Ci), lam, dt, dx, dy, dz,
                             widths[0], widths[1], widths[2], select)


def update_halo(field: np.ndarray, dims, periods, overlap):
    """update_halo! on a field [nsub][nz][ny][nx] of any element type."""
    if not field.flags.c_contiguous or field.ndim != 4:
        raise ValueError("field must be C-contiguous [nsub][nz][ny][nx]")
    nsub, nz, ny, nx = field.shape
    left, right = neighbours(dims, periods)
    if left.shape[0] != nsub:
        raise ValueError("field's subdomain count differs from dims")
    ov = np.ascontiguousarray(overlap, dtype=np.int64)
    _load().oracle_update_halo(nsub, _ptr(left), _ptr(right), nx, ny, nz, _ptr(ov),
                               _ptr(field), field.dtype.itemsize)


def update_halo_adjoint(lam: np.ndarray, dims, periods, overlap):
    """The transpose of update_halo on an FP64 field [nsub][nz][ny][nx], in
    place: every halo entry is added into the entry its value came from and
    set to 0, dimensions z, then y, then x (see oracle.c)."""
    if not lam.flags.c_contiguous or lam.ndim != 4 or lam.dtype != np.float64:
        raise ValueError("lam must be a C-contiguous float64 [nsub][nz][ny][nx]")
    nsub, nz, ny, nx = lam.shape
    left, right = neighbours(dims, periods)
    if left.shape[0] != nsub:
        raise ValueError("field's subdomain count differs from dims")
    ov = np.ascontiguousarray(overlap, dtype=np.int64)
    _load().oracle_update_halo_adjoint(nsub, _ptr(left), _ptr(right), nx, ny, nz, _ptr(ov),
                                       _ptr(lam))


def staggered_overlap(n, nf, overlap):
    """Overlap of a field of local size nf on a grid of local size n and
    overlap o: o + (nf - n) per dimension (the staggered points on a shared
    face are shared too)."""
    return tuple(int(overlap[d]) + int(nf[d]) - int(n[d]) for d in range(3))


def update_halo_staggered(field: np.ndarray, n, dims, periods, overlap):
    """update_halo! on a staggered field [nsub][nf_z][nf_y][nf_x] whose local
    size differs from the grid's n by at most one point per dimension: the
    plain halo update with the field's own overlap (staggered_overlap);
    dimensions where that is below 2 exchange nothing."""
    nf = (field.shape[3], field.shape[2], field.shape[1])
    if any(abs(nf[d] - int(n[d])) > 1 for d in range(3)):
        raise ValueError("a staggered field differs from the grid by at most one point")
    update_halo(field, dims, periods, staggered_overlap(n, nf, overlap))


def acoustic_step(P, Vx, Vy, Vz, rho, K, dt, dx, dy, dz):
    """One leapfrog step of staggered-grid acoustics on one array (see
    oracle.c): P [nz][ny][nx], Vx [nz][ny][nx+1], Vy [nz][ny+1][nx],
    Vz [nz+1][ny][nx], all updated in place."""
    nz, ny, nx = P.shape
    for a, shape in ((P, (nz, ny, nx)), (Vx, (nz, ny, nx + 1)), (Vy, (nz, ny + 1, nx)),
                     (Vz, (nz + 1, ny, nx))):
        _check3(a)
        if a.shape != shape:
            raise ValueError(f"field shape {a.shape}, expected {shape}")
    _load().oracle_acoustic_step(nx, ny, nz, _ptr(P), _ptr(Vx), _ptr(Vy), _ptr(Vz), rho, K, dt,
                                 dx, dy, dz)


def acoustic_run_decomposed(P, Vx, Vy, Vz, nt, rho, K, dt, dx, dy, dz, n, dims, periods,
                            overlap):
    """nt acoustic steps on a decomposed grid (local cell size n, fields
    [nsub][...] in place): every subdomain steps, then update_halo! of P, Vx,
    Vy, Vz with their staggered overlaps."""
    for _ in range(nt):
        for s in range(P.shape[0]):
            acoustic_step(P[s], Vx[s], Vy[s], Vz[s], rho, K, dt, dx, dy, dz)
        for f in (P, Vx, Vy, Vz):
            update_halo_staggered(f, n, dims, periods, overlap)


def acoustic_energy(P_prev, P, Vx, Vy, Vz, rho, K, dx, dy, dz):
    """Energy of the leapfrog scheme between two consecutive steps on one
    array: (sum P_prev*P/(2K) + rho/2 sum |V|^2) * cell volume, with P_prev
    the cell field before and P, V the fields after a step (fsum). With zero
    velocities on the walls the discrete divergence is minus the transpose of
    the discrete gradient, and this quantity is the same after every step."""
    terms = [float(x) for x in (P_prev * P).ravel() / (2.0 * K)]
    for v in (Vx, Vy, Vz):
        terms += [float(x) for x in (0.5 * rho * v * v).ravel()]
    return math.fsum(terms) * (dx * dy * dz)


def gp_half(which, u, v, V, g, dt, dx, dy, dz):
    """One half step of the Gross-Pitaevskii solver on one array (see
    oracle.c): which 0 updates u from v, which 1 updates v from u."""
    for a in (u, v, V):
        _check3(a)
    nz, ny, nx = u.shape
    _load().oracle_gp_half(nx, ny, nz, int(which), _ptr(u), _ptr(v), _ptr(V), g, dt, dx, dy, dz)


def gp_run(u, v, V, nt, g, dt, dx, dy, dz):
    """nt steps (u half, then v half) on one array, in place."""
    for _ in range(nt):
        gp_half(0, u, v, V, g, dt, dx, dy, dz)
        gp_half(1, u, v, V, g, dt, dx, dy, dz)


def gp_run_decomposed(u, v, V, nt, g, dt, dx, dy, dz, dims, periods, overlap):
    """nt steps on a decomposed grid ([nsub][nz][ny][nx] in place): every
    subdomain's u half, update_halo!(u), every subdomain's v half,
    update_halo!(v) (the v half reads the new u at halo points)."""
    for _ in range(nt):
        for which, f in ((0, u), (1, v)):
            for s in range(u.shape[0]):
                gp_half(which, u[s], v[s], V[s], g, dt, dx, dy, dz)
            update_halo(f, dims, periods, overlap)


def gp_invariant(u, v_prev, v):
    """||u^n||^2 + <v^{n+1/2}, v^{n-1/2}> (fsum): with g = 0, zero boundary
    values and a symmetric H, the same after every step."""
    return math.fsum([float(x) for x in (u * u).ravel()] + [float(x) for x in (v * v_prev).ravel()])


def adjoint_step(lam_out, lam_in, Tn, Ci, gCi, lam, dt, dx, dy, dz):
    """One backward step of the adjoint (see oracle.c)."""
    for a in (lam_out, lam_in, Tn, Ci, gCi):
        _check3(a)
    nz, ny, nx = Tn.shape
    _load().oracle_adjoint_step(nx, ny, nz, _ptr(lam_out), _ptr(lam_in), _ptr(Tn), _ptr(Ci),
                                _ptr(gCi), lam, dt, dx, dy, dz)


# --------------------------------------------------------------------------
# drivers: Fig. 1's time loop
# --------------------------------------------------------------------------
def run(T0: np.ndarray, Ci: np.ndarray, nt: int, lam, dt, dx, dy, dz,
        periodic_self_halo=None, overlap=(2, 2, 2)) -> np.ndarray:
    """Fig. 1's loop on one undecomposed array: T2 = copy(T); nt times
    {step!(T2, T); halo update of T2; swap}. `periodic_self_halo` is the
    periods triple of a single-subdomain periodic grid, or None."""
    T = np.array(T0, dtype=np.float64, order="C", copy=True)
    T2 = T.copy()
    for _ in range(nt):
        step(T2, T, Ci, lam, dt, dx, dy, dz)
        if periodic_self_halo is not None and any(periodic_self_halo):
            update_halo(T2[None], (1, 1, 1), periodic_self_halo, overlap)
        T, T2 = T2, T
    return T


def run_decomposed(T0: np.ndarray, Ci: np.ndarray, nt: int, lam, dt, dx, dy, dz,
                   dims, periods, overlap, widths=None) -> np.ndarray:
    """Fig. 1's loop on a grid of subdomains, fields [nsub][nz][ny][nx]:
    per step, step! on every subdomain (or, with `widths`, the boundary set of
    every subdomain, then the halo update, then the inner blocks, which is the
    @hide_communication order), then update_halo!(T2), then the swap."""
    T = np.array(T0, dtype=np.float64, order="C", copy=True)
    T2 = T.copy()
    nsub = T.shape[0]
    for _ in range(nt):
        if widths is None:
            for s in range(nsub):
                step(T2[s], T[s], Ci[s], lam, dt, dx, dy, dz)
            update_halo(T2, dims, periods, overlap)
        else:
            for s in range(nsub):
                step_part(T2[s], T[s], Ci[s], lam, dt, dx, dy, dz, widths, 1)
            update_halo(T2, dims, periods, overlap)
            for s in range(nsub):
                step_part(T2[s], T[s], Ci[s], lam, dt, dx, dy, dz, widths, 0)
        T, T2 = T2, T
    return T


# --------------------------------------------------------------------------
# adjoint drivers (gradient of 0.5*sum((T_nt - T_obs)^2))
# --------------------------------------------------------------------------
def forward_states(T0, Ci, nt, lam, dt, dx, dy, dz):
    """All states T_0..T_nt of the single-array loop (no checkpointing)."""
    states = [np.array(T0, dtype=np.float64, order="C", copy=True)]
    for _ in range(nt):
        T2 = states[-1].copy()
        step(T2, states[-1], Ci, lam, dt, dx, dy, dz)
        states.append(T2)
    return states


def fsum(a: np.ndarray) -> float:
    """Correctly rounded sum of all entries (math.fsum)."""
    return math.fsum(np.asarray(a, dtype=np.float64).ravel().tolist())


def loss(T_nt, T_obs) -> float:
    """J = 0.5*sum((T_nt - T_obs)^2), summed with math.fsum."""
    r = np.asarray(T_nt, dtype=np.float64) - np.asarray(T_obs, dtype=np.float64)
    return 0.5 * fsum(r * r)


def gradient(T0, Ci, T_obs, nt, lam, dt, dx, dy, dz):
    """(J, dJ/dT0, dJ/dCi) by the discrete adjoint, dt held fixed."""
    states = forward_states(T0, Ci, nt, lam, dt, dx, dy, dz)
    J = loss(states[-1], T_obs)
    lam_n = np.ascontiguousarray(states[-1] - T_obs)
    gCi = np.zeros_like(lam_n)
    out = np.empty_like(lam_n)
    for n in range(nt - 1, -1, -1):
        adjoint_step(out, lam_n, states[n], np.ascontiguousarray(Ci, dtype=np.float64), gCi,
                     lam, dt, dx, dy, dz)
        lam_n, out = out, lam_n
    return J, lam_n.copy(), gCi


# --------------------------------------------------------------------------
# reduced precision
# --------------------------------------------------------------------------
def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest BF16 value (8 significant bits, ties
    to even), returned as FP64. Plain definition via frexp/rint; finite,
    normal-range inputs."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)            # x = m * 2^e, 0.5 <= |m| < 1
    q = np.rint(m * 256.0)        # 8 significant bits, ties to even
    return np.ldexp(q / 256.0, e)


def bf16_ulp(x: np.ndarray) -> np.ndarray:
    """Spacing of BF16 values at |x| (normal range)."""
    _, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(1.0, e - 8)


# --------------------------------------------------------------------------
# adjoint on a grid of subdomains
# --------------------------------------------------------------------------
def forward_states_decomposed(T0, Ci, nt, lam, dt, dx, dy, dz, dims, periods, overlap):
    """All states T_0..T_nt of run_decomposed (no checkpointing): per step,
    step! on every subdomain, then update_halo!."""
    states = [np.array(T0, dtype=np.float64, order="C", copy=True)]
    for _ in range(nt):
        T = states[-1]
        T2 = T.copy()
        for s in range(T.shape[0]):
            step(T2[s], T[s], Ci[s], lam, dt, dx, dy, dz)
        update_halo(T2, dims, periods, overlap)
        states.append(T2)
    return states


def gradient_decomposed(T0, Ci, T_obs, nt, lam, dt, dx, dy, dz, dims, periods, overlap):
    """(J, dJ/dT0, dJ/dCi) of J = 0.5*sum((T_nt - T_obs)^2) over every entry
    of the decomposed fields [nsub][nz][ny][nx] (dt held fixed). One step is
    T_{n+1} = H(S(T_n)): S the step on every subdomain (the identity off its
    inner points), H the halo update. Backward in time, lam <- H^T lam
    (update_halo_adjoint), then lam <- S^T lam and gCi += k lam L(T_n) on
    every subdomain (adjoint_step)."""
    states = forward_states_decomposed(T0, Ci, nt, lam, dt, dx, dy, dz, dims, periods, overlap)
    J = loss(states[-1], T_obs)
    lam_n = np.ascontiguousarray(states[-1] - T_obs)
    gCi = np.zeros_like(lam_n)
    out = np.empty_like(lam_n)
    C = np.ascontiguousarray(Ci, dtype=np.float64)
    for n in range(nt - 1, -1, -1):
        update_halo_adjoint(lam_n, dims, periods, overlap)
        for s in range(lam_n.shape[0]):
            adjoint_step(out[s], lam_n[s], states[n][s], C[s], gCi[s], lam, dt, dx, dy, dz)
        lam_n, out = out, lam_n
    return J, lam_n.copy(), gCi
