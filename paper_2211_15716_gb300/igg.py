"""Python binding of libigg.so (ctypes): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
turns torch tensors into device pointers and torch streams into
cudaStream_t handles, checks shapes and dtypes, and raises IggError on a
negative status. There is no fallback: if the library is missing, the first
call raises.

Names follow the paper (Fig. 1): init_global_grid -> Grid(...),
nx_g()/ny_g()/nz_g() -> Grid.global_size(), update_halo! ->
Grid.update_halo(...), step! -> Grid.step(...), @hide_communication ->
Grid.step_hidden(...), the time loop -> Grid.run(...),
finalize_global_grid -> Grid.finalize().
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

F64, F32, BF16 = 0, 1, 2
RED_MAX, RED_SUM, RED_SUM_DIV, RED_SUM_SQDIFF = 0, 1, 2, 3

_TORCH_DTYPE = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}
_lib = None


class IggError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"igg error {code}: {msg}")
        self.code = code


def library_path() -> str:
    """The library the binding loads: the bounds-checked build when the
    environment has IGG_BOUNDS_CHECK=1, else the release build."""
    return _build.LIB_CHECKED if os.environ.get("IGG_BOUNDS_CHECK") == "1" else _build.LIB


def lib():
    """Load libigg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run paper_2211_15716_gb300.build.build() "
                          "(the library has no CPU fallback)")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    IP = ctypes.POINTER(ctypes.c_int)
    L.igg_last_error.restype = ctypes.c_char_p
    L.igg_abi_version.restype = I
    L.igg_init_global_grid.argtypes = [I, I, I, IP, I, IP, IP, ctypes.POINTER(P)]
    L.igg_finalize_global_grid.argtypes = [P]
    L.igg_global_size.argtypes = [P, IP]
    L.igg_grid_shape.argtypes = [P, IP, IP, IP, IP, IP]
    L.igg_subdomain_info.argtypes = [P, I, IP, IP, IP, IP]
    L.igg_update_halo.argtypes = [P, ctypes.POINTER(P), I, I, P]
    L.igg_update_halo_staggered.argtypes = [P, ctypes.POINTER(P), I, I, IP, P]
    L.igg_update_halo_fields.argtypes = [P, ctypes.POINTER(P), IP, I, I, P]
    L.igg_acoustic_step.argtypes = [P, P, P, P, P, I, D, D, D, D, D, D, I, P]
    L.igg_gp_step.argtypes = [P, P, P, P, I, D, D, D, D, D, I, P]
    L.igg_step.argtypes = [P, P, P, P, I, D, D, D, D, D, P]
    L.igg_step_hidden.argtypes = [P, IP, P, P, P, I, D, D, D, D, D, P]
    L.igg_run.argtypes = [P, I, IP, P, P, P, I, D, D, D, D, D, P]
    L.igg_run_host.argtypes = [P, I, IP, P, P, P, P, P, I, D, D, D, D, D, P]
    L.igg_reduce.argtypes = [I, P, P, ctypes.c_size_t, I, P, P]
    L.igg_device_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint), I]
    L.igg_grid_set_option.argtypes = [P, I, I]
    L.igg_phase_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), IP]
    L.igg_fixup_stats.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong), I]
    L.igg_bounds_checked.argtypes = []
    L.igg_bounds_status.argtypes = [ctypes.POINTER(ctypes.c_uint), I]
    for name in ("igg_init_global_grid", "igg_finalize_global_grid", "igg_global_size",
                 "igg_grid_shape", "igg_subdomain_info", "igg_update_halo",
                 "igg_update_halo_staggered", "igg_update_halo_fields",
                 "igg_acoustic_step", "igg_gp_step", "igg_step",
                 "igg_step_hidden", "igg_run", "igg_run_host", "igg_reduce", "igg_device_status",
                 "igg_grid_set_option", "igg_phase_times", "igg_fixup_stats",
                 "igg_bounds_checked", "igg_bounds_status"):
        getattr(L, name).restype = I
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise IggError(rc, lib().igg_last_error().decode(errors="replace"))


def _ints(v):
    return (ctypes.c_int * 3)(*[int(x) for x in v])


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def dtype_code(dtype: torch.dtype) -> int:
    try:
        return _TORCH_DTYPE[dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {dtype}; use float64, float32 or bfloat16") from None


def _ptr(t: torch.Tensor, numel: int, dtype: torch.dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Implicit global grid of nsub subdomains of n = (nx, ny, nz) points in
    one device's memory (Fig. 1 init_global_grid). Fields are tensors of
    shape (nsub, nz, ny, nx)."""

    def __init__(self, n, dims=(0, 0, 0), nsub: int = 0, overlap=(2, 2, 2), periods=(0, 0, 0)):
        L = lib()
        h = ctypes.c_void_p()
        if nsub:
            nsub_arg = nsub
        elif all(dims):
            nsub_arg = dims[0] * dims[1] * dims[2]
        else:
            nsub_arg = 1 if not any(dims) else 0
        _check(L.igg_init_global_grid(int(n[0]), int(n[1]), int(n[2]), _ints(dims), int(nsub_arg),
                                      _ints(overlap), _ints(periods), ctypes.byref(h)))
        self._h = h
        nn, dd, oo, pp, ns = _ints((0, 0, 0)), _ints((0, 0, 0)), _ints((0, 0, 0)), _ints((0, 0, 0)), ctypes.c_int()
        _check(L.igg_grid_shape(h, nn, dd, oo, pp, ctypes.byref(ns)))
        self.n, self.dims, self.overlap = tuple(nn), tuple(dd), tuple(oo)
        self.periods, self.nsub = tuple(pp), ns.value
        self.nloc = self.n[0] * self.n[1] * self.n[2]

    # -- lifetime --------------------------------------------------------
    def finalize(self):
        """Fig. 1 finalize_global_grid."""
        if self._h:
            h, self._h = self._h, None
            _check(lib().igg_finalize_global_grid(h))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.finalize()

    def __del__(self):
        try:
            self.finalize()
        except Exception:
            pass

    def _handle(self):
        if not self._h:
            raise IggError(-4, "grid used after finalize")
        return self._h

    # -- queries ---------------------------------------------------------
    @property
    def shape(self):
        return (self.nsub, self.n[2], self.n[1], self.n[0])

    def global_size(self):
        """(nx_g(), ny_g(), nz_g())."""
        ng = _ints((0, 0, 0))
        _check(lib().igg_global_size(self._handle(), ng))
        return tuple(ng)

    def subdomain_info(self, sub: int):
        """dict(coords, left, right, offset) of subdomain `sub`."""
        c, l, r, o = (_ints((0, 0, 0)) for _ in range(4))
        _check(lib().igg_subdomain_info(self._handle(), int(sub), c, l, r, o))
        return {"coords": tuple(c), "left": tuple(l), "right": tuple(r), "offset": tuple(o)}

    def global_indices(self, sub: int):
        """Per axis, the global index of each local point of `sub`."""
        info = self.subdomain_info(sub)
        ng = self.global_size()
        out = []
        for d in range(3):
            g = torch.arange(self.n[d], dtype=torch.int64) + info["offset"][d]
            out.append((g % ng[d]) if self.periods[d] else g)
        return [t.numpy() for t in out]

    OPT_TMA = 1
    OPT_F64_EMU = 2
    OPT_FUSED_HALO = 3
    OPT_PHASE_TIMES = 4
    OPT_HIDE_HALO = 5

    def set_option(self, option: int, value: int):
        """igg_grid_set_option (OPT_TMA: 1 = TMA kernel for regular boxes)."""
        _check(lib().igg_grid_set_option(self._handle(), int(option), int(value)))

    def device_status(self, clear: bool = False) -> int:
        """Device error word of the pipelined kernels (0 = no error)."""
        st = ctypes.c_uint()
        _check(lib().igg_device_status(self._handle(), ctypes.byref(st), int(clear)))
        return st.value

    def phase_times(self):
        """igg_phase_times: (stencil-phase ms, rest-of-step ms, total ms,
        steps) summed over the steps recorded under OPT_PHASE_TIMES."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int()
        _check(lib().igg_phase_times(self._handle(), ms, ctypes.byref(n)))
        return ms[0], ms[1], ms[2], n.value

    def fixup_stats(self, clear: bool = False):
        """igg_fixup_stats: (row segments, points) left to the emulated FP64
        cell's fix-up launch so far."""
        c = (ctypes.c_ulonglong * 2)()
        _check(lib().igg_fixup_stats(self._handle(), c, int(clear)))
        return int(c[0]), int(c[1])

    def empty(self, dtype=torch.float64, device="cuda"):
        return torch.empty(self.shape, dtype=dtype, device=device)

    # -- hot path --------------------------------------------------------
    def update_halo(self, *fields, stream=None):
        """update_halo!(fields...): all fields must share one dtype."""
        if not fields:
            return
        dt = fields[0].dtype
        arr = (ctypes.c_void_p * len(fields))(*[_ptr(f, self.nsub * self.nloc, dt, "field").value
                                                for f in fields])
        _check(lib().igg_update_halo(self._handle(), arr, len(fields), dtype_code(dt), _stream(stream)))

    def update_halo_staggered(self, nf, *fields, stream=None):
        """update_halo! on staggered fields of local size nf = (nx, ny, nz),
        each within one point of the grid's size (igg_update_halo_staggered)."""
        if not fields:
            return
        dt = fields[0].dtype
        npts = self.nsub * int(nf[0]) * int(nf[1]) * int(nf[2])
        arr = (ctypes.c_void_p * len(fields))(*[_ptr(f, npts, dt, "field").value for f in fields])
        _check(lib().igg_update_halo_staggered(self._handle(), arr, len(fields), dtype_code(dt),
                                               _ints(nf), _stream(stream)))

    def update_halo_fields(self, fields, sizes, stream=None):
        """update_halo!(A...) on fields of possibly different staggered local
        sizes (sizes[i] = (nx, ny, nz) of fields[i]), one launch per dimension."""
        if not fields:
            return
        dt = fields[0].dtype
        ptrs = [_ptr(f, self.nsub * int(s[0]) * int(s[1]) * int(s[2]), dt, "field").value
                for f, s in zip(fields, sizes)]
        arr = (ctypes.c_void_p * len(fields))(*ptrs)
        flat = (ctypes.c_int * (3 * len(fields)))(*[int(v) for s in sizes for v in s])
        _check(lib().igg_update_halo_fields(self._handle(), arr, flat, len(fields), dtype_code(dt),
                                            _stream(stream)))

    def acoustic_fields(self, dtype=torch.float64):
        """Zeroed P, Vx, Vy, Vz of the staggered acoustic layout."""
        nx, ny, nz = self.n
        shp = [(nz, ny, nx), (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
        return [torch.zeros((self.nsub,) + s, dtype=dtype, device="cuda") for s in shp]

    def acoustic_step(self, P, Vx, Vy, Vz, rho, K, dt, dx, dy, dz, halo=True, stream=None):
        """One leapfrog step of staggered-grid acoustics (igg_acoustic_step)."""
        nx, ny, nz = self.n
        d = P.dtype
        ptrs = [_ptr(f, self.nsub * a * b * c, d, name) for f, (a, b, c), name in
                ((P, (nx, ny, nz), "P"), (Vx, (nx + 1, ny, nz), "Vx"), (Vy, (nx, ny + 1, nz), "Vy"),
                 (Vz, (nx, ny, nz + 1), "Vz"))]
        _check(lib().igg_acoustic_step(self._handle(), *ptrs, dtype_code(d), float(rho), float(K),
                                       float(dt), float(dx), float(dy), float(dz), int(bool(halo)),
                                       _stream(stream)))

    def gp_step(self, u, v, V, g, dt, dx, dy, dz, halo=True, stream=None):
        """One Gross-Pitaevskii step (igg_gp_step): u half, halo, v half, halo."""
        n = self.nsub * self.nloc
        d = u.dtype
        _check(lib().igg_gp_step(self._handle(), _ptr(u, n, d, "u"), _ptr(v, n, d, "v"),
                                 _ptr(V, n, d, "V"), dtype_code(d), float(g), float(dt), float(dx),
                                 float(dy), float(dz), int(bool(halo)), _stream(stream)))

    def step(self, T2, T, Ci, lam, dt, dx, dy, dz, stream=None):
        """Fig. 1 step! on every subdomain (inner points of T2)."""
        n = self.nsub * self.nloc
        d = T.dtype
        _check(lib().igg_step(self._handle(), _ptr(T2, n, d, "T2"), _ptr(T, n, d, "T"),
                              _ptr(Ci, n, d, "Ci"), dtype_code(d), float(lam), float(dt),
                              float(dx), float(dy), float(dz), _stream(stream)))

    def step_hidden(self, widths, T2, T, Ci, lam, dt, dx, dy, dz, stream=None):
        """@hide_communication widths { step!(T2, T, ...); update_halo!(T2) }."""
        n = self.nsub * self.nloc
        d = T.dtype
        _check(lib().igg_step_hidden(self._handle(), _ints(widths), _ptr(T2, n, d, "T2"),
                                     _ptr(T, n, d, "T"), _ptr(Ci, n, d, "Ci"), dtype_code(d),
                                     float(lam), float(dt), float(dx), float(dy), float(dz),
                                     _stream(stream)))

    def run(self, nt, T, T2, Ci, lam, dt, dx, dy, dz, widths=None, stream=None):
        """Fig. 1's time loop (graph-captured). Returns the tensor that holds
        the newest state: T for even nt, T2 for odd nt."""
        n = self.nsub * self.nloc
        d = T.dtype
        w = _ints(widths) if widths is not None else None
        _check(lib().igg_run(self._handle(), int(nt), w, _ptr(T, n, d, "T"), _ptr(T2, n, d, "T2"),
                             _ptr(Ci, n, d, "Ci"), dtype_code(d), float(lam), float(dt), float(dx),
                             float(dy), float(dz), _stream(stream)))
        return T if nt % 2 == 0 else T2

    def run_host(self, nt, T_host, Ci_host, T, T2, Ci, lam, dt, dx, dy, dz, widths=None,
                 stream=None):
        """Fig. 1's solver from host fields (igg_run_host): T_host (T0 in,
        the newest state out) and Ci_host are CPU tensors of the fields'
        shape, best page-locked; T, T2, Ci device buffers. Enqueued on the
        stream: synchronise it before reading T_host."""
        n = self.nsub * self.nloc
        d = T.dtype
        for name, h in (("T_host", T_host), ("Ci_host", Ci_host)):
            if not isinstance(h, torch.Tensor) or h.is_cuda or h.dtype != d or not h.is_contiguous() \
                    or h.numel() != n:
                raise ValueError(f"{name} must be a contiguous CPU tensor of {n} {d} elements")
        w = _ints(widths) if widths is not None else None
        _check(lib().igg_run_host(self._handle(), int(nt), w, ctypes.c_void_p(T_host.data_ptr()),
                                  ctypes.c_void_p(Ci_host.data_ptr()), _ptr(T, n, d, "T"),
                                  _ptr(T2, n, d, "T2"), _ptr(Ci, n, d, "Ci"), dtype_code(d),
                                  float(lam), float(dt), float(dx), float(dy), float(dz),
                                  _stream(stream)))


def bounds_status(clear: bool = False) -> int:
    """igg_bounds_status: DEV_ERR_BOUNDS when a bounds-checked kernel skipped
    an out-of-range access (always 0 in the release build)."""
    st = ctypes.c_uint(0)
    _check(lib().igg_bounds_status(ctypes.byref(st), int(clear)))
    return int(st.value)


def selftest_bounded_wait() -> int:
    """igg_selftest_bounded_wait: the device error bits recorded by a kernel
    whose bounded wait on an mbarrier that never completes runs out (expected
    DEV_ERR_TIMEOUT); about 2 s."""
    fn = lib().igg_selftest_bounded_wait
    fn.argtypes = [ctypes.POINTER(ctypes.c_uint)]
    fn.restype = ctypes.c_int
    st = ctypes.c_uint(0)
    _check(fn(ctypes.byref(st)))
    return int(st.value)


def reduce(op: int, a: torch.Tensor, b: torch.Tensor | None = None, out: torch.Tensor | None = None,
           stream=None):
    """FP64 reduction over all elements (RED_MAX, RED_SUM, RED_SUM_DIV,
    RED_SUM_SQDIFF). Returns a 1-element float64 device tensor."""
    n = a.numel()
    pa = _ptr(a, n, a.dtype, "a")
    pb = _ptr(b, n, a.dtype, "b") if b is not None else None
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=a.device)
    _check(lib().igg_reduce(int(op), pa, pb, n, dtype_code(a.dtype), ctypes.c_void_p(out.data_ptr()),
                            _stream(stream)))
    return out


def reduce_noalloc(op: int, a: torch.Tensor, b: torch.Tensor | None = None,
                   out: torch.Tensor | None = None, stream=None):
    """igg_reduce_noalloc: the FP64 reduction without any device allocation
    inside the library (partial sums in a fixed device array of the library).
    For callers that cannot allocate while they reduce; pass a preallocated
    `out` (1-element float64 device tensor) to allocate nothing at all.
    Calls that can overlap on the GPU share that array and must be ordered."""
    L = lib()
    fn = L.igg_reduce_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    n = a.numel()
    pa = _ptr(a, n, a.dtype, "a")
    pb = _ptr(b, n, a.dtype, "b") if b is not None else None
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=a.device)
    _check(fn(int(op), pa, pb, n, dtype_code(a.dtype), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


_batch_sigs_done = False


def _batch_sigs():
    global _batch_sigs_done
    if _batch_sigs_done:
        return lib()
    L = lib()
    P, I = ctypes.c_void_p, ctypes.c_int
    IP = ctypes.POINTER(ctypes.c_int)
    DP = ctypes.POINTER(ctypes.c_double)
    LLP = ctypes.POINTER(ctypes.c_longlong)
    L.igg_batch_create.argtypes = [I, IP, I, ctypes.POINTER(P)]
    L.igg_batch_destroy.argtypes = [P]
    L.igg_batch_layout.argtypes = [P, LLP, LLP]
    L.igg_batch_pitches.argtypes = [P, IP]
    L.igg_batch_set_coefs.argtypes = [P, DP, DP, DP, DP, DP]
    L.igg_batch_configure.argtypes = [P, I, I, I]
    L.igg_batch_get_config.argtypes = [P, IP, IP]
    L.igg_batch_step.argtypes = [P, P, P, P, P]
    L.igg_batch_run.argtypes = [P, I, P, P, P, P]
    L.igg_batch_autotune.argtypes = [P, P, P, P, I, P, IP, ctypes.POINTER(ctypes.c_float)]
    for n in ("igg_batch_create", "igg_batch_destroy", "igg_batch_layout", "igg_batch_pitches",
              "igg_batch_set_coefs",
              "igg_batch_configure", "igg_batch_get_config", "igg_batch_step", "igg_batch_run",
              "igg_batch_autotune"):
        getattr(L, n).restype = I
    _batch_sigs_done = True
    return L


class Batch:
    """Many independent problems of uneven sizes, packed in one buffer per
    field (problem b at element offset offsets[b], shape (nz, ny, nx) with
    rows of pitches[b] elements), advanced by one launch per step."""

    def __init__(self, sizes, dtype=torch.float32):
        L = _batch_sigs()
        self.sizes = [tuple(int(v) for v in s) for s in sizes]
        self.dtype = dtype
        flat = (ctypes.c_int * (3 * len(self.sizes)))(*[v for s in self.sizes for v in s])
        h = ctypes.c_void_p()
        _check(L.igg_batch_create(len(self.sizes), flat, dtype_code(dtype), ctypes.byref(h)))
        self._h = h
        offs = (ctypes.c_longlong * len(self.sizes))()
        tot = ctypes.c_longlong()
        _check(L.igg_batch_layout(h, offs, ctypes.byref(tot)))
        self.offsets = list(offs)
        self.total = tot.value
        pit = (ctypes.c_int * len(self.sizes))()
        _check(L.igg_batch_pitches(h, pit))
        self.pitches = list(pit)

    def destroy(self):
        if self._h:
            h, self._h = self._h, None
            _check(_batch_sigs().igg_batch_destroy(h))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def empty(self, device="cuda"):
        return torch.empty(self.total, dtype=self.dtype, device=device)

    def view(self, field: torch.Tensor, b: int) -> torch.Tensor:
        """Problem b of a batch field as a (nz, ny, nx) view (rows of pitch_b)."""
        nx, ny, nz = self.sizes[b]
        o, pt = self.offsets[b], self.pitches[b]
        return field[o:o + pt * ny * nz].view(nz, ny, pt)[:, :, :nx]

    def set_coefs(self, lam, dt, dx, dy, dz):
        n = len(self.sizes)
        arrs = [(ctypes.c_double * n)(*[float(v) for v in a]) for a in (lam, dt, dx, dy, dz)]
        _check(_batch_sigs().igg_batch_set_coefs(self._h, *arrs))

    def configure(self, variant=3, zb=32, ctas_per_sm=0):
        _check(_batch_sigs().igg_batch_configure(self._h, int(variant), int(zb), int(ctas_per_sm)))

    def config(self):
        cfg = _ints((0, 0, 0))
        nt = ctypes.c_int()
        _check(_batch_sigs().igg_batch_get_config(self._h, cfg, ctypes.byref(nt)))
        return {"variant": cfg[0], "zb": cfg[1], "ctas_per_sm": cfg[2], "ntiles": nt.value}

    def _p(self, t, name):
        return _ptr(t, self.total, self.dtype, name)

    def step(self, T2, T, Ci, stream=None):
        _check(_batch_sigs().igg_batch_step(self._h, self._p(T2, "T2"), self._p(T, "T"), self._p(Ci, "Ci"),
                                            _stream(stream)))

    def run(self, nt, T, T2, Ci, stream=None):
        """nt steps (CUDA graph); returns T for even nt, T2 for odd nt."""
        _check(_batch_sigs().igg_batch_run(self._h, int(nt), self._p(T, "T"), self._p(T2, "T2"),
                                           self._p(Ci, "Ci"), _stream(stream)))
        return T if nt % 2 == 0 else T2

    def autotune(self, T2, T, Ci, reps=3, stream=None):
        """Time every (tile shape, z depth, CTAs/SM) candidate on these fields
        and keep the fastest. Writes T2's inner points; synchronises. The
        choice is cached per (GPU name, dtype, problem sizes), in the process
        and in the file named by IGG_AUTOTUNE_CACHE: a cached key applies
        its tiling without timing (T2 untouched); reps < 0 re-tunes."""
        cfg = _ints((0, 0, 0))
        ms = ctypes.c_float()
        _check(_batch_sigs().igg_batch_autotune(self._h, self._p(T2, "T2"), self._p(T, "T"), self._p(Ci, "Ci"),
                                                int(reps), _stream(stream), cfg, ctypes.byref(ms)))
        return {"variant": cfg[0], "zb": cfg[1], "ctas_per_sm": cfg[2], "ms": ms.value}
