"""torch.autograd.Function around the library's checkpointed forward and
adjoint runs: gradients of any scalar function of T_nt with respect to Ci
and T0 (the differentiated form of Fig. 1's solver; dt held fixed).

Forward keeps one checkpoint every `every` steps (about sqrt(nt) by default);
backward recomputes each segment from its checkpoint and runs the adjoint
kernel backward in time. All compute runs in libigg.so; this module only
allocates the buffers (through torch) and passes pointers.
"""
from __future__ import annotations

import ctypes
import math

import torch

from .igg import Grid, _check, _stream, dtype_code, lib

_sigs = False


def _L():
    global _sigs
    L = lib()
    if not _sigs:
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.igg_checkpoint_slots.argtypes = [I, I]
        L.igg_checkpoint_slots.restype = I
        L.igg_forward_checkpointed.argtypes = [P, I, I, P, P, I, D, D, D, D, D, P, P, P, P]
        L.igg_forward_checkpointed.restype = I
        L.igg_adjoint_checkpointed.argtypes = [P, I, I, P, P, P, I, D, D, D, D, D, P, P, P, P, P]
        L.igg_adjoint_checkpointed.restype = I
        L.igg_adjoint_step.argtypes = [P, P, P, P, P, P, I, D, D, D, D, D, P]
        L.igg_adjoint_step.restype = I
        L.igg_update_halo_adjoint.argtypes = [P, P, I, P]
        L.igg_update_halo_adjoint.restype = I
        L.igg_residual.argtypes = [P, P, P, ctypes.c_size_t, I, P]
        L.igg_residual.restype = I
        _sigs = True
    return L


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def default_every(nt: int) -> int:
    return max(1, int(round(math.sqrt(nt))))


def checkpoint_slots(nt: int, every: int) -> int:
    n = _L().igg_checkpoint_slots(int(nt), int(every))
    _check(min(n, 0))
    return n


def adjoint_step(grid: Grid, lam_out, lam_in, Tn, Ci, gCi, lam, dt, dx, dy, dz, stream=None):
    """One backward step (igg_adjoint_step); gCi is a float64 tensor."""
    _check(_L().igg_adjoint_step(grid._handle(), _p(lam_out), _p(lam_in), _p(Tn), _p(Ci), _p(gCi),
                                 dtype_code(Tn.dtype), float(lam), float(dt), float(dx), float(dy),
                                 float(dz), _stream(stream)))


def update_halo_adjoint(grid: Grid, lam, stream=None):
    """The transpose of the halo update, in place (igg_update_halo_adjoint)."""
    _check(_L().igg_update_halo_adjoint(grid._handle(), _p(lam), dtype_code(lam.dtype),
                                        _stream(stream)))
    return lam


def residual(a, b, out=None, stream=None):
    """a - b (igg_residual)."""
    out = torch.empty_like(a) if out is None else out
    _check(_L().igg_residual(_p(out), _p(a), _p(b), a.numel(), dtype_code(a.dtype), _stream(stream)))
    return out


def forward_checkpointed(grid, nt, every, T0, Ci, lam, dt, dx, dy, dz):
    """(T_nt, checkpoints) of nt steps from T0."""
    n = grid.nsub * grid.nloc
    slots = checkpoint_slots(nt, every)
    ckpt = torch.empty((slots, n), dtype=T0.dtype, device=T0.device)
    work = torch.empty((2, n), dtype=T0.dtype, device=T0.device)
    T_out = torch.empty_like(T0)
    _check(_L().igg_forward_checkpointed(grid._handle(), int(nt), int(every), _p(T0), _p(Ci),
                                         dtype_code(T0.dtype), float(lam), float(dt), float(dx),
                                         float(dy), float(dz), _p(ckpt), _p(work), _p(T_out),
                                         _stream(None)))
    return T_out, ckpt


def adjoint_checkpointed(grid, nt, every, ckpt, Ci, lam_nt, lam, dt, dx, dy, dz):
    """(dJ/dT0 in the field dtype, dJ/dCi in float64) from dJ/dT_nt."""
    n = grid.nsub * grid.nloc
    seg = torch.empty((max(every - 1, 1), n), dtype=Ci.dtype, device=Ci.device)
    work = torch.empty((2, n), dtype=Ci.dtype, device=Ci.device)
    gT0 = torch.empty_like(Ci)
    gCi = torch.empty(Ci.shape, dtype=torch.float64, device=Ci.device)
    lam_nt = lam_nt.contiguous()
    _check(_L().igg_adjoint_checkpointed(grid._handle(), int(nt), int(every), _p(ckpt), _p(Ci),
                                         _p(lam_nt), dtype_code(Ci.dtype), float(lam), float(dt),
                                         float(dx), float(dy), float(dz), _p(seg), _p(work), _p(gT0),
                                         _p(gCi), _stream(None)))
    return gT0, gCi


class DiffusionSolve(torch.autograd.Function):
    """T_nt = nt steps of Fig. 1's loop from (T0, Ci) on a 3-D grid of any
    topology (each step: step!, then update_halo!); differentiable in T0 and
    Ci (per entry of the decomposed fields)."""

    @staticmethod
    def forward(ctx, T0, Ci, grid, nt, lam, dt, dx, dy, dz, every):
        T0 = T0.contiguous()
        Ci = Ci.contiguous()
        T_nt, ckpt = forward_checkpointed(grid, nt, every, T0, Ci, lam, dt, dx, dy, dz)
        ctx.save_for_backward(Ci, ckpt)
        ctx.args = (grid, nt, every, lam, dt, dx, dy, dz)
        return T_nt

    @staticmethod
    def backward(ctx, grad_T):
        Ci, ckpt = ctx.saved_tensors
        grid, nt, every, lam, dt, dx, dy, dz = ctx.args
        gT0, gCi = adjoint_checkpointed(grid, nt, every, ckpt, Ci, grad_T.to(Ci.dtype), lam, dt, dx, dy, dz)
        return gT0, gCi.to(Ci.dtype), None, None, None, None, None, None, None, None


def solve(T0, Ci, grid, nt, lam, dt, dx, dy, dz, every=None):
    """Differentiable nt-step solve (checkpoint every ~sqrt(nt) steps)."""
    every = default_every(nt) if every is None else int(every)
    return DiffusionSolve.apply(T0, Ci, grid, int(nt), float(lam), float(dt), float(dx), float(dy),
                                float(dz), every)
