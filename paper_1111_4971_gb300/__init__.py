"""GB300 open-rectangular-pipe Poisson solver (Ryne, FFT-based mixed convolutions
and correlations; integrated Green function).

Thin Python layer over the C ABI in ``include/pipe_poisson.h``: PyTorch
supplies device memory and streams, every arithmetic step runs in the CUDA
kernels of ``libpipepoisson.so``.

    solver = PipeSolver(geometry, grid, igf=True, dtype=torch.float32)
    phi = solver.solve(rho)                 # rho: cuda tensor [nx, ny, nz]
    phi = PipePoissonFunction.apply(rho, solver)   # differentiable
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import PipeError, PipeGeometry, PipeGrid, check

__all__ = ["PipeSolver", "PipePoissonFunction", "CICDeposit", "solve_batched", "batch_status",
           "batch_inject_fault", "batch_plan_info", "batch_select", "batch_side_streams",
           "batch_select_streams", "batch_grouped", "batch_select_groups", "PipeError", "field_energy"]


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _spans(geometry, grid) -> bool:
    """The mesh spans the pipe with integer 2*x0/hx, 2*y0/hy (the octant form)."""
    def near_int(x):
        return abs(x - round(x)) <= 1e-9 * max(1.0, abs(x))
    return (abs(grid.nx * grid.hx - geometry.a) <= 1e-12 * geometry.a
            and abs(grid.ny * grid.hy - geometry.b) <= 1e-12 * geometry.b
            and near_int(2.0 * geometry.x0 / grid.hx) and near_int(2.0 * geometry.y0 / grid.hy))


class PipeSolver:
    """One Green-function setup (Sec. 5: computed once, reused) and its solves.

    ``geometry``: object with a, b, x0, y0, modes_m, modes_n.
    ``grid``: object with nx, ny, nz, hx, hy, hz.
    ``dtype``: torch.float32 or torch.float64 (the solve's arithmetic type).
    ``banded``: None for the full solve (Eq. 10); an int n >= 0 for the banded
    reduction of Sec. 5 (Eq. 17-18) keeping source planes within n of each
    output plane.
    ``fp16_spectra``: with dtype float32, keep the z half-spectrum between the
    kernels as complex FP16 with per-slab scales (PIPE_F32_C16; about 1e-3
    relative error, cell-centred meshes).
    """

    def __init__(self, geometry, grid, igf: bool = True, dtype=torch.float32, *,
                 free_space: bool = False, self_value: float = 0.0, banded: int | None = None,
                 fp16_spectra: bool = False, device=None):
        self.lib = _lib.load()
        self.dtype = dtype
        self.shape = (int(grid.nx), int(grid.ny), int(grid.nz))
        self.grid = grid
        self.geometry = geometry
        self.igf = bool(igf)
        self.free_space = free_space
        self.banded = banded
        # a mesh that does not span the pipe at integer correlation shifts
        # (a transverse window) uses the general four-table form
        self.general = (not free_space) and not _spans(geometry, grid)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if fp16_spectra and dtype != torch.float32:
            raise ValueError("fp16_spectra needs dtype torch.float32")
        code = _lib.PIPE_F64 if dtype == torch.float64 else \
            (_lib.PIPE_F32_C16 if fp16_spectra else _lib.PIPE_F32)
        self.fp16_spectra = bool(fp16_spectra)
        g = PipeGrid(int(grid.nx), int(grid.ny), int(grid.nz), float(grid.hx), float(grid.hy),
                     float(grid.hz), code)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if free_space:
                st = self.lib.pipe_free_space_setup(ctypes.byref(g), float(self_value), ctypes.byref(h))
            else:
                geo = PipeGeometry(float(geometry.a), float(geometry.b), float(geometry.x0),
                                   float(geometry.y0), int(geometry.modes_m), int(geometry.modes_n))
                if banded is None:
                    st = self.lib.pipe_green_setup(ctypes.byref(geo), ctypes.byref(g), int(bool(igf)),
                                                   ctypes.byref(h))
                else:
                    st = self.lib.pipe_banded_setup(ctypes.byref(geo), ctypes.byref(g), int(bool(igf)),
                                                    int(banded), ctypes.byref(h))
        check(st, "pipe_free_space_setup" if free_space else
              ("pipe_green_setup" if banded is None else "pipe_banded_setup"))
        self.handle = h

    # -- helpers ---------------------------------------------------------
    def _check_field(self, t: torch.Tensor, name: str):
        if t.dtype != self.dtype or t.device != self.device or tuple(t.shape) != self.shape \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of shape "
                             f"{self.shape} on {self.device}")

    def empty(self):
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    # -- solves ----------------------------------------------------------
    def solve(self, rho: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        self._check_field(rho, "rho")
        out = self.empty() if out is None else out
        self._check_field(out, "out")
        check(self.lib.pipe_poisson_solve(self.handle, _ptr(rho), _ptr(out), _stream_ptr(stream)),
              "pipe_poisson_solve")
        return out

    def adjoint(self, dphi: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        self._check_field(dphi, "dphi")
        out = self.empty() if out is None else out
        self._check_field(out, "out")
        check(self.lib.pipe_poisson_adjoint(self.handle, _ptr(dphi), _ptr(out), _stream_ptr(stream)),
              "pipe_poisson_adjoint")
        return out

    def solve_host(self, rho_host: torch.Tensor, phi_host: torch.Tensor | None = None, stream=None):
        """Host arrays in, host array out (copies inside the call)."""
        if rho_host.device.type != "cpu" or rho_host.dtype != self.dtype or not rho_host.is_contiguous():
            raise ValueError("rho_host must be a contiguous CPU tensor of the solver dtype")
        if phi_host is None:
            phi_host = torch.empty(self.shape, dtype=self.dtype, pin_memory=True)
        check(self.lib.pipe_poisson_solve_host(self.handle, _ptr(rho_host), _ptr(phi_host),
                                               _stream_ptr(stream)), "pipe_poisson_solve_host")
        return phi_host

    def solve_host_stream(self, rho_hosts, phi_hosts=None, stream=None):
        """A sequence of host fields in, host results out, with the copies of
        neighbouring solves overlapped with the compute (pinned tensors)."""
        n = len(rho_hosts)
        for r in rho_hosts:
            if r.device.type != "cpu" or r.dtype != self.dtype or not r.is_contiguous() \
                    or tuple(r.shape) != self.shape:
                raise ValueError("rho_hosts must be contiguous CPU tensors of the solver dtype and shape")
        if phi_hosts is None:
            phi_hosts = [torch.empty(self.shape, dtype=self.dtype, pin_memory=True) for _ in range(n)]
        rs = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rho_hosts])
        ps = (ctypes.c_void_p * n)(*[p.data_ptr() for p in phi_hosts])
        check(self.lib.pipe_poisson_solve_host_stream(self.handle, rs, ps, n, _stream_ptr(stream)),
              "pipe_poisson_solve_host_stream")
        return phi_hosts

    def green_spectrum(self):
        import numpy as np
        nx, ny, nz = self.shape
        if self.general:
            # four complex tables [cc, cr, rc, rr][kz][ky][kx] on the doubled transverse grid
            raw = np.empty((4, nz + 1, 2 * ny, 2 * nx, 2), dtype=np.float64)
            check(self.lib.pipe_green_spectrum(self.handle, raw.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               raw.size), "pipe_green_spectrum")
            return raw[..., 0] + 1j * raw[..., 1]
        planes = nz + 1 if self.banded is None else self.banded + 1
        out = np.empty((planes, ny + 1, nx + 1), dtype=np.float64)
        check(self.lib.pipe_green_spectrum(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           out.size), "pipe_green_spectrum")
        return out

    def spectrum_buffer(self):
        nx, ny, nz = self.shape
        cdt = torch.complex128 if self.dtype == torch.float64 else torch.complex64
        return torch.empty((nz + 1, nx, ny), dtype=cdt, device=self.device)

    def stage_z_forward(self, rho, spec, adjoint=False, stream=None):
        check(self.lib.pipe_stage_z_forward(self.handle, _ptr(rho), _ptr(spec), int(adjoint),
                                            _stream_ptr(stream)), "pipe_stage_z_forward")
        return spec

    def stage_transverse(self, spec, adjoint=False, stream=None):
        check(self.lib.pipe_stage_transverse(self.handle, _ptr(spec), int(adjoint), _stream_ptr(stream)),
              "pipe_stage_transverse")
        return spec

    def stage_z_inverse(self, spec, phi, adjoint=False, stream=None):
        check(self.lib.pipe_stage_z_inverse(self.handle, _ptr(spec), _ptr(phi), int(adjoint),
                                            _stream_ptr(stream)), "pipe_stage_z_inverse")
        return phi

    # -- the mode-space form (plan t_kind 3) -----------------------------
    def mode_layout(self):
        """(mx, mxp, myp, fold, xblocks) of the mode-space form (pipe_mode_layout)."""
        v = [ctypes.c_int() for _ in range(5)]
        check(self.lib.pipe_mode_layout(self.handle, *[ctypes.byref(x) for x in v]), "pipe_mode_layout")
        return tuple(x.value for x in v)

    def mode_spectrum(self):
        """FP64 kernel spectra [mxp*myp, nz+1] of the mode columns (pipe_mode_spectrum)."""
        import numpy as np
        _, mxp, myp, _, _ = self.mode_layout()
        out = np.empty((mxp * myp, self.shape[2] + 1), dtype=np.float64)
        check(self.lib.pipe_mode_spectrum(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          out.size), "pipe_mode_spectrum")
        return out

    def mode_buffers(self):
        """Empty (part, psi) device arrays for the mode-space stages."""
        _, mxp, myp, _, xb = self.mode_layout()
        nz = self.shape[2]
        return (torch.empty((xb, mxp * myp, nz), dtype=self.dtype, device=self.device),
                torch.empty((mxp * myp, nz), dtype=self.dtype, device=self.device))

    def stage_modes(self, stage: int, inp: torch.Tensor, out: torch.Tensor, stream=None):
        """One stage of the mode-space form: 0 rho -> part, 1 part -> psi, 2 psi -> phi."""
        check(self.lib.pipe_stage_modes(self.handle, int(stage), _ptr(inp), _ptr(out), _stream_ptr(stream)),
              "pipe_stage_modes")
        return out

    def autotune(self, stream=None):
        check(self.lib.pipe_autotune(self.handle, _stream_ptr(stream)), "pipe_autotune")
        return self.plan

    @property
    def plan(self):
        z, zp, h, t, k = (ctypes.c_int() for _ in range(5))
        check(self.lib.pipe_get_plan(self.handle, ctypes.byref(z), ctypes.byref(zp), ctypes.byref(h),
                                     ctypes.byref(t), ctypes.byref(k)), "pipe_get_plan")
        return {"z_warps": z.value, "z_pipe": zp.value, "t_h": h.value, "t_threads": t.value,
                "t_kind": k.value}

    def status(self):
        """The handle's device error word, read and cleared (pipe_status)."""
        st = self.lib.pipe_status(self.handle)
        if st not in (_lib.PIPE_OK, _lib.PIPE_ETIMEOUT):
            check(st, "pipe_status")
        return st

    def inject_stage_fault(self, drop_copy=0, poll_limit=4096):
        """Failure-detection test hook (pipe_inject_stage_fault)."""
        check(self.lib.pipe_inject_stage_fault(self.handle, int(drop_copy), int(poll_limit)),
              "pipe_inject_stage_fault")

    def set_plan(self, z_warps=8, z_pipe=1, t_h=1, t_threads=256, t_kind=0):
        check(self.lib.pipe_set_plan(self.handle, int(z_warps), int(z_pipe), int(t_h), int(t_threads),
                                     int(t_kind)), "pipe_set_plan")

    def electric_field(self, phi: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """E = -grad phi on the mesh, shape (3, nx, ny, nz)."""
        self._check_field(phi, "phi")
        out = torch.empty((3,) + self.shape, dtype=self.dtype, device=self.device) if out is None else out
        check(self.lib.pipe_electric_field(self.handle, _ptr(phi), _ptr(out), _stream_ptr(stream)),
              "pipe_electric_field")
        return out

    def cic_deposit(self, xyz: torch.Tensor, charge: float, out: torch.Tensor | None = None,
                    stream=None):
        out = torch.zeros(self.shape, dtype=self.dtype, device=self.device) if out is None else out
        xyz = xyz.contiguous()
        check(self.lib.pipe_cic_deposit(self.handle, _ptr(xyz), xyz.shape[0], float(charge), _ptr(out),
                                        _stream_ptr(stream)), "pipe_cic_deposit")
        return out

    def cic_gather_grad(self, xyz: torch.Tensor, charge: float, grad_rho: torch.Tensor, stream=None):
        out = torch.empty_like(xyz)
        check(self.lib.pipe_cic_gather_grad(self.handle, _ptr(xyz), xyz.shape[0], float(charge),
                                            _ptr(grad_rho.contiguous()), _ptr(out), _stream_ptr(stream)),
              "pipe_cic_gather_grad")
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.pipe_green_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(solvers, rhos, phis, stream=None):
    """n independent solves: a persistent launch over a work list, with the
    largest solves possibly left to single-solve launches (pipe_poisson_solve_batched)."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    rs = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    ps = (ctypes.c_void_p * n)(*[p.data_ptr() for p in phis])
    check(lib.pipe_poisson_solve_batched(hs, rs, ps, n, _stream_ptr(stream)), "pipe_poisson_solve_batched")
    return phis


def batch_status(solvers):
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    return lib.pipe_batch_status(hs, n)


def batch_side_streams(solvers):
    """Side streams (0, 2 or 3) the tuned plan deals the single-solve launches to."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    k = ctypes.c_int(0)
    check(lib.pipe_batch_side_streams(hs, n, ctypes.byref(k)), "pipe_batch_side_streams")
    return k.value


def batch_grouped(solvers, with_groups=False):
    """Solves the tuned batched call runs in mode-form groups (pipe_batch_grouped);
    with_groups: (solves, groups)."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    k, g = ctypes.c_int(-1), ctypes.c_int(-1)
    check(lib.pipe_batch_grouped(hs, n, ctypes.byref(k), ctypes.byref(g)), "pipe_batch_grouped")
    return (k.value, g.value) if with_groups else k.value


def batch_select_groups(solvers, on):
    """Run the mode-form groups together (True) or solve by solve (pipe_batch_select_groups)."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    check(lib.pipe_batch_select_groups(hs, n, 1 if on else 0), "pipe_batch_select_groups")


def batch_select_streams(solvers, nside):
    """Override the tuned number of side streams (0, 2 or 3) for this set."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    check(lib.pipe_batch_select_streams(hs, n, int(nside)), "pipe_batch_select_streams")


def batch_plan_info(solvers):
    """(solves in the persistent launch, work-list order) chosen for this set."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    k, o = ctypes.c_int(0), ctypes.c_int(0)
    check(lib.pipe_batch_plan_info(hs, n, ctypes.byref(k), ctypes.byref(o)), "pipe_batch_plan_info")
    return k.value, o.value


def batch_select(solvers, variant: int, order: int):
    """Override the tuned split (variant 0: every solve persistent) and work-list order."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    check(lib.pipe_batch_select(hs, n, int(variant), int(order)), "pipe_batch_select")


def batch_inject_fault(solvers, drop_stage: int, spin_limit: int):
    """Test hook: the next batched call with these solvers drops one stage."""
    lib = _lib.load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    check(lib.pipe_batch_inject_fault(hs, n, int(drop_stage), int(spin_limit)), "pipe_batch_inject_fault")


class PipePoissonFunction(torch.autograd.Function):
    """phi = A rho with backward g -> A^T g through the hand-written adjoint."""

    @staticmethod
    def forward(ctx, rho, solver):
        ctx.solver = solver
        return solver.solve(rho.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.solver.adjoint(g.contiguous()), None


class CICDeposit(torch.autograd.Function):
    """rho = CIC(xyz) on the solver's mesh; backward gives d/dxyz through the
    derivative of the trilinear weights."""

    @staticmethod
    def forward(ctx, xyz, solver, charge):
        xyz = xyz.contiguous()
        ctx.save_for_backward(xyz)
        ctx.solver = solver
        ctx.charge = charge
        return solver.cic_deposit(xyz, charge)

    @staticmethod
    def backward(ctx, g):
        (xyz,) = ctx.saved_tensors
        return ctx.solver.cic_gather_grad(xyz, ctx.charge, g.contiguous()), None, None


def field_energy(rho: torch.Tensor, phi: torch.Tensor) -> torch.Tensor:
    """W = 1/2 sum rho phi."""
    return 0.5 * (rho * phi).sum()
