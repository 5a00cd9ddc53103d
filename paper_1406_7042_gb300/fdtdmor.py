"""Thin ctypes binding of the C ABI in include/fdtdmor.h.

Argument marshalling only: every step of the method runs in libfdtdmor.so.
Device memory for the library's handles comes from PyTorch's caching
allocator (installed through fdtd_set_allocator); u, y and other caller
buffers are torch tensors passed by pointer on the current torch stream.
If the library is missing this module raises on first use; there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import sys
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FDTDMOR_CHECKED=1 loads the checked build (paper_1406_7042_gb300.build with
# checked=True): a synchronisation after every launch, no CUDA graphs, index
# checks of the port lists; for debugging, not for timing.
LIB_PATH = os.path.join(_HERE, "libfdtdmor_checked.so" if os.environ.get("FDTDMOR_CHECKED") == "1"
                        else "libfdtdmor.so")

FDTD_OK, FDTD_EINVAL, FDTD_ENOMEM, FDTD_ECUDA, FDTD_ENOCONV, FDTD_EUNSTABLE, FDTD_ETIMEOUT = range(7)
FDTD_F64, FDTD_F32 = 0, 1
STATUS_NAMES = {0: "FDTD_OK", 1: "FDTD_EINVAL", 2: "FDTD_ENOMEM", 3: "FDTD_ECUDA",
                4: "FDTD_ENOCONV", 5: "FDTD_EUNSTABLE", 6: "FDTD_ETIMEOUT"}


class FdtdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.POINTER(C.c_double)), ("dy", C.POINTER(C.c_double)),
                ("dz", C.POINTER(C.c_double)), ("nmat", C.c_int),
                ("eps_r", C.POINTER(C.c_double)), ("mu_r", C.POINTER(C.c_double)),
                ("sig_e", C.POINTER(C.c_double)), ("sig_m", C.POINTER(C.c_double)),
                ("pec", C.POINTER(C.c_uint8)), ("mat_id", C.POINTER(C.c_uint16)),
                ("prec", C.c_int)]


class PortDesc(C.Structure):
    _fields_ = [("comp", C.c_int), ("n", C.c_int64), ("cell", C.POINTER(C.c_int64)),
                ("w", C.POINTER(C.c_double))]


class MorOpts(C.Structure):
    _fields_ = [("q", C.c_int), ("L", C.c_int), ("M", C.c_double), ("fmax", C.c_double),
                ("dt0", C.c_double), ("include_center", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("defl_tol", C.c_double), ("orth", C.c_int), ("solver", C.c_int)]


MOR_ORTH = {"native": 0, "tf32": 1, "bf16": 2}
MOR_GRAM = {"native": 0, "tf32": 1, "bf16": 2, "tf32x3": 3, "bf16x3": 4}
MOR_SOLVER = {"auto": 0, "cgs": 1, "bicgstab": 2, "cocg": 3}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
_alloc_cbs = None
_live = None  # weak set of open handles, closed at interpreter exit


def _close_all():
    if _live is not None:
        for h in list(_live):
            try:
                h.close()
            except Exception:
                pass


def _track(obj):
    global _live
    import atexit
    import weakref
    if _live is None:
        _live = weakref.WeakSet()
        atexit.register(_close_all)
    _live.add(obj)

# (name, restype, argtypes)
_SIGS = [
    ("fdtd_set_allocator", C.c_int, [ALLOC_FN, FREE_FN]),
    ("fdtd_last_error", C.c_char_p, []),
    ("fdtd_grid_create", C.c_int, [C.POINTER(GridDesc), C.c_int, C.POINTER(PortDesc), C.c_int,
                                   C.POINTER(PortDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("fdtd_grid_destroy", C.c_int, [C.c_void_p]),
    ("fdtd_cfl_dt", C.c_double, [C.c_void_p]),
    ("fdtd_step", C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                            C.c_void_p]),
    ("fdtd_step_host", C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p]),
    ("fdtd_fields_get", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("fdtd_fields_set", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("fdtd_planes_get", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    ("fdtd_planes_set", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    ("fdtd_launch_count", C.c_int64, [C.c_int]),
    ("fdtd_edge_props_get", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("fdtd_check", C.c_int, [C.c_void_p, C.c_void_p]),
    ("fdtd_dft", C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                           C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    ("fdtd_sparams", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_int,
                               C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    ("fdtd_resonances", C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                  C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.c_void_p]),
    ("fdtd_grid_set_kernel", C.c_int, [C.c_void_p, C.c_int]),
    ("fdtd_grid_set_watchdog", C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int]),
    ("fdtd_grid_set_wait_limit", C.c_int, [C.c_void_p, C.c_longlong]),
    ("fdtd_grid_autotune", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.c_void_p]),
    ("fdtd_step_batched", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double), C.c_int64,
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    ("fdtd_grid_set_materials", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_uint8),
                                          C.c_void_p]),
    ("fdtd_adjoint", C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                               C.c_void_p, C.c_void_p]),
    ("mor_opts_default", C.c_int, [C.POINTER(MorOpts)]),
    ("mor_gram", C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                           C.c_void_p, C.c_void_p, C.c_void_p]),
    ("mor_schur_apply", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    ("mor_shifted_solve", C.c_int, [C.c_void_p, C.POINTER(MorOpts), C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]),
    ("mor_build_basis", C.c_int, [C.c_void_p, C.POINTER(MorOpts), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("mor_basis_info", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_double)]),
    ("mor_basis_get", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("mor_basis_destroy", C.c_int, [C.c_void_p]),
    ("mor_build_basis_batched", C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(MorOpts), C.c_void_p,
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
    ("mor_project", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("mor_perturb", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_int), C.c_void_p]),
    ("mor_run", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("mor_model_get", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.c_void_p]),
    ("mor_model_destroy", C.c_int, [C.c_void_p]),
    ("mor_model_save", C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p]),
    ("mor_model_load", C.c_int, [C.c_char_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("mor_gradient", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    ("mor_compare", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                              C.POINTER(C.c_double), C.c_void_p]),
    ("mor_compare_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                      C.c_int, C.POINTER(C.c_double), C.c_void_p]),
]


def declared_symbols() -> List[str]:
    """Function names declared in include/fdtdmor.h (parsed from the header)."""
    import re
    hdr = open(os.path.join(_HERE, "..", "include", "fdtdmor.h")).read()
    return sorted(set(re.findall(r"FDTD_API\s+[\w\s\*]+?\b((?:fdtd|mor)_\w+)\s*\(", hdr)))


def lib(install_allocator: bool = True):
    """Load libfdtdmor.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FdtdError(FDTD_ECUDA, f"{LIB_PATH} not built: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
        if install_allocator:
            _install_torch_allocator()
    return _lib


def _install_torch_allocator():
    global _alloc_cbs
    import torch
    if not torch.cuda.is_available():
        return

    def _alloc(nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:  # out of memory -> NULL, the library reports FDTD_ENOMEM
            return None

    def _free(ptr, stream):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    _alloc_cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _lib.fdtd_set_allocator(*_alloc_cbs)


def check(status: int):
    if status != FDTD_OK:
        raise FdtdError(status, lib().fdtd_last_error().decode(errors="replace"))


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dptr(t) -> Optional[int]:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensor must be CUDA and contiguous"
    return int(t.data_ptr())


def launch_count(reset: bool = False) -> int:
    return int(lib().fdtd_launch_count(1 if reset else 0))


class Grid:
    """Owns an fdtd_grid handle built from a workloads.GridSpec."""

    def __init__(self, spec, prec: str = "f32", stream=None):
        import torch
        self.spec = spec
        self.prec = prec
        self.dtype = torch.float64 if prec == "f64" else torch.float32
        self.np_dtype = np.float64 if prec == "f64" else np.float32
        L = lib()
        keep = []

        def arr(a, ct, dt):
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(ct))

        d = GridDesc()
        d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
        d.dx = arr(spec.dx, C.c_double, np.float64)
        d.dy = arr(spec.dy, C.c_double, np.float64)
        d.dz = arr(spec.dz, C.c_double, np.float64)
        d.nmat = spec.nmat
        d.eps_r = arr(spec.eps_r, C.c_double, np.float64)
        d.mu_r = arr(spec.mu_r, C.c_double, np.float64)
        d.sig_e = arr(spec.sig_e, C.c_double, np.float64)
        d.sig_m = arr(spec.sig_m, C.c_double, np.float64)
        d.pec = arr(spec.pec, C.c_uint8, np.uint8)
        d.mat_id = arr(spec.mat_id, C.c_uint16, np.uint16)
        d.prec = FDTD_F64 if prec == "f64" else FDTD_F32

        def ports(lst):
            P = (PortDesc * max(1, len(lst)))()
            for n, p in enumerate(lst):
                cells = (np.asarray(p.k, np.int64) * spec.ny + np.asarray(p.j, np.int64)) * spec.nx \
                    + np.asarray(p.i, np.int64)
                P[n].comp = int(p.comp)
                P[n].n = int(cells.size)
                P[n].cell = arr(cells, C.c_int64, np.int64)
                P[n].w = arr(p.w, C.c_double, np.float64)
            return P

        P = ports(spec.ports)
        Q = ports(spec.probes)
        h = C.c_void_p()
        check(L.fdtd_grid_create(C.byref(d), len(spec.ports), P, len(spec.probes), Q,
                                 _stream_ptr(stream), C.byref(h)))
        self.h = h
        self.m = len(spec.ports)
        self.p = len(spec.probes)
        _track(self)

    def close(self):
        if getattr(self, "h", None):
            lib().fdtd_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None):
        """Raise if a bounded device wait of an earlier step gave up
        (FDTD_ETIMEOUT) or the field watchdog fired (FDTD_EUNSTABLE)."""
        check(lib().fdtd_check(self.h, _stream_ptr(stream)))

    def set_watchdog(self, enable: bool = True, growth: float = 0.0, sync: bool = False):
        """Field watchdog of step(): NaN/Inf always (when enabled); with
        growth > 0 also energy growth of source-free calls; sync makes step()
        raise FDTD_EUNSTABLE itself."""
        check(lib().fdtd_grid_set_watchdog(self.h, 1 if enable else 0, float(growth), 1 if sync else 0))

    def set_wait_limit(self, polls: int = -1):
        """Polls of the dataflow form's counter waits before they give up (-1: default)."""
        check(lib().fdtd_grid_set_wait_limit(self.h, int(polls)))

    def set_kernel(self, kernel: str):
        """Leap-frog kernel form: 'auto', 'persist', 'split', 'tma', 'fused' or 'march'."""
        check(lib().fdtd_grid_set_kernel(self.h, KERNELS[kernel]))

    def set_materials(self, eps_r, mu_r=None, sig_e=None, sig_m=None, pec=None, stream=None):
        """Replace the material table (host arrays of nmat values; unspecified
        columns keep the grid spec's values)."""
        sp = self.spec
        cols = []
        for v, d, dt in ((eps_r, sp.eps_r, np.float64), (mu_r, sp.mu_r, np.float64), (sig_e, sp.sig_e, np.float64),
                         (sig_m, sp.sig_m, np.float64), (pec, sp.pec, np.uint8)):
            cols.append(np.ascontiguousarray(np.asarray(d if v is None else v, dtype=dt)))
        ptr = lambda a, ct: a.ctypes.data_as(C.POINTER(ct))
        check(lib().fdtd_grid_set_materials(self.h, int(sp.nmat), ptr(cols[0], C.c_double), ptr(cols[1], C.c_double),
                                            ptr(cols[2], C.c_double), ptr(cols[3], C.c_double),
                                            ptr(cols[4], C.c_uint8), _stream_ptr(stream)))

    def adjoint(self, dt: float, u, dloss_dy, ncheckpoints: int = 0, per_cell: bool = True,
                per_material: bool = True, stream=None):
        """dL/d eps_r by the discrete adjoint: returns (per-cell (nz, ny, nx)
        FP64 tensor or None, per-material (nmat,) FP64 tensor or None)."""
        import torch
        n = int(u.shape[0] if self.m else dloss_dy.shape[0])
        s = self.spec
        gc = torch.empty((s.nz, s.ny, s.nx), dtype=torch.float64, device="cuda") if per_cell else None
        gm = torch.empty((s.nmat,), dtype=torch.float64, device="cuda") if per_material else None
        check(lib().fdtd_adjoint(self.h, float(dt), n, _dptr(u) if self.m else None,
                                 _dptr(dloss_dy) if self.p else None, int(ncheckpoints), _dptr(gc), _dptr(gm),
                                 _stream_ptr(stream)))
        return gc, gm

    def autotune(self, dt: float, trial_steps: int = 64, stream=None):
        """Time the split form's tile shapes and keep the fastest; returns
        (x cells per thread, z planes per thread)."""
        vw, lz = C.c_int(), C.c_int()
        check(lib().fdtd_grid_autotune(self.h, float(dt), int(trial_steps), C.byref(vw), C.byref(lz),
                                       _stream_ptr(stream)))
        return vw.value, lz.value

    def cfl_dt(self) -> float:
        return float(lib().fdtd_cfl_dt(self.h))

    def step(self, dt: float, u, y=None, reset: bool = False, stream=None, nsteps: int = None):
        """Run len(u) (or nsteps) steps; u: (nsteps, m) device tensor; returns y (nsteps, p)."""
        import torch
        n = int(nsteps if nsteps is not None else u.shape[0])
        if y is None and self.p:
            y = torch.empty((n, self.p), dtype=self.dtype, device="cuda")
        check(lib().fdtd_step(self.h, float(dt), n, _dptr(u) if self.m else None,
                              _dptr(y) if self.p else None, 1 if reset else 0, _stream_ptr(stream)))
        return y

    def step_host(self, dt: float, u_host, y_host, reset: bool = False, stream=None):
        """Host-buffer variant: u_host, y_host are (pinned) CPU tensors."""
        n = int(u_host.shape[0])
        check(lib().fdtd_step_host(self.h, float(dt), n, int(u_host.data_ptr()) if self.m else None,
                                   int(y_host.data_ptr()) if self.p else None, 1 if reset else 0,
                                   _stream_ptr(stream)))
        return y_host

    def fields(self, stream=None):
        """(6, nz, ny, nx) tensor copy of Ex, Ey, Ez, Hx, Hy, Hz."""
        import torch
        s = self.spec
        out = torch.empty((6, s.nz, s.ny, s.nx), dtype=self.dtype, device="cuda")
        check(lib().fdtd_fields_get(self.h, _dptr(out), _stream_ptr(stream)))
        return out

    def edge_props(self, stream=None):
        """(4, 3, nz, ny, nx): eps, sigma_e on E edges; mu, sigma_m on H edges."""
        import torch
        s = self.spec
        out = torch.empty((4, 3, s.nz, s.ny, s.nx), dtype=self.dtype, device="cuda")
        check(lib().fdtd_edge_props_get(self.h, _dptr(out), _stream_ptr(stream)))
        return out

    def set_fields(self, f, stream=None):
        f = f.contiguous()
        check(lib().fdtd_fields_set(self.h, _dptr(f), _stream_ptr(stream)))

    def planes(self, k0: int, nk: int, stream=None):
        """(6, nk, ny, nx) device copy of z planes [k0, k0 + nk) (fdtd_planes_get)."""
        import torch
        s = self.spec
        out = torch.empty((6, nk, s.ny, s.nx), dtype=self.dtype, device="cuda")
        check(lib().fdtd_planes_get(self.h, int(k0), int(nk), _dptr(out), _stream_ptr(stream)))
        return out

    def set_planes(self, k0: int, f, stream=None):
        """Overwrite z planes [k0, k0 + f.shape[1]) with f (6, nk, ny, nx) (fdtd_planes_set)."""
        f = f.contiguous()
        check(lib().fdtd_planes_set(self.h, int(k0), int(f.shape[1]), _dptr(f), _stream_ptr(stream)))


KERNELS = {"auto": 0, "persist": 1, "split": 2, "tma": 3, "fused": 4, "march": 5}

MODEL_FIELDS = {"De": 0, "Dse": 1, "Dm": 2, "Dsm": 3, "K": 4, "Kp": 5, "BE": 6, "CE": 7, "sigma": 8}


def _mor_opts(q: int, dt0: float, L: int = 2, M: float = 1.1, fmax: float = 0.0, include_center: bool = True,
              tol: float = None, maxit: int = 20000, defl_tol: float = None, orth: str = None,
              solver: str = "auto") -> MorOpts:
    o = MorOpts()
    check(lib().mor_opts_default(C.byref(o)))
    o.q, o.L, o.M, o.fmax, o.dt0 = int(q), int(L), float(M), float(fmax), float(dt0)
    o.include_center = 1 if include_center else 0
    if tol is not None:
        o.tol = float(tol)
    o.maxit = int(maxit)
    if defl_tol is not None:
        o.defl_tol = float(defl_tol)
    if orth is not None:
        o.orth = MOR_ORTH[orth]
    o.solver = MOR_SOLVER[solver]
    return o


class Basis:
    """mor_basis handle: V1 (3nc x q1), V2 (3nc x q2) on the device."""

    def __init__(self, grid: "Grid", q: int, dt0: float, L: int = 2, M: float = 1.1, fmax: float = 0.0,
                 include_center: bool = True, tol: float = None, maxit: int = 20000,
                 defl_tol: float = None, orth: str = None, solver: str = "auto", stream=None,
                 allow_noconv: bool = False):
        o = _mor_opts(q, dt0, L, M, fmax, include_center, tol, maxit, defl_tol, orth, solver)
        h = C.c_void_p()
        st = lib().mor_build_basis(grid.h, C.byref(o), _stream_ptr(stream), C.byref(h))
        self._adopt(grid, h, st, allow_noconv)

    def _adopt(self, grid, h, st, allow_noconv):
        self.status = st
        if st != FDTD_OK and not (allow_noconv and st == FDTD_ENOCONV and h):
            if h:
                lib().mor_basis_destroy(h)
            check(st)
        self.h = h
        self.grid = grid
        _track(self)

    def info(self):
        q1, q2, it = C.c_int(), C.c_int(), C.c_int()
        r = C.c_double()
        check(lib().mor_basis_info(self.h, C.byref(q1), C.byref(q2), C.byref(it), C.byref(r)))
        return {"q1": q1.value, "q2": q2.value, "max_iters": it.value, "max_resid": r.value}

    def V(self, which: int, stream=None):
        import torch
        inf = self.info()
        q = inf["q1"] if which == 1 else inf["q2"]
        out = torch.empty((q, 3 * self.grid.spec.ncells), dtype=self.grid.dtype, device="cuda")
        check(lib().mor_basis_get(self.h, int(which), _dptr(out), _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().mor_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def build_bases(grids, opts, stream=None, allow_noconv: bool = False):
    """Bases of several grids built side by side (mor_build_basis_batched):
    opts holds one dict of Basis keyword arguments per grid (q and dt0
    required).  Returns a list of Basis in the order of grids."""
    n = len(grids)
    if len(opts) != n:
        raise ValueError("one opts dict per grid")
    arr = (MorOpts * n)(*[_mor_opts(**o) for o in opts])
    hg = (C.c_void_p * n)(*[g.h for g in grids])
    out = (C.c_void_p * n)()
    sts = (C.c_int * n)()
    st = lib().mor_build_basis_batched(n, hg, arr, _stream_ptr(stream), out, sts)
    if st != FDTD_OK and not (allow_noconv and st == FDTD_ENOCONV):
        msg = lib().fdtd_last_error().decode(errors="replace")
        for h in out:
            if h:
                lib().mor_basis_destroy(C.c_void_p(h))
        raise FdtdError(st, msg)
    res = []
    for i in range(n):
        b = Basis.__new__(Basis)
        b._adopt(grids[i], C.c_void_p(out[i]), sts[i], allow_noconv)
        res.append(b)
    return res


class Model:
    """mor_model handle: projected reduced model, perturbation and reduced run."""

    def __init__(self, grid: "Grid", basis: Basis, stream=None):
        h = C.c_void_p()
        check(lib().mor_project(grid.h, basis.h, _stream_ptr(stream), C.byref(h)))
        self.h = h
        self.grid = grid
        _track(self)

    def save(self, path: str, stream=None):
        """Write the projected (unperturbed) model to a file (mor_model_save)."""
        check(lib().mor_model_save(self.h, os.fsencode(path), _stream_ptr(stream)))

    @classmethod
    def load(cls, path: str, grid: "Grid", stream=None) -> "Model":
        """A model read back from mor_model_save's file, for the grid it was
        reduced from (whose sources, probes and precision it carries)."""
        h = C.c_void_p()
        check(lib().mor_model_load(os.fsencode(path), _stream_ptr(stream), C.byref(h)))
        self = cls.__new__(cls)
        self.h = h
        self.grid = grid
        _track(self)
        return self

    def perturb(self, dt: float, gamma: float = 0.9999, stream=None) -> int:
        n = C.c_int()
        check(lib().mor_perturb(self.h, float(dt), float(gamma), C.byref(n), _stream_ptr(stream)))
        return n.value

    def run(self, u, y=None, reset: bool = True, stream=None, nsteps: int = None):
        import torch
        n = int(nsteps if nsteps is not None else u.shape[0])
        if y is None:
            y = torch.empty((n, self.grid.p), dtype=self.grid.dtype, device="cuda")
        check(lib().mor_run(self.h, n, _dptr(u) if self.grid.m else None, _dptr(y) if self.grid.p else None,
                            1 if reset else 0, _stream_ptr(stream)))
        return y

    def gradient(self, basis: "Basis", u, dloss_dy, stream=None):
        """dL/d eps_r of a probe loss of this reduced model with the basis
        frozen (mor_gradient): returns (per-cell (nz, ny, nx) FP64 tensor,
        per-material (nmat,) FP64 tensor, dL/dD~eps (q1, q1) numpy array)."""
        import torch
        s = self.grid.spec
        n = int(u.shape[0] if self.grid.m else dloss_dy.shape[0])
        gc = torch.empty((s.nz, s.ny, s.nx), dtype=torch.float64, device="cuda")
        gm = torch.empty((s.nmat,), dtype=torch.float64, device="cuda")
        q1 = basis.info()["q1"]
        gd = np.zeros((q1, q1), np.float64)
        check(lib().mor_gradient(self.h, basis.h, self.grid.h, n, _dptr(u) if self.grid.m else None,
                                 _dptr(dloss_dy) if self.grid.p else None, _dptr(gc), _dptr(gm),
                                 gd.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
        return gc, gm, gd

    def get(self, name: str, stream=None) -> np.ndarray:
        which = MODEL_FIELDS[name]
        r, c = C.c_int(), C.c_int()
        check(lib().mor_model_get(self.h, which, None, C.byref(r), C.byref(c), _stream_ptr(stream)))
        out = np.zeros((r.value, c.value), np.float64)
        if out.size:
            check(lib().mor_model_get(self.h, which, out.ctypes.data_as(C.POINTER(C.c_double)), None, None,
                                      _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().mor_model_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


ORTH = {"native": 0, "tf32": 1, "bf16": 2}


def gram(A, B, w=None, arith: str = "tf32", stream=None):
    """G = A^T diag(w) B (mor_gram) for column-major FP32 device matrices given
    as (M, n) and (N, n) row-major torch tensors (row r = column r); returns an
    (M, N) FP64 tensor."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    M, n = A.shape
    N = B.shape[0]
    G = torch.empty((M, N), dtype=torch.float64, device="cuda")
    check(lib().mor_gram(MOR_GRAM[arith], int(n), _dptr(A), int(n), int(M), _dptr(B), int(n), int(N),
                         _dptr(w.contiguous()) if w is not None else None, _dptr(G), _stream_ptr(stream)))
    return G


def schur_apply(grid: "Grid", dt0: float, z, x, out=None, stream=None):
    """y_b = S(z_b) x_b (mor_schur_apply): x complex (nb, 3, nz, ny, nx) device
    tensor of the grid's precision; z: nb complex numbers."""
    import torch
    zz = np.asarray(z, np.complex128).ravel()
    zarr = (C.c_double * (2 * zz.size))(*[v for c in zz for v in (c.real, c.imag)])
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    check(lib().mor_schur_apply(grid.h, float(dt0), int(zz.size), zarr, _dptr(x), _dptr(out), _stream_ptr(stream)))
    return out


def shifted_solve(grid: "Grid", dt0: float, z, b, tol: float = 1e-4, maxit: int = 20000, solver: str = "auto",
                  out=None, stream=None, allow_noconv: bool = False):
    """x_b = S(z_b)^{-1} b_b (mor_shifted_solve): b complex (nb, 3, nz, ny, nx)
    device tensor of the grid's precision; z: nb complex numbers.  Returns
    (x, iterations per RHS, final relative residual per RHS)."""
    import torch
    L_ = lib()
    o = MorOpts()
    check(L_.mor_opts_default(C.byref(o)))
    o.dt0, o.tol, o.maxit, o.solver = float(dt0), float(tol), int(maxit), MOR_SOLVER[solver]
    zz = np.asarray(z, np.complex128).ravel()
    zarr = (C.c_double * (2 * zz.size))(*[v for c in zz for v in (c.real, c.imag)])
    b = b.contiguous()
    if out is None:
        out = torch.empty_like(b)
    it = (C.c_int * zz.size)()
    rs = (C.c_double * zz.size)()
    st = L_.mor_shifted_solve(grid.h, C.byref(o), int(zz.size), zarr, _dptr(b), _dptr(out), it, rs,
                              _stream_ptr(stream))
    if st != FDTD_OK and not (allow_noconv and st == FDTD_ENOCONV):
        check(st)
    return out, list(it), list(rs)


def dft(y, dt: float, freqs, hann: bool = False, stream=None) -> np.ndarray:
    """(p, nf) complex spectra of the probe waveforms y (nsteps, p) (fdtd_dft)."""
    import torch
    y = y.contiguous()
    f = np.ascontiguousarray(np.asarray(freqs, np.float64))
    out = np.zeros((y.shape[1], f.size, 2), np.float64)
    prec = FDTD_F64 if y.dtype == torch.float64 else FDTD_F32
    check(lib().fdtd_dft(_dptr(y), int(y.shape[0]), int(y.shape[1]), prec, float(dt), int(f.size),
                         f.ctypes.data_as(C.POINTER(C.c_double)), 1 if hann else 0,
                         out.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
    return out[..., 0] + 1j * out[..., 1]


def sparams(y, y_inc, dt: float, freqs, port_in: int = 0, hann: bool = False, stream=None) -> np.ndarray:
    """(p, nf) complex S-parameters of the probes against the incident wave of a
    reference run (fdtd_sparams); y and y_inc: device (nsteps, p), same type."""
    import torch
    y = y.contiguous()
    y_inc = y_inc.to(y.dtype).contiguous()
    if tuple(y_inc.shape) != tuple(y.shape):
        raise ValueError("y_inc must have the shape of y")
    f = np.ascontiguousarray(np.asarray(freqs, np.float64))
    out = np.zeros((y.shape[1], f.size, 2), np.float64)
    prec = FDTD_F64 if y.dtype == torch.float64 else FDTD_F32
    check(lib().fdtd_sparams(_dptr(y), _dptr(y_inc), int(y.shape[0]), int(y.shape[1]), prec, float(dt), int(f.size),
                             f.ctypes.data_as(C.POINTER(C.c_double)), 1 if hann else 0, int(port_in),
                             out.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)))
    return out[..., 0] + 1j * out[..., 1]


def resonances(y, dt: float, fmin: float, fmax: float, nf: int = 4000, hann: bool = True, rel_floor: float = 0.05,
               npk: int = 16, stream=None) -> np.ndarray:
    """Resonance frequencies (Hz) read off the summed probe spectra (fdtd_resonances)."""
    import torch
    y = y.contiguous()
    pk = np.zeros(npk, np.float64)
    nfound = C.c_int()
    prec = FDTD_F64 if y.dtype == torch.float64 else FDTD_F32
    check(lib().fdtd_resonances(_dptr(y), int(y.shape[0]), int(y.shape[1]), prec, float(dt), float(fmin),
                                float(fmax), int(nf), 1 if hann else 0, float(rel_floor), int(npk),
                                pk.ctypes.data_as(C.POINTER(C.c_double)), C.byref(nfound), _stream_ptr(stream)))
    return pk[:nfound.value]


def compare(y_red, y_ref, stride: int, offset: int, stream=None) -> float:
    """Relative L2 error of y_red against rows offset + i*stride of y_ref (device tensors)."""
    import torch
    prec = FDTD_F64 if y_red.dtype == torch.float64 else FDTD_F32
    err = C.c_double()
    check(lib().mor_compare(_dptr(y_red), _dptr(y_ref), int(y_red.shape[0]), int(stride), int(offset),
                            int(y_red.shape[1]), prec, C.byref(err), _stream_ptr(stream)))
    return err.value


def compare_noalloc(y_red, y_ref, stride: int, offset: int, stream=None) -> float:
    """compare() through mor_compare_noalloc: no device allocation (static scratch)."""
    import torch
    prec = FDTD_F64 if y_red.dtype == torch.float64 else FDTD_F32
    err = C.c_double()
    check(lib().mor_compare_noalloc(_dptr(y_red), _dptr(y_ref), int(y_red.shape[0]), int(stride), int(offset),
                                    int(y_red.shape[1]), prec, C.byref(err), _stream_ptr(stream)))
    return err.value


def step_batched(grids, dts, us, nsteps: int = None, reset: bool = True, stream=None):
    """Advance several grids together (fdtd_step_batched).  us[q]: (nsteps, m_q)
    device tensors (or None for a grid without sources); returns the list of
    probe tensors (nsteps, p_q) (None for a grid without probes)."""
    import torch
    n = len(grids)
    if nsteps is None:
        nsteps = next(int(u.shape[0]) for u in us if u is not None)
    ys = [torch.empty((nsteps, g.p), dtype=g.dtype, device="cuda") if g.p else None for g in grids]
    H = (C.c_void_p * n)(*[g.h.value for g in grids])
    D = (C.c_double * n)(*[float(d) for d in dts])
    U = (C.c_void_p * n)(*[_dptr(u) if (u is not None and g.m) else None for g, u in zip(grids, us)])
    Y = (C.c_void_p * n)(*[_dptr(y) if y is not None else None for y in ys])
    check(lib().fdtd_step_batched(H, n, D, int(nsteps), U, Y, 1 if reset else 0, _stream_ptr(stream)))
    return ys


def probe_response(grid: "Grid", eps_r, dt: float, u, ncheckpoints: int = 0):
    """Probe waveforms y (nsteps, p) of `grid` driven by u, as a differentiable
    function of the per-material relative permittivities eps_r (a torch tensor
    of nmat values): the forward is fdtd_step after fdtd_grid_set_materials,
    the backward the discrete adjoint (fdtd_adjoint)."""
    import torch

    class _ProbeResponse(torch.autograd.Function):
        @staticmethod
        def forward(ctx, eps):
            grid.set_materials(eps.detach().cpu().numpy())
            y = grid.step(dt, u, reset=True)
            return y

        @staticmethod
        def backward(ctx, gy):
            _, gm = grid.adjoint(dt, u, gy.contiguous().to(grid.dtype), ncheckpoints, per_cell=False)
            return gm.to(eps_r.dtype).to(eps_r.device)

    return _ProbeResponse.apply(eps_r)

