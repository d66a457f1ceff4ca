"""Thin ctypes binding of libpfm.so (include/pfm.h): the pseudo-spectral
phase-field model of Sec. 3 on the GPU.  Argument marshalling only; every step
runs in the library's kernels and cuFFT.  Raises if the library is missing:
there is no CPU fallback.

    from paper_1112_5547_gb300 import phase_field
    s = phase_field.PFM((nz, ny, nx), rho=1.4, tau=0.6, g=0.3, dt=0.1, precision="f32")
    s.init(phi).step(100)
    phi, u = s.fields()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import lbm_sc

PFM_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpfm.so")
PFM_F64, PFM_F32 = 0, 1
PRECISIONS = {"f64": PFM_F64, "f32": PFM_F32}
EXPORTS = ("pfm_workspace_bytes", "pfm_create", "pfm_init", "pfm_step", "pfm_fields", "pfm_destroy")


class pfm_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rho", ctypes.c_double), ("tau", ctypes.c_double), ("g", ctypes.c_double), ("dt", ctypes.c_double),
                ("body_A", ctypes.c_double)]


_lib = None


def load(path: str = PFM_LIB):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libpfm.so not found at %s: run paper_1112_5547_gb300.build.build() (nvcc, sm_103a); "
                          "there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    vp, P = ctypes.c_void_p, ctypes.POINTER(pfm_params)
    lib.pfm_workspace_bytes.argtypes = [P]
    lib.pfm_workspace_bytes.restype = ctypes.c_size_t
    lib.pfm_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    lib.pfm_create.restype = ctypes.c_int
    lib.pfm_init.argtypes = [vp, vp, vp]
    lib.pfm_init.restype = ctypes.c_int
    lib.pfm_step.argtypes = [vp, ctypes.c_int]
    lib.pfm_step.restype = ctypes.c_int
    lib.pfm_fields.argtypes = [vp, vp, vp]
    lib.pfm_fields.restype = ctypes.c_int
    lib.pfm_destroy.argtypes = [vp]
    lib.pfm_destroy.restype = None
    _lib = lib
    return lib


def make_params(shape, rho: float, tau: float, g: float, dt: float, precision="f64",
                body_A: float = 0.0) -> pfm_params:
    shape = tuple(int(s) for s in shape)
    if len(shape) == 2:
        dim, nz, (ny, nx) = 2, 1, shape
    else:
        dim, (nz, ny, nx) = 3, shape
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return pfm_params(dim, prec, nx, ny, nz, 0, float(rho), float(tau), float(g), float(dt), float(body_A))


def workspace_bytes(params: pfm_params) -> int:
    return load().pfm_workspace_bytes(ctypes.byref(params))


def _check(status: int, where: str):
    if status != lbm_sc.LBM_OK:
        raise lbm_sc.LbmError(status, where)


class PFM:
    """One phase-field solver on a periodic box of numpy-order ``shape`` with its
    spectral state in a torch-owned workspace (see include/pfm.h)."""

    def __init__(self, shape, rho: float, tau: float, g: float, dt: float = 1.0, precision="f64", device="cuda",
                 stream=None, body_A: float = 0.0):
        import torch
        self.torch = torch
        self.shape = tuple(int(s) for s in shape)
        self.D = len(self.shape)
        self.params = make_params(shape, rho, tau, g, dt, precision, body_A)
        self.dtype = torch.float64 if self.params.precision == PFM_F64 else torch.float32
        nbytes = workspace_bytes(self.params)
        if nbytes == 0:
            raise lbm_sc.LbmError(lbm_sc.LBM_ERR_INVALID_ARG, "pfm_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(load().pfm_create(ctypes.byref(self.params), aligned, nbytes, self.stream.cuda_stream,
                                 ctypes.byref(h)), "pfm_create")
        self.handle = h.value
        self.N = int(np.prod(self.shape))

    def _dev(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=self.dtype).contiguous()

    def init(self, phi, u=None):
        """phi of ``shape``; u of shape + (D,) (component last), divergence-free, or None."""
        self._keep = [self._dev(phi).reshape(-1)]
        du = None
        if u is not None:
            uu = self._dev(u).reshape(-1, self.D).t().contiguous()
            self._keep.append(uu)
            du = uu.data_ptr()
        _check(load().pfm_init(self.handle, self._keep[0].data_ptr(), du), "pfm_init")
        return self

    def step(self, nsteps: int = 1):
        _check(load().pfm_step(self.handle, int(nsteps)), "pfm_step")
        return self

    def fields(self):
        """(phi of ``shape``, u of shape + (D,)) as device tensors."""
        t = self.torch
        phi = t.empty(self.N, dtype=self.dtype, device=self.device)
        u = t.empty(self.D * self.N, dtype=self.dtype, device=self.device)
        _check(load().pfm_fields(self.handle, phi.data_ptr(), u.data_ptr()), "pfm_fields")
        return phi.view(self.shape), u.view(self.D, self.N).t().reshape(self.shape + (self.D,))

    def close(self):
        if getattr(self, "handle", None):
            load().pfm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
