"""Thin ctypes binding of liblbm_sc.so (C ABI in include/lbm_sc.h).

Every function with an ``lbm_sc_`` name marshals its arguments and calls the
C entry point of the same name; all lattice arithmetic runs in the library's
CUDA kernels.  PyTorch is used only to own device memory and streams.  There is
no fallback: if the compiled library is missing the import fails loudly.

``Lattice`` bundles a workspace tensor and a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm_sc.so")

LBM_OK = 0
LBM_ERR_INVALID_ARG = 1
LBM_ERR_OUT_OF_MEMORY = 2
LBM_ERR_CUDA = 3
LBM_ERR_UNSTABLE = 4
LBM_ERR_TIMEOUT = 5

LBM_D2Q9 = 0
LBM_D3Q19 = 1

LBM_F64 = 0
LBM_F32 = 1
LBM_F32_STORE_BF16 = 2
LBM_F32_STORE_F16 = 3
LBM_F32_STORE_BF16_REST = 4
LBM_F32_STORE_F16_REST = 5

PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "bf16": LBM_F32_STORE_BF16, "f16": LBM_F32_STORE_F16,
              "bf16_rest": LBM_F32_STORE_BF16_REST, "f16_rest": LBM_F32_STORE_F16_REST}
REST_PRECISIONS = (LBM_F32_STORE_BF16_REST, LBM_F32_STORE_F16_REST)

LBM_FORCING_SHIFT = 0
LBM_FORCING_GUO = 1
FORCINGS = {"shift": LBM_FORCING_SHIFT, "guo": LBM_FORCING_GUO}
LBM_MODEL_SC = 0
LBM_MODEL_FE = 1

# Every entry point declared in include/lbm_sc.h.
EXPORTS = (
    "lbm_sc_workspace_bytes", "lbm_sc_create", "lbm_sc_set_stream", "lbm_sc_init_fields", "lbm_sc_step",
    "lbm_sc_moments", "lbm_sc_diagnostics", "lbm_sc_host_staging_bytes", "lbm_sc_run_host", "lbm_sc_layout",
    "lbm_sc_destroy", "lbm_sc_status_string", "lbm_sc_set_tuning", "lbm_sc_get_tuning",
    "lbm_sc_diagnostics_noalloc", "lbm_sc_batch_workspace_bytes", "lbm_sc_batch_create", "lbm_sc_batch_step",
    "lbm_sc_batch_destroy", "lbm_sc_set_wait_probe", "lbm_sc_error_word", "lbm_sc_host_alloc", "lbm_sc_host_free",
)

# CTA tiles of the ragged-batch step (x columns by y columns); the TMA-fed ones
# take D3Q19 lattices with FP32 storage at least one tile wide in x and y
# (tile 13: the paired 16-bit rest-offset storages instead).
# Persistent grids over an atomic work counter, or (GRID) one CTA per work item.
# Tile 9 gives each lattice its own tile: 64x4 when it is at least 64 wide, else 32x8;
# tiles 10 (32x12) and 11 (64x6 / 32x12 per lattice) run 384-thread CTAs.
BATCH_TILES = ((32, 8), (32, 4), (64, 4), (32, 8), (64, 4), (32, 8), (64, 4), (32, 8), (64, 4), (32, 8), (32, 12),
               (32, 12), (32, 12), (32, 8))
BATCH_TILE_TMA = (False, False, False, True, True, True, True, False, False, True, True, True, True, True)
BATCH_TILE_GRID = (False, False, False, False, False, True, True, True, True, True, True, True, True, True)
BATCH_TILE_SHAPE3 = 12  # each lattice in the best of 64x6, 48x8, 32x12 for its size
BATCH_TILE_REST = 13    # rest-offset 16-bit storage, 32x8 tiles, two CTAs per SM
SHAPE3 = ((32, 12), (64, 6), (48, 8))


def batch_shape3(nx: int, ny: int) -> int:
    """Mirror of the library's choice of a lattice's tile in batch tile 12: the index
    into SHAPE3 of the shape with the least work per lattice node (ragged padding
    times the box columns read per tile column), among the shapes at most as large
    as the lattice; -1 if none fits."""
    best, best_cost = -1, 0.0
    for k, (tx, ty) in enumerate(SHAPE3):
        if nx < tx or ny < ty:
            continue
        pad = (-(-nx // tx) * tx) * (-(-ny // ty) * ty) / (nx * ny)
        cost = pad * (tx + 8) / tx
        if best < 0 or cost < best_cost - 1e-12:
            best, best_cost = k, cost
    return best


def batch_tile_fits(tile: int, lattice: "Lattice") -> bool:
    """Mirror of the library's rule for one lattice of a batch."""
    if not 0 <= tile < len(BATCH_TILES):
        return False
    if not BATCH_TILE_TMA[tile]:
        return True
    tx, ty = BATCH_TILES[tile]
    p = lattice.params
    storage_ok = p.precision in REST_PRECISIONS if tile == BATCH_TILE_REST else p.precision == LBM_F32
    if not (p.lattice == LBM_D3Q19 and storage_ok and p.forcing == LBM_FORCING_SHIFT and p.model == LBM_MODEL_SC):
        return False
    if tile == BATCH_TILE_SHAPE3:
        return batch_shape3(p.nx, p.ny) >= 0
    return p.nx >= tx and p.ny >= ty

# CTA tiles (x columns by y columns) the step kernel can be launched with, and
# their shared-memory stages or CTAs per SM.
# kind 0: register-pipelined kernel;
# 3: low-register re-pull kernel (stages = CTAs per SM asked of the register allocator).
# 4: register-pipelined kernel, three planes of pulls in registers (D3Q19, 32- and 16-bit storage).
# 5: TMA-fed kernel (D3Q19, FP32 storage, lattices at least one tile wide), stages = smem stages.
# 6: the TMA-fed kernel for 16-bit storage (reference- or rest-offset; D3Q19, same size rule).
# RETIRED (-1): ids 5-10 and 26-29 keep their slot so the other ids stay stable; the library
# rejects them (kernels measured slower at every size and removed).
TILES = ((32, 8), (32, 16), (64, 8), (32, 4), (64, 4), (32, 8), (32, 8), (64, 4), (32, 8), (64, 4), (32, 4),
         (32, 4), (32, 8), (64, 4), (32, 4), (32, 4), (32, 8), (16, 8), (32, 8), (64, 4), (32, 4), (32, 4),
         (64, 4), (64, 4), (64, 4), (32, 8), (64, 4), (64, 4),
         (32, 8), (32, 8), (64, 4), (64, 4), (32, 8), (64, 6), (64, 6), (64, 6), (32, 12), (32, 12), (32, 12),
         (64, 8), (48, 8), (48, 8), (64, 4), (32, 8), (64, 4))
RETIRED = -1
TILE_KIND = (0, 0, 0, 0, 0, -1, -1, -1, -1, -1, -1, 3, 3, 3, 3, 4, 4, 4, 5, 5, 5, 5, 5, 5, 5, 5, -1, -1, -1, -1, 6, 6, 6,
             5, 5, 6, 5, 5, 6, 6, 5, 5, 6, 6, 6)
TILE_STAGES = (0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 6, 3, 3, 4, 3, 1, 3, 3, 3, 4, 2, 3, 3, 3, 3, 0, 0, 0, 0, 3, 4, 3, 2, 2, 3, 2,
               2, 3, 2, 2, 2, 2, 2, 2)
# thread-block cluster of the TMA tiles (tiles in x, tiles in y)
TILE_CLUSTER = ((1, 1),) * 22 + ((1, 2), (1, 4), (2, 2), (2, 2), (1, 2), (1, 2), (1, 1), (1, 1), (1, 2), (1, 2),
                                   (1, 1), (1, 2), (1, 1), (1, 2), (1, 2), (1, 1), (1, 2), (1, 2), (1, 2), (1, 1),
                                   (1, 2), (1, 2), (1, 1))


def tile_supported(tile: int, lattice: int, precision: int, forcing: int = 0, model: int = 0) -> bool:
    """Mirror of the library's rule: kind 5 needs D3Q19 with FP32 storage, kind 6 D3Q19 with 16-bit
    storage, kind 4 D3Q19 with 32-bit or reference-offset 16-bit storage; Guo forcing and the FE
    model run on kinds 0 and 3 and on tile 34; retired ids are rejected."""
    if not 0 <= tile < len(TILES):
        return False
    kind = TILE_KIND[tile]
    if kind == RETIRED:
        return False
    if (forcing == LBM_FORCING_GUO or model == LBM_MODEL_FE) and kind not in (0, 3) and tile != 34:
        return False
    if kind in (0, 3):
        return True
    if kind == 5:
        return lattice == LBM_D3Q19 and precision == LBM_F32
    if kind == 6:
        return lattice == LBM_D3Q19 and precision in (LBM_F32_STORE_BF16, LBM_F32_STORE_F16) + REST_PRECISIONS
    if kind == 4:
        return lattice == LBM_D3Q19 and precision in (LBM_F32, LBM_F32_STORE_BF16, LBM_F32_STORE_F16)
    return lattice == LBM_D3Q19 and precision not in REST_PRECISIONS


class lbm_sc_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("precision", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("forcing", ctypes.c_int32),
                ("tau_A", ctypes.c_double), ("tau_B", ctypes.c_double), ("G", ctypes.c_double),
                ("rho_ref_A", ctypes.c_double), ("rho_ref_B", ctypes.c_double), ("body_A", ctypes.c_double),
                ("model", ctypes.c_int32), ("reserved", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("gamma", ctypes.c_double)]


class lbm_sc_window(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("r_in", ctypes.c_double), ("r_out", ctypes.c_double)]


class lbm_sc_diag(ctypes.Structure):
    _fields_ = [("mass_A", ctypes.c_double), ("mass_B", ctypes.c_double), ("momentum", ctypes.c_double * 3),
                ("kinetic_energy", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("min_rho_A", ctypes.c_double), ("min_rho_B", ctypes.c_double), ("nonfinite", ctypes.c_double),
                ("in_count", ctypes.c_double), ("in_rho_A", ctypes.c_double), ("in_p", ctypes.c_double),
                ("out_count", ctypes.c_double), ("out_rho_A", ctypes.c_double), ("out_p", ctypes.c_double),
                ("droplet_nodes", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "momentum"}
        d["momentum"] = tuple(self.momentum)
        return d


class lbm_sc_tuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("zchunk", ctypes.c_int32)]


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s" % (where, lbm_sc_status_string(status)))


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbm_sc.so (built by paper_1112_5547_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblbm_sc.so not found at %s: run paper_1112_5547_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P = ctypes.POINTER(lbm_sc_params)
    lib.lbm_sc_workspace_bytes.argtypes = [P]
    lib.lbm_sc_workspace_bytes.restype = ctypes.c_size_t
    lib.lbm_sc_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    lib.lbm_sc_set_stream.argtypes = [vp, vp]
    lib.lbm_sc_init_fields.argtypes = [vp, vp, vp, vp]
    lib.lbm_sc_step.argtypes = [vp, ctypes.c_int]
    lib.lbm_sc_moments.argtypes = [vp, vp, vp, vp, vp]
    lib.lbm_sc_diagnostics.argtypes = [vp, ctypes.POINTER(lbm_sc_window), ctypes.POINTER(lbm_sc_diag)]
    lib.lbm_sc_host_staging_bytes.argtypes = [P]
    lib.lbm_sc_host_staging_bytes.restype = ctypes.c_size_t
    lib.lbm_sc_run_host.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp]
    lib.lbm_sc_host_alloc.argtypes = [ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.lbm_sc_host_free.argtypes = [vp, ctypes.c_size_t]
    ip = ctypes.POINTER(ctypes.c_int)
    lib.lbm_sc_layout.argtypes = [vp, ip, ip, ip, ip, ip, ip, ctypes.POINTER(vp)]
    lib.lbm_sc_set_tuning.argtypes = [vp, ctypes.POINTER(lbm_sc_tuning)]
    lib.lbm_sc_set_wait_probe.argtypes = [vp, ctypes.c_int]
    lib.lbm_sc_error_word.argtypes = [vp, ip]
    lib.lbm_sc_get_tuning.argtypes = [vp, ctypes.POINTER(lbm_sc_tuning)]
    lib.lbm_sc_diagnostics_noalloc.argtypes = [P, vp, ctypes.POINTER(lbm_sc_window), vp, vp]
    lib.lbm_sc_diagnostics_noalloc.restype = ctypes.c_int
    lib.lbm_sc_destroy.argtypes = [vp]
    lib.lbm_sc_destroy.restype = None
    HP = ctypes.POINTER(vp)
    lib.lbm_sc_batch_workspace_bytes.argtypes = [HP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.lbm_sc_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.lbm_sc_batch_create.argtypes = [HP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                        ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    lib.lbm_sc_batch_step.argtypes = [vp, ctypes.c_int]
    lib.lbm_sc_batch_destroy.argtypes = [vp]
    lib.lbm_sc_batch_destroy.restype = None
    lib.lbm_sc_status_string.argtypes = [ctypes.c_int]
    lib.lbm_sc_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        getattr(lib, name)
    for name in ("lbm_sc_create", "lbm_sc_set_stream", "lbm_sc_init_fields", "lbm_sc_step", "lbm_sc_moments",
                 "lbm_sc_diagnostics", "lbm_sc_run_host", "lbm_sc_layout", "lbm_sc_set_tuning",
                 "lbm_sc_get_tuning", "lbm_sc_batch_create", "lbm_sc_batch_step", "lbm_sc_set_wait_probe",
                 "lbm_sc_error_word", "lbm_sc_host_alloc", "lbm_sc_host_free"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != LBM_OK:
        raise LbmError(status, where)


def make_params(lattice: int, shape, tau_A: float, tau_B: float, G: float, precision="f32",
                rho_ref_A: float = 0.0, rho_ref_B: float = 0.0, body_A: float = 0.0,
                forcing="shift", model=LBM_MODEL_SC, kappa: float = 0.0, gamma: float = 0.0) -> lbm_sc_params:
    """Parameters for a lattice of numpy-style shape (ny, nx) or (nz, ny, nx);
    body_A is the Kolmogorov forcing amplitude of Eq. kolmo (0: none); forcing
    "shift" (the paper's velocity shift) or "guo" (lbm_forcing)."""
    shape = tuple(int(s) for s in shape)
    if len(shape) == 2:
        nz, (ny, nx) = 1, shape
    else:
        nz, ny, nx = shape
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    frc = FORCINGS[forcing] if isinstance(forcing, str) else int(forcing)
    return lbm_sc_params(int(lattice), prec, nx, ny, nz, frc, float(tau_A), float(tau_B), float(G),
                         float(rho_ref_A), float(rho_ref_B), float(body_A), int(model), 0, float(kappa), float(gamma))


# ---- one Python function per C entry point ----------------------------------
def lbm_sc_workspace_bytes(params: lbm_sc_params) -> int:
    return int(load().lbm_sc_workspace_bytes(ctypes.byref(params)))


def lbm_sc_diagnostics_noalloc(params: lbm_sc_params, d_populations: int, window: Optional[lbm_sc_window],
                               d_out: int, stream: int = 0) -> None:
    """Diagnostics into a device lbm_sc_diag at d_out, scratch in the library's static memory."""
    _check(load().lbm_sc_diagnostics_noalloc(ctypes.byref(params), ctypes.c_void_p(d_populations),
                                             ctypes.byref(window) if window is not None else None,
                                             ctypes.c_void_p(d_out), ctypes.c_void_p(stream)),
           "lbm_sc_diagnostics_noalloc")


def lbm_sc_host_staging_bytes(params: lbm_sc_params) -> int:
    return int(load().lbm_sc_host_staging_bytes(ctypes.byref(params)))


def lbm_sc_create(params: lbm_sc_params, d_workspace: int, workspace_bytes: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().lbm_sc_create(ctypes.byref(params), ctypes.c_void_p(d_workspace), ctypes.c_size_t(workspace_bytes),
                                ctypes.c_void_p(stream), ctypes.byref(h)), "lbm_sc_create")
    return h.value


def lbm_sc_set_stream(h: int, stream: int) -> None:
    _check(load().lbm_sc_set_stream(ctypes.c_void_p(h), ctypes.c_void_p(stream)), "lbm_sc_set_stream")


def lbm_sc_init_fields(h: int, d_rhoA: int, d_rhoB: int, d_u: Optional[int] = None) -> None:
    _check(load().lbm_sc_init_fields(ctypes.c_void_p(h), ctypes.c_void_p(d_rhoA), ctypes.c_void_p(d_rhoB),
                                     ctypes.c_void_p(d_u or 0)), "lbm_sc_init_fields")


def lbm_sc_step(h: int, nsteps: int) -> None:
    _check(load().lbm_sc_step(ctypes.c_void_p(h), int(nsteps)), "lbm_sc_step")


def lbm_sc_moments(h: int, d_rhoA=None, d_rhoB=None, d_u=None, d_p=None) -> None:
    _check(load().lbm_sc_moments(ctypes.c_void_p(h), ctypes.c_void_p(d_rhoA or 0), ctypes.c_void_p(d_rhoB or 0),
                                 ctypes.c_void_p(d_u or 0), ctypes.c_void_p(d_p or 0)), "lbm_sc_moments")


def lbm_sc_diagnostics(h: int, window: Optional[lbm_sc_window] = None, check: bool = True):
    """Returns (status, lbm_sc_diag).  With check=True a status other than LBM_OK raises."""
    out = lbm_sc_diag()
    st = load().lbm_sc_diagnostics(ctypes.c_void_p(h), ctypes.byref(window) if window is not None else None,
                                   ctypes.byref(out))
    if check:
        _check(st, "lbm_sc_diagnostics")
    return st, out


def lbm_sc_run_host(h: int, d_staging: int, staging_bytes: int, h_rhoA: int, h_rhoB: int, h_u: Optional[int],
                    nsteps: int, h_rhoA_out=None, h_rhoB_out=None, h_u_out=None, h_p_out=None) -> None:
    v = ctypes.c_void_p
    _check(load().lbm_sc_run_host(v(h), v(d_staging), ctypes.c_size_t(staging_bytes), v(h_rhoA), v(h_rhoB),
                                  v(h_u or 0), int(nsteps), v(h_rhoA_out or 0), v(h_rhoB_out or 0), v(h_u_out or 0),
                                  v(h_p_out or 0)), "lbm_sc_run_host")


def lbm_sc_host_alloc(nbytes: int) -> int:
    """Address of a driver-allocated, page-locked host buffer of nbytes (release with lbm_sc_host_free)."""
    p = ctypes.c_void_p()
    _check(load().lbm_sc_host_alloc(ctypes.c_size_t(nbytes), ctypes.byref(p)), "lbm_sc_host_alloc")
    return p.value


def lbm_sc_host_free(p: int, nbytes: int) -> None:
    _check(load().lbm_sc_host_free(ctypes.c_void_p(p), ctypes.c_size_t(nbytes)), "lbm_sc_host_free")


class HostBuffer:
    """A buffer of lbm_sc_host_alloc seen as a CPU torch tensor of `count` values
    of `dtype` (``.tensor``); freed by close() or when the object goes away (the
    tensor must not outlive it)."""

    def __init__(self, count: int, dtype=None):
        import torch
        dtype = dtype or torch.float32
        self.nbytes = int(count) * torch.empty((), dtype=dtype).element_size()
        self.ptr = lbm_sc_host_alloc(max(self.nbytes, 1))
        raw = (ctypes.c_uint8 * self.nbytes).from_address(self.ptr)
        self.tensor = torch.frombuffer(raw, dtype=dtype, count=int(count)) if count else torch.empty(0, dtype=dtype)

    def close(self) -> None:
        if self.ptr:
            self.tensor = None
            lbm_sc_host_free(self.ptr, max(self.nbytes, 1))
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_sc_layout(h: int):
    """(elem_bytes, Q, pitch_x, pitch_y, ghost_x, ghost_y, device pointer of the current populations)."""
    vals = [ctypes.c_int() for _ in range(6)]
    ptr = ctypes.c_void_p()
    _check(load().lbm_sc_layout(ctypes.c_void_p(h), *(ctypes.byref(v) for v in vals), ctypes.byref(ptr)),
           "lbm_sc_layout")
    return tuple(v.value for v in vals) + (ptr.value,)


def lbm_sc_set_wait_probe(h: int, tries: int) -> None:
    _check(load().lbm_sc_set_wait_probe(ctypes.c_void_p(h), int(tries)), "lbm_sc_set_wait_probe")


def lbm_sc_error_word(h: int) -> int:
    w = ctypes.c_int()
    _check(load().lbm_sc_error_word(ctypes.c_void_p(h), ctypes.byref(w)), "lbm_sc_error_word")
    return w.value


def lbm_sc_set_tuning(h: int, tile: int, zchunk: int = 0) -> None:
    t = lbm_sc_tuning(int(tile), int(zchunk))
    _check(load().lbm_sc_set_tuning(ctypes.c_void_p(h), ctypes.byref(t)), "lbm_sc_set_tuning")


def lbm_sc_get_tuning(h: int):
    t = lbm_sc_tuning()
    _check(load().lbm_sc_get_tuning(ctypes.c_void_p(h), ctypes.byref(t)), "lbm_sc_get_tuning")
    return t.tile, t.zchunk


def lbm_sc_destroy(h: int) -> None:
    load().lbm_sc_destroy(ctypes.c_void_p(h))


def _handle_array(handles):
    return (ctypes.c_void_p * len(handles))(*[ctypes.c_void_p(h) for h in handles])


def lbm_sc_batch_workspace_bytes(handles, tile: int = 0, zchunk: int = 0) -> int:
    arr = _handle_array(handles)
    return int(load().lbm_sc_batch_workspace_bytes(arr, len(handles), int(tile), int(zchunk)))


def lbm_sc_batch_create(handles, tile: int, zchunk: int, graph_steps: int, d_workspace: int, workspace_bytes: int,
                        stream: int = 0) -> int:
    arr = _handle_array(handles)
    b = ctypes.c_void_p()
    _check(load().lbm_sc_batch_create(arr, len(handles), int(tile), int(zchunk), int(graph_steps),
                                      ctypes.c_void_p(d_workspace), ctypes.c_size_t(workspace_bytes),
                                      ctypes.c_void_p(stream), ctypes.byref(b)), "lbm_sc_batch_create")
    return b.value


def lbm_sc_batch_step(b: int, nsteps: int) -> None:
    _check(load().lbm_sc_batch_step(ctypes.c_void_p(b), int(nsteps)), "lbm_sc_batch_step")


def lbm_sc_batch_destroy(b: int) -> None:
    load().lbm_sc_batch_destroy(ctypes.c_void_p(b))


def lbm_sc_status_string(status: int) -> str:
    return load().lbm_sc_status_string(int(status)).decode()


# ---- convenience wrapper over torch-owned device memory ---------------------
@dataclass
class Window:
    centre: tuple
    r_in: float
    r_out: float

    def to_c(self) -> lbm_sc_window:
        c = list(self.centre) + [0.0] * (3 - len(self.centre))
        return lbm_sc_window(float(c[0]), float(c[1]), float(c[2]), float(self.r_in), float(self.r_out))


def FELattice(lattice: int, shape, tau: float, tau_g: float, g: float, precision="f32", kappa: float = None,
              gamma: float = 1.0, device="cuda", stream=None) -> "Lattice":
    """A lattice of the free-energy model of Sec. 2.2 (lbm_model LBM_MODEL_FE):
    relaxation times tau (f) and tau_g (g), coupling g of the Eq. FEtau functional,
    gradient coefficient kappa (None: the library's default, g cs2^2 / 4 as in Eq. FEtau) and Gamma."""
    if kappa is None:
        kappa = -1.0  # a negative kappa selects the library's Eq. FEtau coefficient
    return Lattice(lattice, shape, tau, tau_g, g, precision, device=device, stream=stream, model=LBM_MODEL_FE,
                   kappa=kappa, gamma=gamma)


class Lattice:
    """A lattice whose workspace is a torch uint8 tensor on ``device``.

    ``shape`` is numpy order: (ny, nx) for D2Q9, (nz, ny, nx) for D3Q19.
    ``body_A`` switches on the Kolmogorov forcing F_x = rho A sin(2 pi y / ny)
    of Eq. kolmo (Sec. 4.2); ``forcing`` is "shift" (Sec. 2.1) or "guo" (Sec. 2.3).
    """

    def __init__(self, lattice: int, shape, tau_A: float, tau_B: float, G: float, precision="f32",
                 rho_ref_A: float = 0.0, rho_ref_B: float = 0.0, device="cuda", stream=None, body_A: float = 0.0,
                 forcing="shift", model=LBM_MODEL_SC, kappa: float = 0.0, gamma: float = 0.0):
        import torch

        self.torch = torch
        self.params = make_params(lattice, shape, tau_A, tau_B, G, precision, rho_ref_A, rho_ref_B, body_A,
                                  forcing, model, kappa, gamma)
        self.shape = tuple(int(s) for s in shape)
        self.lattice = int(lattice)
        self.D = 2 if self.lattice == LBM_D2Q9 else 3
        self.N = int(np.prod(self.shape))
        self.cdtype = torch.float64 if self.params.precision == LBM_F64 else torch.float32
        nbytes = lbm_sc_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(LBM_ERR_INVALID_ARG, "lbm_sc_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = lbm_sc_create(self.params, aligned, nbytes, self.stream.cuda_stream)
        self.workspace_bytes = nbytes

    def close(self):
        if getattr(self, "handle", None):
            lbm_sc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=self.cdtype).contiguous()

    def init(self, rhoA, rhoB, u=None):
        """rhoA, rhoB of ``shape``; u of shape + (D,) (component last) or None."""
        self._keep = [self._dev(rhoA).reshape(-1), self._dev(rhoB).reshape(-1)]
        du = None
        if u is not None:
            uu = self._dev(u).reshape(-1, self.D).t().contiguous()
            self._keep.append(uu)
            du = uu.data_ptr()
        lbm_sc_init_fields(self.handle, self._keep[0].data_ptr(), self._keep[1].data_ptr(), du)
        return self

    def step(self, nsteps: int = 1):
        lbm_sc_step(self.handle, nsteps)
        return self

    def set_tuning(self, tile: int, zchunk: int = 0):
        lbm_sc_set_tuning(self.handle, tile, zchunk)
        return self

    def tile_fits(self, tile: int) -> bool:
        """Whether the library accepts this tile for this lattice (kind, precision, size)."""
        old = self.tuning()
        try:
            lbm_sc_set_tuning(self.handle, tile, 0)
        except LbmError:
            return False
        lbm_sc_set_tuning(self.handle, old[0], old[1])
        return True

    def tuning(self):
        return lbm_sc_get_tuning(self.handle)

    def moments(self):
        """(rho_A, rho_B, u (shape + (D,)), p) as device tensors in the compute dtype."""
        t = self.torch
        rA = t.empty(self.N, dtype=self.cdtype, device=self.device)
        rB = t.empty_like(rA)
        u = t.empty(self.D * self.N, dtype=self.cdtype, device=self.device)
        p = t.empty_like(rA)
        lbm_sc_moments(self.handle, rA.data_ptr(), rB.data_ptr(), u.data_ptr(), p.data_ptr())
        u = u.view(self.D, self.N).t().reshape(self.shape + (self.D,))
        return rA.view(self.shape), rB.view(self.shape), u, p.view(self.shape)

    def diagnostics(self, window: Optional[Window] = None, check: bool = True):
        st, d = lbm_sc_diagnostics(self.handle, window.to_c() if window is not None else None, check=check)
        out = d.as_dict()
        out["status"] = st
        return out

    def state(self):
        """The whole current population buffer as raw bytes (with the float2 density
        plane of the rest-offset precisions): save and restore it to rewind."""
        eb, q, px, py, gx, gy, ptr = lbm_sc_layout(self.handle)
        planes = q if self.params.precision in REST_PRECISIONS else 2 * q
        n = planes * self.params.nz * py * px * eb
        if self.params.precision in REST_PRECISIONS:
            n += self.params.nz * py * px * 8
        off = ptr - self.workspace.data_ptr()
        return self.workspace[off: off + n]

    def populations(self):
        """The current population buffer as a (2, Q, nz, pitch_y, pitch_x) tensor view
        (GPU velocity order, ghost-padded; see lbm_sc_layout).  The rest-offset
        precisions pair the species in one word per direction: their view is
        (Q, nz, pitch_y, pitch_x, 2), the last index the species."""
        t = self.torch
        eb, q, px, py, gx, gy, ptr = lbm_sc_layout(self.handle)
        rest = self.params.precision in REST_PRECISIONS
        nz = self.params.nz
        off = ptr - self.workspace.data_ptr()
        if rest:
            dt = t.bfloat16 if self.params.precision == LBM_F32_STORE_BF16_REST else t.float16
            n = q * nz * py * px * 2
            return self.workspace[off: off + n * 2].view(dt).view(q, nz, py, px, 2)
        dt = {8: t.float64, 4: t.float32}.get(eb)
        if dt is None:
            dt = t.bfloat16 if self.params.precision == LBM_F32_STORE_BF16 else t.float16
        n = 2 * q * nz * py * px
        return self.workspace[off: off + n * eb].view(dt).view(2, q, nz, py, px)


class Batch:
    """Lattices (``Lattice`` objects of one lattice kind and precision) advanced
    together by one launch per step; the batch workspace is a torch uint8 tensor.
    The lattices must stay alive as long as the batch, and be stepped only
    through it while it exists."""

    def __init__(self, lattices, tile: int = 0, zchunk: int = 0, graph_steps: int = 0, stream=None):
        import torch

        if not lattices:
            raise ValueError("a batch needs at least one lattice")
        self.lattices = list(lattices)
        dev = self.lattices[0].device
        self.stream = stream if stream is not None else self.lattices[0].stream
        hs = [lat.handle for lat in self.lattices]
        nbytes = lbm_sc_batch_workspace_bytes(hs, tile, zchunk)
        if nbytes == 0:
            raise LbmError(LBM_ERR_INVALID_ARG, "lbm_sc_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.handle = lbm_sc_batch_create(hs, tile, zchunk, graph_steps, aligned, nbytes, self.stream.cuda_stream)
        self.workspace_bytes = nbytes

    def step(self, nsteps: int = 1):
        lbm_sc_batch_step(self.handle, nsteps)
        return self

    def close(self):
        if getattr(self, "handle", None):
            lbm_sc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
