"""FP64 CPU oracle for the two-component Shan-Chen lattice Boltzmann step.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_1112_5547_gb300``) and never imports it.

The arithmetic lives in ``sc_oracle.c`` (plain C, FP64, no fused multiply-add);
this module builds it with gcc and wraps it with ctypes + numpy.  Each function
follows the paper's Sec. 2.1 (Eq. eq:be, the moment definitions, Eq. FORCE, the
isotropy sums) and the F dt/2 momentum shift of Sec. 2.3, or, for OracleFE, the
free-energy model of Sec. 2.2; see the C file for the formulas.

Array conventions (numpy, float64):
  * scalar fields: shape (nz, ny, nx) (x fastest), or (ny, nx) for D2Q9;
  * velocity fields: shape field_shape + (3,) (component last);
  * populations: opaque node-major array of shape (N, 2, Q).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB = os.path.join(_HERE, "libsc_oracle.so")

D2Q9 = 0
D3Q19 = 1


def build(force: bool = False) -> str:
    """Compile sc_oracle.c into libsc_oracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
           "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("tau_A", ctypes.c_double), ("tau_B", ctypes.c_double),
                ("G", ctypes.c_double), ("body_A", ctypes.c_double), ("body_y0", ctypes.c_int),
                ("body_ly", ctypes.c_int), ("forcing", ctypes.c_int)]


class _FEParams(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("tau_g", ctypes.c_double), ("g", ctypes.c_double),
                ("kappa", ctypes.c_double), ("gamma", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.oracle_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
        lib.oracle_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        lib.oracle_init.argtypes = [pp, dp, dp, dp, dp]
        lib.oracle_step.argtypes = [pp, dp, dp, ctypes.c_int]
        lib.oracle_moments.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.oracle_total_momentum.argtypes = [pp, dp, dp]
        fp = ctypes.POINTER(_FEParams)
        lib.oracle_fe_equilibria.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_fe_init.argtypes = [fp, dp, dp, dp]
        lib.oracle_fe_step.argtypes = [fp, dp, dp, ctypes.c_int]
        lib.oracle_fe_moments.argtypes = [fp, dp, dp, dp, dp, dp]
        lib.oracle_fe_fields.argtypes = [fp, dp, dp, dp, dp, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def lattice(lat: int):
    """Velocity set of the oracle: (c as (Q, 3) int array, w as (Q,) float64)."""
    lib = _load()
    c = (ctypes.c_int * (19 * 3))()
    w = np.zeros(19)
    q = lib.oracle_lattice(lat, c, _ptr(w))
    return np.array(c[: q * 3], dtype=np.int64).reshape(q, 3), w[:q].copy()


def equilibrium(lat: int, rho: float, u) -> np.ndarray:
    """Second-order truncated Maxwellian of one node (Sec. 2.1)."""
    lib = _load()
    u3 = np.zeros(3)
    u3[: len(u)] = u
    feq = np.zeros(19)
    q = lib.oracle_equilibrium(lat, float(rho), _ptr(u3), _ptr(feq))
    return feq[:q].copy()


class OracleSC:
    """One lattice of the two-component Shan-Chen model, advanced by the oracle.

    ``lat`` is D2Q9 (0) or D3Q19 (1); ``shape`` is (ny, nx) for D2Q9 or
    (nz, ny, nx) for D3Q19; tau_A, tau_B, G as in Eq. eq:be / Eq. FORCE.
    ``body_A`` is the amplitude of the Kolmogorov force of Eq. kolmo (Sec. 4.2),
    F_s,x = rho_s A sin(2 pi (y + body_y0) / body_ly) (body_ly = 0: ny); the
    offset and period let a window of a larger lattice see its forcing.
    ``forcing`` selects how forces enter the collision: "shift" (the velocity
    shift of Sec. 2.1, the paper's model) or "guo" (the Guo et al. source term
    that Sec. 2.3 names as the cure of the tau-dependent coupling).
    """

    FORCING = {"shift": 0, "guo": 1}

    def __init__(self, lat: int, shape, tau_A: float, tau_B: float, G: float, body_A: float = 0.0,
                 body_y0: int = 0, body_ly: int = 0, forcing: str = "shift"):
        self.lat = int(lat)
        shape = tuple(int(s) for s in shape)
        if self.lat == D2Q9:
            assert len(shape) == 2
            ny, nx = shape
            nz = 1
        else:
            assert len(shape) == 3
            nz, ny, nx = shape
        self.shape = shape
        self.p = _Params(self.lat, nx, ny, nz, float(tau_A), float(tau_B), float(G), float(body_A),
                         int(body_y0), int(body_ly), self.FORCING[forcing])
        self.N = nx * ny * nz
        self.Q = 9 if self.lat == D2Q9 else 19
        self.f = np.zeros((self.N, 2, self.Q))
        self._tmp = np.zeros_like(self.f)
        self.t = 0

    def init(self, rhoA, rhoB, u=None):
        """Populations at rest-frame equilibrium f^eq(rho_s, u) (u=None: rest)."""
        lib = _load()
        rA = np.ascontiguousarray(rhoA, dtype=np.float64).reshape(-1)
        rB = np.ascontiguousarray(rhoB, dtype=np.float64).reshape(-1)
        assert rA.size == self.N and rB.size == self.N
        uu = None
        if u is not None:
            u = np.asarray(u, dtype=np.float64)
            uu = np.zeros((self.N, 3))
            d = u.shape[-1]
            uu[:, :d] = u.reshape(self.N, d)
        rc = lib.oracle_init(ctypes.byref(self.p), _ptr(rA), _ptr(rB), _ptr(uu), _ptr(self.f))
        if rc != 0:
            raise ValueError("oracle_init rejected the parameters")
        self.t = 0
        return self

    def step(self, nsteps: int = 1):
        rc = _load().oracle_step(ctypes.byref(self.p), _ptr(self.f), _ptr(self._tmp), int(nsteps))
        if rc != 0:
            raise ValueError("oracle_step failed (%d)" % rc)
        self.t += int(nsteps)
        return self

    def moments(self):
        """(rho_A, rho_B, u_phys (shape + (3,)), p) of the current populations."""
        lib = _load()
        rA = np.zeros(self.N)
        rB = np.zeros(self.N)
        u = np.zeros((self.N, 3))
        pr = np.zeros(self.N)
        rc = lib.oracle_moments(ctypes.byref(self.p), _ptr(self.f), _ptr(rA), _ptr(rB), _ptr(u),
                                _ptr(pr))
        if rc != 0:
            raise ValueError("oracle_moments failed")
        s = self.shape
        return rA.reshape(s), rB.reshape(s), u.reshape(s + (3,)), pr.reshape(s)

    def kinetic_energy(self) -> float:
        """Total kinetic energy sum_x (rho/2) |u_phys|^2 (Sec. 4.2)."""
        a, b, u, _ = self.moments()
        return float(0.5 * ((a + b) * (u * u).sum(-1)).sum())

    def droplet_nodes(self, phi_T: float = 0.0) -> int:
        """Nodes inside the drop, phi = rho_A - rho_B >= phi_T (Sec. 4.2, M(t) of
        the mass leakage L(t) = M(t) / M_0)."""
        a, b, _, _ = self.moments()
        return int(np.count_nonzero(a - b >= phi_T))

    def total_momentum(self) -> np.ndarray:
        out = np.zeros(3)
        _load().oracle_total_momentum(ctypes.byref(self.p), _ptr(self.f), _ptr(out))
        return out


def fe_equilibria(lat: int, g: float, kappa: float, gamma: float, rho: float, phi: float, u, grad_phi,
                  lap_phi: float):
    """(f^eq, g^eq) of one node of the free-energy model (Sec. 2.2, Eqs. EQFE1, EQFE2)."""
    lib = _load()
    u3 = np.zeros(3)
    u3[: len(u)] = u
    g3 = np.zeros(3)
    g3[: len(grad_phi)] = grad_phi
    feq = np.zeros(19)
    geq = np.zeros(19)
    q = lib.oracle_fe_equilibria(lat, float(g), float(kappa), float(gamma), float(rho), float(phi), _ptr(u3),
                                 _ptr(g3), float(lap_phi), _ptr(feq), _ptr(geq))
    return feq[:q].copy(), geq[:q].copy()


class OracleFE:
    """The free-energy two-population model of Sec. 2.2 (Eqs. FE1, FE2) with the
    functional of Eq. FEtau: relaxation times tau (f) and tau_g (g), coupling g,
    gradient coefficient kappa (default g cs2^2 / 4, as in Eq. FEtau) and Gamma
    (mobility M = Gamma (tau_g - 1/2)).  Same shapes and field conventions as
    OracleSC; moments() reports rho_A = (rho + phi)/2, rho_B = (rho - phi)/2, u
    and the bulk pressure."""

    def __init__(self, lat: int, shape, tau: float, tau_g: float, g: float, kappa: float = None,
                 gamma: float = 1.0):
        self.lat = int(lat)
        shape = tuple(int(s) for s in shape)
        if self.lat == D2Q9:
            ny, nx = shape
            nz = 1
        else:
            nz, ny, nx = shape
        self.shape = shape
        if kappa is None:
            kappa = g / 9.0 / 4.0
        self.p = _FEParams(self.lat, nx, ny, nz, float(tau), float(tau_g), float(g), float(kappa), float(gamma))
        self.N = nx * ny * nz
        self.Q = 9 if self.lat == D2Q9 else 19
        self.f = np.zeros((self.N, 2, self.Q))
        self._tmp = np.zeros_like(self.f)

    def init(self, rhoA, rhoB):
        rA = np.ascontiguousarray(rhoA, dtype=np.float64).reshape(-1)
        rB = np.ascontiguousarray(rhoB, dtype=np.float64).reshape(-1)
        if _load().oracle_fe_init(ctypes.byref(self.p), _ptr(rA), _ptr(rB), _ptr(self.f)) != 0:
            raise ValueError("oracle_fe_init rejected the parameters")
        return self

    def step(self, nsteps: int = 1):
        if _load().oracle_fe_step(ctypes.byref(self.p), _ptr(self.f), _ptr(self._tmp), int(nsteps)) != 0:
            raise ValueError("oracle_fe_step failed")
        return self

    def fields(self):
        """(rho, phi, u, grad phi, lap phi) of the current populations (lattice stencils)."""
        rho, phi, lp = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        u, gp = np.zeros((self.N, 3)), np.zeros((self.N, 3))
        _load().oracle_fe_fields(ctypes.byref(self.p), _ptr(self.f), _ptr(rho), _ptr(phi), _ptr(u), _ptr(gp),
                                 _ptr(lp))
        s = self.shape
        return rho.reshape(s), phi.reshape(s), u.reshape(s + (3,)), gp.reshape(s + (3,)), lp.reshape(s)

    def moments(self):
        rA, rB, pr = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        u = np.zeros((self.N, 3))
        if _load().oracle_fe_moments(ctypes.byref(self.p), _ptr(self.f), _ptr(rA), _ptr(rB), _ptr(u),
                                     _ptr(pr)) != 0:
            raise ValueError("oracle_fe_moments failed")
        s = self.shape
        return rA.reshape(s), rB.reshape(s), u.reshape(s + (3,)), pr.reshape(s)


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))


from .pfm import OraclePFM  # noqa: E402  (the phase-field oracle of Sec. 3)
