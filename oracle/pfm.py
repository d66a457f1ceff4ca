"""FP64 numpy oracle of the phase-field model (PFM) of Sec. 3.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests, the smoke check and
bench.py's CPU-baseline leg use it.  It shares no code with the CUDA path.

The model, in lattice units (grid spacing 1, the LBM's), for a density-matched,
viscosity-matched incompressible binary fluid on a periodic box (Sec. 3):
  div u = 0                                                         (Eq. eq8.1)
  d phi/dt + u.grad phi = M lap mu_tau(phi)                         (Eq. eq2.2)
  du/dt + u.grad u = -grad p + nu lap u + mu(phi) grad phi / rho    (Eq. eq3.2)
  mu_tau = cs2/2 ln((rho+phi)/(rho-phi)) - g_tau cs2 phi/2 - g_tau cs2^2/4 lap phi   (Eq. eq45)
  mu     = the same with g in place of g_tau                        (Eq. eq45.2)
  M = rho (tau - 1/2), nu = cs2 (tau - 1/2), g_tau = tau g / (tau - 1/2).
The paper writes the momentum equation per unit mass; its capillary term is
read here as mu grad phi / rho (rho uniform).  Optional Kolmogorov forcing of
Eq. kolmo (Sec. 4.2): F_x / rho = A sin(2 pi y / L_y) added to the explicit
momentum right-hand side (it is divergence-free, the projection keeps it).

Time stepping (Sec. 3.1, Eqs. eq10-eq13), pseudo-spectral: with
beta = g_tau cs2 / 2, D = M beta and xi^2 = cs2 / 2 the Cahn-Hilliard equation
is D lap[(1/g_tau) ln(..) - phi - xi^2 lap phi] - u.grad phi, split into
  S   = -u.grad phi + D lap[(1/g_tau) ln((rho+phi)/(rho-phi)) - 3 phi]
        - D (xi^2 - dt D / 2) lap^2 phi                              (explicit, Eq. eq12)
  Psi = D (2 lap phi - (dt D / 2) lap^2 phi)                        (implicit, Eq. eq13)
  (phi^{n+1} - phi^n)/dt = (3 S^n - S^{n-1})/2 + (Psi^{n+1} + Psi^n)/2   (Eq. eq11)
(the lap^2 in the second bracket of Eq. eq10 is read as lap, as in Eq. eq13);
the velocity the same way with the nonlinear and capillary terms explicit
(AB2, projected onto divergence-free fields) and nu lap u implicit (CN).
Derivatives are exact spectral ones: i k for first derivatives with the
Nyquist wavenumber of an even axis set to zero (its mode has no first
derivative on the grid), -|k|^2 with the full wavenumbers for the Laplacian;
the projection uses the first-derivative wavenumbers, so the projected field
is divergence-free for the grid's own divergence.  Products are formed in
physical space (no dealiasing: the paper names none).  The first step takes
S^{-1} = S^0.

Fields: phi (scalar) and u (D components), numpy arrays of the box shape
(ny, nx) or (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


class OraclePFM:
    """Phase-field model of Sec. 3 on a periodic box of ``shape`` (numpy order),
    uniform density rho, LBM relaxation time tau and SC coupling g, time step dt."""

    def __init__(self, shape, rho: float, tau: float, g: float, dt: float = 1.0, body_A: float = 0.0):
        if not g > 0:
            raise ValueError("the PFM needs g > 0 (its explicit bracket carries 1/g_tau)")
        self.shape = tuple(int(s) for s in shape)
        self.body_A = float(body_A)
        self.D = len(self.shape)
        self.rho, self.tau, self.g, self.dt = float(rho), float(tau), float(g), float(dt)
        self.M = self.rho * (self.tau - 0.5)
        self.nu = CS2 * (self.tau - 0.5)
        self.g_tau = self.tau * self.g / (self.tau - 0.5)
        self.Dc = self.M * self.g_tau * CS2 / 2.0
        self.xi2 = CS2 / 2.0
        # wave vectors, numpy axis order; k[a] for axis a (last axis = x)
        ks = [2 * np.pi * np.fft.fftfreq(n) for n in self.shape]
        kd = []
        for n, kk in zip(self.shape, ks):
            kk = kk.copy()
            if n % 2 == 0:
                kk[n // 2] = 0.0  # Nyquist: no first derivative
            kd.append(kk)
        self.k = np.meshgrid(*kd, indexing="ij")  # first derivatives and projection
        self.k2 = sum(kk * kk for kk in np.meshgrid(*ks, indexing="ij"))  # Laplacian
        self.kd2 = sum(kk * kk for kk in self.k)
        self.phi_h = None
        self.u_h = None
        self.S_prev = None
        self.N_prev = None
        self.t = 0

    # physical-space axis a of a D-vector: component 0 is x (last numpy axis)
    def _kx(self, comp):
        return self.k[self.D - 1 - comp]

    def init(self, phi, u=None):
        self.phi_h = np.fft.fftn(np.asarray(phi, dtype=np.float64))
        if u is None:
            u = np.zeros(self.shape + (self.D,))
        self.u_h = [np.fft.fftn(np.asarray(u[..., c], dtype=np.float64)) for c in range(self.D)]
        self.S_prev = None
        self.N_prev = None
        self.t = 0
        return self

    def _real(self, a_h):
        return np.real(np.fft.ifftn(a_h))

    def _explicit(self):
        """S^n (Eq. eq12) and the projected momentum right-hand side N^n, in Fourier space."""
        rho, Dc, dt = self.rho, self.Dc, self.dt
        phi = self._real(self.phi_h)
        grad = [self._real(1j * self._kx(c) * self.phi_h) for c in range(self.D)]
        lap = self._real(-self.k2 * self.phi_h)
        u = [self._real(uh) for uh in self.u_h]
        adv = sum(u[c] * grad[c] for c in range(self.D))
        bracket = np.log((rho + phi) / (rho - phi)) / self.g_tau - 3.0 * phi
        S = (np.fft.fftn(-adv) - Dc * self.k2 * np.fft.fftn(bracket)
             - Dc * (self.xi2 - dt * Dc / 2.0) * self.k2 * self.k2 * self.phi_h)
        mu = 0.5 * CS2 * np.log((rho + phi) / (rho - phi)) - 0.5 * self.g * CS2 * phi - 0.25 * self.g * CS2 * CS2 * lap
        N = []
        for a in range(self.D):
            # -d_b (u_a u_b) + mu d_a phi / rho (+ the Kolmogorov force along x)
            div = sum(1j * self._kx(b) * np.fft.fftn(u[a] * u[b]) for b in range(self.D))
            N.append(-div + np.fft.fftn(mu * grad[a]) / rho)
        if self.body_A != 0.0:
            ny = self.shape[-2]
            y = np.arange(ny).reshape([ny if ax == self.D - 2 else 1 for ax in range(self.D)])
            N[0] = N[0] + np.fft.fftn(np.broadcast_to(self.body_A * np.sin(2 * np.pi * y / ny), self.shape))
        # projection onto divergence-free fields: N - k (k.N) / k^2 (first-derivative k);
        # the mean (k = 0) of the right-hand side is dropped: no net force on a periodic box
        kd2 = np.where(self.kd2 == 0, 1.0, self.kd2)
        kN = sum(self._kx(a) * N[a] for a in range(self.D))
        N = [N[a] - self._kx(a) * kN / kd2 for a in range(self.D)]
        for a in range(self.D):
            N[a] = np.where(self.k2 == 0, 0.0, N[a])
        return S, N

    def step(self, nsteps: int = 1):
        dt = self.dt
        lam = self.Dc * (2.0 * self.k2 + dt * self.Dc / 2.0 * self.k2 * self.k2)
        vis = self.nu * self.k2
        for _ in range(int(nsteps)):
            S, N = self._explicit()
            Sp = S if self.S_prev is None else self.S_prev
            Np = N if self.N_prev is None else self.N_prev
            self.phi_h = (self.phi_h * (1 - dt * lam / 2) + dt * (3 * S - Sp) / 2) / (1 + dt * lam / 2)
            self.u_h = [(self.u_h[a] * (1 - dt * vis / 2) + dt * (3 * N[a] - Np[a]) / 2) / (1 + dt * vis / 2)
                        for a in range(self.D)]
            self.S_prev, self.N_prev = S, N
            self.t += 1
        return self

    def fields(self):
        """(phi, u (shape + (D,))) in physical space."""
        phi = self._real(self.phi_h)
        u = np.stack([self._real(uh) for uh in self.u_h], axis=-1)
        return phi, u

    def moments(self):
        """rho_A = (rho + phi)/2, rho_B = (rho - phi)/2, u, and p = cs2 rho + g cs2 rho_A rho_B
        (the SC bulk pressure of the same state, for side-by-side comparisons)."""
        phi, u = self.fields()
        a, b = (self.rho + phi) / 2, (self.rho - phi) / 2
        return a, b, u, CS2 * self.rho + self.g * CS2 * a * b
