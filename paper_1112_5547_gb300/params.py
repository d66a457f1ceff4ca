"""Physical parameters of the Shan-Chen model and the paper's phase-field mapping.

Host-side helpers only (no lattice arithmetic).  Definitions of Table 1
(tab:Coll_map_par) and the tau-modified coupling of Sec. 2.1:
  g_tau = tau g / (tau - 1/2),       nu = cs2 (tau - 1/2),   M = rho (tau - 1/2),
  kappa = g cs2^2 / 4,  beta = g cs2 / 2,  beta_tau = g_tau cs2 / 2,  xi = sqrt(kappa/beta),
  Pe = U H / (beta_tau M),  Ch = xi / H,  Ca = nu rho U / sqrt(beta kappa),  Re = U H / nu.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

CS2 = 1.0 / 3.0


def g_tau(tau: float, g: float) -> float:
    """tau-modified coupling of the SC chemical potential (Sec. 2.1)."""
    return tau * g / (tau - 0.5)


def viscosity(tau: float) -> float:
    """Kinematic viscosity nu = cs2 (tau - 1/2) (Sec. 2.1)."""
    return CS2 * (tau - 0.5)


def coupling_from_product(G_rho_tot: float, rho_tot: float) -> float:
    """G such that G * rho_tot equals the given product."""
    return G_rho_tot / rho_tot


@dataclass(frozen=True)
class PhaseFieldGroups:
    """Dimensionless groups of Table 1 for a box L = 2 pi H and velocity scale U."""

    g_tau: float
    nu: float
    M: float
    kappa: float
    beta: float
    beta_tau: float
    xi: float
    Pe: float
    Ch: float
    Ca: float
    Re: float


def phase_field_groups(rho: float, tau: float, g: float, L: float, U: float) -> PhaseFieldGroups:
    H = L / (2.0 * math.pi)
    gt = g_tau(tau, g)
    nu = viscosity(tau)
    M = rho * (tau - 0.5)
    kappa = g * CS2 * CS2 / 4.0
    beta = g * CS2 / 2.0
    beta_tau = gt * CS2 / 2.0
    xi = math.sqrt(kappa / beta)
    return PhaseFieldGroups(gt, nu, M, kappa, beta, beta_tau, xi,
                            Pe=U * H / (beta_tau * M), Ch=xi / H,
                            Ca=nu * rho * U / math.sqrt(beta * kappa), Re=U * H / nu)


def velocity_for_peclet(rho: float, tau: float, g: float, L: float, Pe: float) -> float:
    """The velocity scale U that gives the Peclet number Pe (Table 1)."""
    H = L / (2.0 * math.pi)
    return Pe * g_tau(tau, g) * CS2 / 2.0 * rho * (tau - 0.5) / H
