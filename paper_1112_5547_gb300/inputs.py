"""Seeded synthetic initial fields for drop, slab and linear-mode runs.

This module holds only input recipes (shapes, profiles, seeded noise); it
does none of the lattice Boltzmann arithmetic, so both the CUDA path and the
CPU oracle can be fed from it.  Fields are numpy arrays of shape (ny, nx) in
2D or (nz, ny, nx) in 3D, x fastest.

Recipes (the paper's static-drop set-up, Sec. 4.1: a drop of one component at
rest in the other on a fully periodic box):
  * drop: rho_A(r) = rho_lo + (rho_hi - rho_lo) * (1 - tanh((r - R) / width)) / 2,
    r the periodic minimum-image distance from the centre in node units,
    rho_B = rho_hi + rho_lo - rho_A; then independent uniform noise in
    [-noise, +noise] is added to rho_A and rho_B (numpy PCG64, fixed seed);
  * slab: the same profile with r = |x - x_c| along the first axis, giving two
    flat interfaces;
  * phi_mode: rho_A, rho_B = rho/2 +- a sin(2 pi k x / nx) (no noise);
  * shear_wave: uniform densities with u_x = U sin(2 pi y / ny).
"""
from __future__ import annotations

import numpy as np


def _axis_dist(n: int, c: float) -> np.ndarray:
    d = np.abs(np.arange(n, dtype=np.float64) - c)
    return np.minimum(d, n - d)


def radial_distance(shape, centre) -> np.ndarray:
    """Periodic minimum-image distance of every node from ``centre``.

    ``shape`` is (ny, nx) or (nz, ny, nx); ``centre`` is (cx, cy) or (cx, cy, cz).
    """
    shape = tuple(shape)
    if len(shape) == 2:
        ny, nx = shape
        dx = _axis_dist(nx, centre[0])[None, :]
        dy = _axis_dist(ny, centre[1])[:, None]
        return np.sqrt(dx * dx + dy * dy)
    nz, ny, nx = shape
    dx = _axis_dist(nx, centre[0])[None, None, :]
    dy = _axis_dist(ny, centre[1])[None, :, None]
    dz = _axis_dist(nz, centre[2])[:, None, None]
    return np.sqrt(dx * dx + dy * dy + dz * dz)


def _profile(r, R, rho_hi, rho_lo, width):
    return rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 - np.tanh((r - R) / width))


def _add_noise(rhoA, rhoB, noise, seed):
    if noise > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        rhoA += rng.uniform(-noise, noise, size=rhoA.shape)
        rhoB += rng.uniform(-noise, noise, size=rhoB.shape)


def drop(shape, R, centre=None, rho_hi=1.0, rho_lo=0.04, width=2.0, noise=1e-3, seed=0,
         dtype=np.float64):
    """Component A as a drop of radius R inside component B (periodic box)."""
    shape = tuple(int(s) for s in shape)
    if centre is None:
        centre = tuple(n / 2.0 for n in reversed(shape))  # (nx/2, ny/2[, nz/2])
    r = radial_distance(shape, centre)
    rhoA = _profile(r, float(R), rho_hi, rho_lo, width)
    del r
    rhoB = (rho_hi + rho_lo) - rhoA
    _add_noise(rhoA, rhoB, noise, seed)
    return rhoA.astype(dtype, copy=False), rhoB.astype(dtype, copy=False)


def slab(shape, half_width, centre_x=None, rho_hi=1.0, rho_lo=0.04, width=2.0, noise=1e-3,
         seed=0, dtype=np.float64):
    """Component A as a slab |x - x_c| < half_width: two flat interfaces normal to x."""
    shape = tuple(int(s) for s in shape)
    nx = shape[-1]
    if centre_x is None:
        centre_x = nx / 2.0
    d = _axis_dist(nx, centre_x)
    prof = _profile(d, float(half_width), rho_hi, rho_lo, width)
    rhoA = np.broadcast_to(prof, shape).astype(np.float64)
    rhoB = (rho_hi + rho_lo) - rhoA
    _add_noise(rhoA, rhoB, noise, seed)
    return rhoA.astype(dtype, copy=False), rhoB.astype(dtype, copy=False)


def phi_mode(shape, rho=1.0, amplitude=1e-4, k=1, dtype=np.float64):
    """rho_A = rho/2 + a sin(2 pi k x/nx), rho_B = rho/2 - a sin(...): a pure phi mode."""
    shape = tuple(int(s) for s in shape)
    nx = shape[-1]
    s = np.sin(2.0 * np.pi * k * np.arange(nx) / nx)
    rhoA = np.broadcast_to(0.5 * rho + amplitude * s, shape).astype(np.float64)
    rhoB = np.broadcast_to(0.5 * rho - amplitude * s, shape).astype(np.float64)
    return rhoA.astype(dtype, copy=False), rhoB.astype(dtype, copy=False)


def shear_wave(shape, rhoA=0.5, rhoB=0.5, U=1e-4, k=1, dtype=np.float64):
    """Uniform densities with u_x(y) = U sin(2 pi k y / ny); returns (rhoA, rhoB, u)."""
    shape = tuple(int(s) for s in shape)
    ny = shape[-2]
    d = len(shape)
    ux = U * np.sin(2.0 * np.pi * k * np.arange(ny) / ny)
    u = np.zeros(shape + (d,))
    if d == 2:
        u[..., 0] = ux[:, None]
    else:
        u[..., 0] = ux[None, :, None]
    ra = np.full(shape, rhoA)
    rb = np.full(shape, rhoB)
    return ra.astype(dtype), rb.astype(dtype), u.astype(dtype)


def uniform_velocity(shape, U):
    """A uniform velocity field with components U (len 2 or 3)."""
    shape = tuple(int(s) for s in shape)
    u = np.zeros(shape + (len(shape),))
    for a, v in enumerate(U):
        u[..., a] = v
    return u


RHO_TOT = 1.04  # rho_hi + rho_lo of the drop recipe


def ragged_drop_specs(n=64, sizes=(32, 48, 64, 96, 128), dim=3, seed=3):
    """Specifications of a ragged batch of independent drop lattices.

    Per lattice, drawn from one numpy PCG64 stream: the edge L uniformly from
    ``sizes`` (a cube, or a square for dim=2), G rho_tot uniformly in
    [2.2, 2.8], tau_A and tau_B uniformly in [0.6, 1.5], a drop radius
    uniformly in [L/8, L/3] at a uniformly random centre, and the noise seed.
    Returns dicts with keys shape, G, tau_A, tau_B, R, centre, seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for k in range(n):
        L = int(sizes[int(rng.integers(len(sizes)))])
        g_rho = float(rng.uniform(2.2, 2.8))
        tau_A = float(rng.uniform(0.6, 1.5))
        tau_B = float(rng.uniform(0.6, 1.5))
        R = float(rng.uniform(L / 8.0, L / 3.0))
        centre = tuple(float(c) for c in rng.uniform(0.0, L, size=dim))
        specs.append(dict(shape=(L,) * dim, G=g_rho / RHO_TOT, tau_A=tau_A, tau_B=tau_B, R=R, centre=centre,
                          seed=int(seed) * 1000003 + k))
    return specs


def spec_fields(spec, dtype=np.float64):
    """Initial (rho_A, rho_B) of one ragged_drop_specs entry."""
    return drop(spec["shape"], spec["R"], centre=spec["centre"], seed=spec["seed"], dtype=dtype)
