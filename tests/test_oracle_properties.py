"""Randomised checks of the FP64 oracle (hypothesis): over random small lattices,
relaxation times, couplings, forcing schemes and densities, one oracle step
equals the independent exact rational trace (tests/exact_sc.py), and several
steps conserve each species' mass and the total momentum.  They widen the
fixed-parameter pins of test_oracle_pins.py to the whole parameter range."""
from fractions import Fraction

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from tests import exact_sc  # noqa: E402

taus = st.sampled_from([Fraction(11, 20), Fraction(3, 5), Fraction(4, 5), Fraction(1), Fraction(3, 2), Fraction(2)])
couplings = st.sampled_from([Fraction(0), Fraction(1, 2), Fraction(3, 2), Fraction(5, 2), Fraction(-1, 2)])


@settings(max_examples=25, deadline=None, derandomize=True)
@given(nx=st.integers(1, 4), ny=st.sampled_from([1, 2, 4]), tau_A=taus, tau_B=taus, G=couplings,
       A=st.sampled_from([Fraction(0), Fraction(1, 40), Fraction(-1, 25)]), guo=st.booleans(),
       seed=st.integers(0, 10 ** 6))
def test_one_step_equals_the_exact_trace(oracle_mod, nx, ny, tau_A, tau_B, G, A, guo, seed):
    rng = np.random.default_rng(seed)
    nums = rng.integers(2, 40, size=(2, ny, nx))
    rA = [[Fraction(int(nums[0, y, x]), 20) for x in range(nx)] for y in range(ny)]
    rB = [[Fraction(int(nums[1, y, x]), 25) for x in range(nx)] for y in range(ny)]
    ex = exact_sc.ExactSC(nx, ny, tau_A, tau_B, G, body_A=A, guo=guo).init(rA, rB).step()
    o = oracle_mod.OracleSC(0, (ny, nx), float(tau_A), float(tau_B), float(G), body_A=float(A),
                            forcing="guo" if guo else "shift")
    o.init(np.array(rA, dtype=float), np.array(rB, dtype=float)).step(1)
    a, b, u, p = o.moments()
    eA, eB, eux, euy, ep = (np.array([float(v) for v in arr]).reshape(ny, nx) for arr in ex.fields())
    np.testing.assert_allclose(a, eA, rtol=1e-14, atol=0)
    np.testing.assert_allclose(b, eB, rtol=1e-14, atol=0)
    np.testing.assert_allclose(u[..., 0], eux, rtol=0, atol=1e-13)
    np.testing.assert_allclose(u[..., 1], euy, rtol=0, atol=1e-13)
    np.testing.assert_allclose(p, ep, rtol=1e-14, atol=0)


@settings(max_examples=12, deadline=None, derandomize=True)
@given(nx=st.integers(1, 3), ny=st.sampled_from([1, 2, 4]), nz=st.integers(1, 3), tau_A=taus, tau_B=taus,
       G=couplings, A=st.sampled_from([Fraction(0), Fraction(1, 40)]), guo=st.booleans(),
       seed=st.integers(0, 10 ** 6))
def test_one_d3q19_step_equals_the_exact_trace(oracle_mod, nx, ny, nz, tau_A, tau_B, G, A, guo, seed):
    """The D3Q19 exact trace (tests/exact_sc.py ExactSC3) over random small boxes,
    one-node-thick directions included (a node is then its own periodic image)."""
    rng = np.random.default_rng(seed)
    nums = rng.integers(2, 40, size=(2, nz, ny, nx))
    rA = [[[Fraction(int(nums[0, z, y, x]), 20) for x in range(nx)] for y in range(ny)] for z in range(nz)]
    rB = [[[Fraction(int(nums[1, z, y, x]), 25) for x in range(nx)] for y in range(ny)] for z in range(nz)]
    ex = exact_sc.ExactSC3(nx, ny, nz, tau_A, tau_B, G, body_A=A, guo=guo).init(rA, rB).step()
    o = oracle_mod.OracleSC(1, (nz, ny, nx), float(tau_A), float(tau_B), float(G), body_A=float(A),
                            forcing="guo" if guo else "shift")
    o.init(np.array(rA, dtype=float), np.array(rB, dtype=float)).step(1)
    a, b, u, p = o.moments()
    ex_f = [np.array([float(v) for v in arr]).reshape(nz, ny, nx) for arr in ex.fields()]
    np.testing.assert_allclose(a, ex_f[0], rtol=1e-14, atol=0)
    np.testing.assert_allclose(b, ex_f[1], rtol=1e-14, atol=0)
    for k in range(3):
        np.testing.assert_allclose(u[..., k], ex_f[2 + k], rtol=0, atol=1e-13)
    np.testing.assert_allclose(p, ex_f[5], rtol=1e-14, atol=0)


@settings(max_examples=20, deadline=None, derandomize=True)
@given(lat=st.sampled_from([0, 1]), n=st.integers(3, 7), tau_A=st.floats(0.55, 2.0), tau_B=st.floats(0.55, 2.0),
       G=st.floats(-0.5, 2.5), guo=st.booleans(), seed=st.integers(0, 10 ** 6))
def test_mass_and_momentum_conservation(oracle_mod, lat, n, tau_A, tau_B, G, guo, seed):
    rng = np.random.default_rng(seed)
    shape = (n, n + 1) if lat == 0 else (n, n + 1, n + 2)
    rA = 0.3 + rng.random(shape)
    rB = 0.3 + rng.random(shape)
    o = oracle_mod.OracleSC(lat, shape, tau_A, tau_B, G, forcing="guo" if guo else "shift").init(rA, rB)
    m0 = o.total_momentum()
    o.step(5)
    a, b, _, _ = o.moments()
    assert abs(a.sum() / rA.sum() - 1) < 1e-13 and abs(b.sum() / rB.sum() - 1) < 1e-13
    assert np.abs(o.total_momentum() - m0).max() < 1e-12 * (rA.sum() + rB.sum())


@settings(max_examples=15, deadline=None, derandomize=True)
@given(L=st.sampled_from([8, 12, 16, 24, 32]), mode=st.integers(1, 3), tau=st.floats(0.55, 1.5),
       g=st.floats(0.05, 1.5), dt=st.sampled_from([0.05, 0.2, 0.5, 1.0]))
def test_pfm_linear_modes_follow_the_scheme_recurrence(L, mode, tau, g, dt):
    """Any small phi mode of the PFM at rest follows the two-level recurrence of
    Eqs. eq11-eq13 (see test_pfm_linear_mode_follows_the_ab2_cn_recurrence_and_the_sc_rate).

    The oracle is nonlinear; the recurrence is its linearisation, so the two
    differ by an amount the test derives per draw instead of a fixed tolerance.
    The explicit bracket (1/g_tau) ln((rho + phi)/(rho - phi)) - 3 phi of Eq. eq12
    departs from its linear part by (a) the cubic term of the logarithm,
    (2/3)(eps/rho)^3 / g_tau, and (b) the rounding of the ratio (rho + phi)/(rho - phi)
    near 1 before the logarithm, a few units of 2^-53 absolute, divided by g_tau
    (at eps = 1e-7 that is ~5e-10 of the linear part: a cancellation, not an
    error of the oracle).  Each step passes that bracket error into the mode
    with weight dt D k^2 (|3/2| + |1/2|) / (1 + dt lam / 2), and the recurrence
    carries earlier errors forward by at most the modulus of its larger root per
    step (above 1 where dt makes the explicit part unstable, e.g. the
    sign-alternating mode at dt = 1).  The bound is twice that budget plus
    1e-13 of the amplitude for the transforms; the draws are fixed
    (derandomised) so the check is reproducible, and the budget stays below
    1e-4 of the amplitude over the whole drawn range, so a wrong coefficient
    (an O(1) change of lam or sig) still fails."""
    import oracle
    rho, eps, cs2, steps = 1.0, 1e-7, 1.0 / 3.0, 12
    x = np.arange(L)
    s = np.sin(2 * np.pi * mode * x / L)
    o = oracle.OraclePFM((2, L), rho, tau, g, dt).init(eps * np.broadcast_to(s, (2, L)))
    k2 = (2 * np.pi * mode / L) ** 2
    g_tau = tau * g / (tau - 0.5)
    D, xi2 = rho * (tau - 0.5) * g_tau * cs2 / 2, cs2 / 2
    lam = D * (2 * k2 + dt * D / 2 * k2 * k2)
    sig = -D * k2 * (2 / (g_tau * rho) - 3) - D * (xi2 - dt * D / 2) * k2 * k2
    c1 = (1 - dt * lam / 2 + 1.5 * dt * sig) / (1 + dt * lam / 2)
    c0 = -0.5 * dt * sig / (1 + dt * lam / 2)
    growth = max(1.0, float(np.abs(np.roots([1.0, -c1, -c0])).max()))
    bracket_err = (2.0 / 3.0) * (eps / rho) ** 3 / g_tau + 4 * 2.0 ** -53 / g_tau
    per_step = dt * D * k2 * bracket_err * 2.0 / (1 + dt * lam / 2)
    budget = sum(per_step * growth ** n for n in range(steps))
    a_prev = a = eps
    for _ in range(steps):
        a_prev, a = a, (a * (1 - dt * lam / 2) + dt * (3 * sig * a - sig * a_prev) / 2) / (1 + dt * lam / 2)
        p, _ = o.step(1).fields()
        amp = 2 * (p * s).mean()
        scale = max(abs(a), eps)
        assert budget < 1e-4 * scale
        assert abs(amp - a) <= 2 * budget + 1e-13 * scale, (amp, a, budget)


@settings(max_examples=30, deadline=None, derandomize=True)
@given(lat=st.sampled_from([0, 1]), rho=st.floats(0.5, 2.0), frac=st.floats(-0.9, 0.9),
       g=st.floats(-1.0, 4.0), kappa=st.floats(0.0, 0.2), gamma=st.floats(0.1, 2.0),
       u=st.lists(st.floats(-0.1, 0.1), min_size=3, max_size=3),
       gp=st.lists(st.floats(-0.3, 0.3), min_size=3, max_size=3), lp=st.floats(-0.3, 0.3))
def test_fe_equilibria_meet_the_moment_conditions_everywhere(oracle_mod, lat, rho, frac, g, kappa, gamma, u, gp, lp):
    """Eqs. EQFE1 / EQFE2 over random states (the fixed-state pin, widened)."""
    D = 2 if lat == 0 else 3
    phi = frac * rho
    u, gp = np.array(u[:D]), np.array(gp[:D])
    c, _ = oracle_mod.lattice(lat)
    cc = c[:, :D].astype(float)
    fe, ge = oracle_mod.fe_equilibria(lat, g, kappa, gamma, rho, phi, u, gp, lp)
    cs2 = 1.0 / 3.0
    mu = 0.5 * cs2 * np.log((rho + phi) / (rho - phi)) - 0.5 * g * cs2 * phi - kappa * lp
    pb = cs2 * rho + 0.25 * g * cs2 * (rho * rho - phi * phi)
    P = (pb - kappa * phi * lp - 0.5 * kappa * (gp @ gp)) * np.eye(D) + kappa * np.outer(gp, gp)
    tol = 1e-14 * max(1.0, abs(mu), abs(pb))
    assert abs(fe.sum() - rho) < tol and abs(ge.sum() - phi) < tol
    assert np.abs(fe @ cc - rho * u).max() < tol and np.abs(ge @ cc - phi * u).max() < tol
    assert np.abs(np.einsum("i,ia,ib->ab", fe, cc, cc) - P - rho * np.outer(u, u)).max() < tol
    assert np.abs(np.einsum("i,ia,ib->ab", ge, cc, cc) - gamma * mu * np.eye(D) - phi * np.outer(u, u)).max() < tol
