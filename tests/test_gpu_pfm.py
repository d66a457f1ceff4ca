"""The pseudo-spectral phase-field model of Sec. 3 on the GPU (libpfm.so,
include/pfm.h: cuFFT transforms, the library's spectral and physical-space
kernels) against the FP64 numpy oracle (oracle.OraclePFM).

Tolerances: FP64 1e-10 relative to the field's maximum (the two sides use
different FFT algorithms, whose rounding differs at 1e-16 per transform and
grows through the nonlinear terms); FP32 1e-5 on phi and 1e-3 of max|u| on u.
Drops use rho = 1.4 with rho_A 1.2 / rho_B 0.2 (phi = +-1, the paper's Sec. 4
example), tau = 0.6, g = 0.3 (g_tau = 1.8) and dt = 0.1: the explicit
logarithmic term of the scheme needs a small step on a two-node interface.
"""
import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO, TAU, G, DT = 1.4, 0.6, 0.3, 0.1


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, phase_field
    build.build()
    return phase_field


def _phi(shape, seed):
    rA, rB = inputs.drop(shape, min(shape) / 4.0, rho_hi=1.2, rho_lo=0.2, seed=seed)
    return rA - rB


def _gpu(s):
    import torch
    phi, u = s.fields()
    torch.cuda.synchronize()
    return phi.double().cpu().numpy(), u.double().cpu().numpy()


def _rel(a, b, floor=1e-300):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


@pytest.mark.parametrize("shape", [(48, 64), (15, 21), (16, 20, 24), (9, 12, 15)])
def test_pfm_f64_vs_oracle(pf, oracle_mod, shape):
    """Even axes (Nyquist modes) and odd ones, 2D and 3D, 60 steps."""
    phi0 = _phi(shape, 3)
    s = pf.PFM(shape, RHO, TAU, G, DT, "f64").init(phi0).step(60)
    o = oracle_mod.OraclePFM(shape, RHO, TAU, G, DT).init(phi0).step(60)
    gp, gu = _gpu(s)
    op, ou = o.fields()
    assert _rel(gp, op) < 1e-10
    assert _rel(gu, ou) < 1e-9
    assert np.abs(ou).max() > 1e-6  # the capillary force has moved the fluid


def test_pfm_f32_vs_oracle(pf, oracle_mod):
    shape = (16, 20, 24)
    phi0 = _phi(shape, 4)
    s = pf.PFM(shape, RHO, TAU, G, DT, "f32").init(phi0).step(40)
    o = oracle_mod.OraclePFM(shape, RHO, TAU, G, DT).init(phi0).step(40)
    gp, gu = _gpu(s)
    op, ou = o.fields()
    assert np.abs(gp - op).max() < 1e-5
    assert np.abs(gu - ou).max() < 1e-3 * np.abs(ou).max()


def test_pfm_linear_mode_and_shear_wave_on_gpu(pf):
    """The closed forms pinned on the oracle, on the CUDA path (FP64): a small phi
    mode follows the AB2/CN recurrence, a shear wave decays by the CN factor."""
    L, rho, tau, g, dt, eps = 64, 1.0, 0.8, 1.0, 1.0, 1e-6
    x = np.arange(L)
    sn = np.sin(2 * np.pi * x / L)
    s = pf.PFM((4, L), rho, tau, g, dt, "f64").init(eps * np.broadcast_to(sn, (4, L)))
    amps = []
    for _ in range(40):
        amps.append(2 * (_gpu(s.step(1))[0] * sn).mean())
    cs2, k2 = 1 / 3, (2 * np.pi / L) ** 2
    g_tau = tau * g / (tau - 0.5)
    D, xi2 = rho * (tau - 0.5) * g_tau * cs2 / 2, cs2 / 2
    lam = D * (2 * k2 + dt * D / 2 * k2 * k2)
    sig = -D * k2 * (2 / (g_tau * rho) - 3) - D * (xi2 - dt * D / 2) * k2 * k2
    a_prev = a = eps
    rec = []
    for _ in range(40):
        a_prev, a = a, (a * (1 - dt * lam / 2) + dt * (3 * sig * a - sig * a_prev) / 2) / (1 + dt * lam / 2)
        rec.append(a)
    assert np.abs(np.array(amps) - rec).max() < 1e-11 * eps
    u = np.zeros((L, 4, 2))
    u[..., 0] = 1e-3 * np.sin(2 * np.pi * x / L)[:, None]
    s = pf.PFM((L, 4), 1.0, 0.9, 1.0, 0.7, "f64").init(np.zeros((L, 4)), u).step(25)
    nu = cs2 * 0.4
    f = (1 - 0.7 * nu * k2 / 2) / (1 + 0.7 * nu * k2 / 2)
    np.testing.assert_allclose(_gpu(s)[1][..., 0], u[..., 0] * f ** 25, rtol=0, atol=1e-17)


@pytest.mark.slow
def test_pfm_128_whole_field_and_256_invariants(pf, oracle_mod):
    """The bench's PFM configuration: 128^3 FP32 against the oracle on the whole
    field after 5 steps; 256^3 FP32 (the bench size): sum phi conserved and div u = 0
    to FP32 rounding (a field that missed the projection would have |div u| ~ k |u|,
    of order max|u|; FP32 rounding of the transforms leaves ~2e-5 max|u|)."""
    import torch
    shape = (128, 128, 128)
    phi0 = _phi(shape, 5)
    s = pf.PFM(shape, RHO, TAU, G, DT, "f32").init(phi0).step(5)
    o = oracle_mod.OraclePFM(shape, RHO, TAU, G, DT).init(phi0).step(5)
    gp, gu = _gpu(s)
    op, ou = o.fields()
    assert np.abs(gp - op).max() < 1e-5
    assert np.abs(gu - ou).max() < 1e-3 * np.abs(ou).max()
    del s, o
    shape = (256, 256, 256)
    phi0 = _phi(shape, 6).astype(np.float32)
    s = pf.PFM(shape, RHO, TAU, G, DT, "f32").init(phi0).step(20)
    phi, u = s.fields()
    assert abs(float(phi.double().sum()) - float(phi0.astype(np.float64).sum())) < 1e-4 * float(np.abs(phi0).sum())
    uh = [torch.fft.fftn(u[..., a].double()) for a in range(3)]
    k = [2 * np.pi * torch.fft.fftfreq(n, device=u.device, dtype=torch.float64) for n in shape]
    for kk in k:
        kk[len(kk) // 2] = 0.0
    kz, ky, kx = torch.meshgrid(*k, indexing="ij")
    div = torch.fft.ifftn(1j * (kx * uh[0] + ky * uh[1] + kz * uh[2])).real
    assert float(div.abs().max()) < 2e-4 * float(u.abs().max())
    del s, u, uh, div
    torch.cuda.empty_cache()


def test_pfm_kolmogorov_forcing_on_gpu(pf, oracle_mod):
    """The forcing of Eq. kolmo in the PFM (FP64): a forced drop matches the oracle
    (1e-10), and a forced uniform fluid reaches the exact steady profile
    u_x = A sin(k y) / (nu k^2)."""
    shape = (24, 32)
    phi0 = _phi(shape, 7)
    s = pf.PFM(shape, RHO, TAU, G, DT, "f64", body_A=1e-4).init(phi0).step(50)
    o = oracle_mod.OraclePFM(shape, RHO, TAU, G, DT, body_A=1e-4).init(phi0).step(50)
    gp, gu = _gpu(s)
    op, ou = o.fields()
    assert _rel(gp, op) < 1e-10 and _rel(gu, ou) < 1e-9
    A, tau, ny = 1e-6, 0.8, 32
    k, nu = 2 * np.pi / ny, (tau - 0.5) / 3
    s = pf.PFM((ny, 8), 1.4, tau, 0.3, 1.0, "f64", body_A=A).init(np.zeros((ny, 8))).step(int(30 / (nu * k * k)))
    u = _gpu(s)[1]
    expect = A * np.sin(k * np.arange(ny)) / (nu * k * k)
    np.testing.assert_allclose(u[..., 0], np.broadcast_to(expect[:, None], (ny, 8)), rtol=0, atol=1e-9 * expect.max())
