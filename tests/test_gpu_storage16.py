"""16-bit population storage (FP32 arithmetic) against the FP64 oracle on the
drop observables: the mass-equivalent drop radius, the Laplace pressure jump
P_in - P_out and the peak spurious speed max |u_phys|.

Definitions (drop of component A centred in a periodic box):
  rho_in, rho_out = mean rho_A over r < R0/4 and over r > R0 + 8;
  V = sum (rho_A - rho_out) / (rho_in - rho_out),  R = sqrt(V/pi) (2D) or
  (3V/(4 pi))^(1/3) (3D);  P_in, P_out = mean bulk pressure p over r < R/4 and
  r > R + 8 (Sec. 4.1).
Bar: relative error under 1% for each observable with the rest-offset storage
(h = f - w_i rho_s(node), FP32 densities); the reference-offset storage
(h = f - w_i rho_ref) is held to what it reaches, recorded in the bounds below.
"""
import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

G0 = 2.4 / 1.04


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


def drop_observables(rhoA, p, u, R0):
    shape = rhoA.shape
    centre = tuple(n / 2.0 for n in reversed(shape))
    r = inputs.radial_distance(shape, centre)
    rin = rhoA[r < R0 / 4].mean()
    rout = rhoA[r > R0 + 8].mean()
    V = (rhoA - rout).sum() / (rin - rout)
    R = np.sqrt(V / np.pi) if rhoA.ndim == 2 else (3 * V / (4 * np.pi)) ** (1 / 3)
    dP = p[r < R / 4].mean() - p[r > R + 8].mean()
    umax = np.sqrt((u.astype(np.float64) ** 2).sum(-1)).max()
    return np.array([R, dP, umax])


CASES = {
    # lattice, shape, R0, steps
    "d2q9_64": (0, (64, 64), 16, 1000),
    "d3q19_48": (1, (48, 48, 48), 12, 1000),
}
_ref_cache = {}


def _oracle_obs(oracle_mod, case):
    if case not in _ref_cache:
        lattice, shape, R0, steps = CASES[case]
        f = inputs.drop(shape, R0, seed=0)
        o = oracle_mod.OracleSC(lattice, shape, 1.0, 1.0, G0).init(*f).step(steps)
        a, b, u, p = o.moments()
        D = 2 if lattice == 0 else 3
        _ref_cache[case] = drop_observables(a, p, u[..., :D], R0)
    return _ref_cache[case]


def _gpu_obs(sc, case, precision, ref=(1.0, 0.04)):
    import torch
    lattice, shape, R0, steps = CASES[case]
    f = inputs.drop(shape, R0, seed=0)
    lat = sc.Lattice(lattice, shape, 1.0, 1.0, G0, precision, rho_ref_A=ref[0], rho_ref_B=ref[1])
    lat.init(*f).step(steps)
    rA, rB, u, p = lat.moments()
    torch.cuda.synchronize()
    return drop_observables(rA.double().cpu().numpy(), p.double().cpu().numpy(), u.double().cpu().numpy(), R0)


# (precision, bound on the relative error of R, dP, max|u|)
BARS = {
    "f32": (1e-4, 1e-3, 1e-3),
    "bf16_rest": (1e-2, 1e-2, 1e-2),
    "f16_rest": (1e-2, 1e-2, 1e-2),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", sorted(BARS))
def test_drop_observables_vs_oracle(sc, oracle_mod, case, precision):
    o = _oracle_obs(oracle_mod, case)
    g = _gpu_obs(sc, case, precision)
    err = np.abs(g / o - 1.0)
    print(case, precision, "R dP umax rel err", err)
    assert np.all(err < np.array(BARS[precision])), (case, precision, err, o, g)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_reference_offset_storage_error_recorded(sc, oracle_mod, case, precision):
    """The reference-offset 16-bit storage with rho_ref = (1.0, 0.04) does NOT
    meet the 1% bar (its offsets are as large as the density contrast in one
    of the two phases, so the 16-bit rounding error is too): its errors are
    printed for the record, and only bounded here (finite, radius within 10%),
    so that a regression to garbage still fails."""
    o = _oracle_obs(oracle_mod, case)
    g = _gpu_obs(sc, case, precision)
    err = np.abs(g / o - 1.0)
    print(case, precision, "R dP umax rel err", err)
    assert np.all(np.isfinite(g))
    assert err[0] < 0.1
