"""Guo forcing on the CUDA path (the discrete-forcing cure of the tau-dependent
coupling that Sec. 2.3 names; formulas in include/lbm_sc.h, lbm_forcing),
against the FP64 oracle through the C ABI.

Tolerances as in test_gpu_parity (FP64 1e-12 per field; FP32 1e-5 on the
densities, 1e-3 on u_phys relative to max(max|u|, 1e-3)).  Guo forcing runs on
the kernels that choose the collision at run time (tile kinds 0 and 3, the
z-marching batch tiles) and on the 64x6 TMA tile 34; every one of them gives
bit-identical fields.  The paper's point is checked on the GPU too: with Guo
forcing the spinodal decay follows the plain coupling g, with the velocity
shift the tau-modified g_tau.
"""
import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

G0 = 2.4 / 1.04
CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


def _fields(lat):
    import torch
    out = [t.double().cpu().numpy() for t in lat.moments()]
    torch.cuda.synchronize()
    return out


def _rel(a, b, floor=1e-300):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


def test_guo_drop_d2q9_f64(sc, oracle_mod):
    """64^2 drop, unequal tau, G rho_tot = 2.4, 1000 steps: every field to 1e-12."""
    f = inputs.drop((64, 64), 16, centre=(32, 32), seed=0)
    lat = sc.Lattice(0, (64, 64), 0.8, 1.2, G0, "f64", forcing="guo").init(*f).step(1000)
    o = oracle_mod.OracleSC(0, (64, 64), 0.8, 1.2, G0, forcing="guo").init(*f).step(1000)
    g = _fields(lat)
    a, b, u, p = o.moments()
    for name, x, y in zip(("rhoA", "rhoB", "u", "p"), g, (a, b, u[..., :2], p)):
        assert _rel(x, y, 1e-3 if name == "u" else 1e-300) < 1e-12, name
    shift = _fields(sc.Lattice(0, (64, 64), 0.8, 1.2, G0, "f64").init(*f).step(1000))
    assert _rel(shift[0], a) > 1e-4  # the schemes really differ


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_guo_d3q19_ragged_with_body_force(sc, oracle_mod, precision, tol):
    shape = (28, 36, 44)
    f = inputs.drop(shape, 8, seed=21)
    lat = sc.Lattice(1, shape, 0.9, 1.1, G0, precision, body_A=2e-4, forcing="guo").init(*f).step(100)
    o = oracle_mod.OracleSC(1, shape, 0.9, 1.1, G0, body_A=2e-4, forcing="guo").init(*f).step(100)
    g = _fields(lat)
    a, b, u, _ = o.moments()
    assert _rel(g[0], a) < tol and _rel(g[1], b) < tol
    assert _rel(g[2], u, 1e-3) < (1e-3 if precision == "f32" else 1e-12)


@pytest.mark.parametrize("precision", ["f32", "bf16_rest", "f64"])
def test_guo_every_launch_shape_bit_identical(sc, precision):
    shape = (40, 32, 70)
    f = inputs.drop(shape, 8, seed=12)
    probe = sc.Lattice(1, shape, 0.9, 1.1, G0, precision, forcing="guo")
    tiles = [t for t in range(len(sc.TILES)) if probe.tile_fits(t)]
    assert set(sc.TILE_KIND[t] for t in tiles) <= {0, 3, 5}
    assert (34 in tiles) == (precision == "f32")
    assert all(sc.tile_supported(t, 1, probe.params.precision, sc.LBM_FORCING_GUO) for t in tiles)
    ref = None
    for tile in tiles:
        for z in (0, 40):
            lat = sc.Lattice(1, shape, 0.9, 1.1, G0, precision, body_A=3e-5, forcing="guo")
            got = _fields(lat.init(*f).set_tuning(tile, z).step(6))
            if ref is None:
                ref = got
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), (tile, z)


def test_guo_and_shift_lattices_in_one_batch(sc):
    """Guo and shift lattices mixed in the z-marching batch tiles equal solo
    steps bitwise; the TMA batch tiles refuse a batch with a Guo lattice."""
    mix = [((40, 20, 48), 1.0, 1.0, G0, "guo"), ((17, 33, 70), 0.8, 1.3, 2.0, "shift"),
           ((20, 16, 32), 1.1, 0.9, 2.2, "guo"), ((9, 12, 128), 1.0, 1.0, G0, "shift")]

    def make():
        out = []
        for k, (shape, tA, tB, G, frc) in enumerate(mix):
            rA, rB = inputs.drop(shape, min(shape) / 4.0, seed=k)
            out.append(sc.Lattice(1, shape, tA, tB, G, "f32", forcing=frc, body_A=1e-5 * k).init(rA, rB))
        return out
    solo = make()
    for lat in solo:
        lat.step(9)
    ref = [_fields(lat) for lat in solo]
    tiles = [t for t in range(len(sc.BATCH_TILES)) if all(sc.batch_tile_fits(t, lat) for lat in solo)]
    assert tiles == [t for t in range(len(sc.BATCH_TILES)) if not sc.BATCH_TILE_TMA[t]]
    for tile in tiles:
        lats = make()
        b = sc.Batch(lats, tile=tile, zchunk=8)
        b.step(4).step(5)
        for k, lat in enumerate(lats):
            for x, y in zip(_fields(lat), ref[k]):
                assert np.array_equal(x, y), (tile, k)
        b.close()
    with pytest.raises(sc.LbmError):
        sc.Batch(make(), tile=5, zchunk=8)


def _mode_amp(field, axis):
    n = field.shape[axis]
    s = np.sin(2 * np.pi * np.arange(n) / n)
    shape = [1] * field.ndim
    shape[axis] = n
    return 2.0 * (field * s.reshape(shape)).sum() / field.size


@pytest.mark.parametrize("forcing", ["guo", "shift"])
def test_spinodal_rate_on_gpu_follows_the_schemes_coupling(sc, forcing):
    """Sec. 2.3 on the CUDA path (FP64): a small phi mode below the spinodal
    decays at the linear-theory rate with the plain g under Guo forcing and
    with g_tau = tau g / (tau - 1/2) under the velocity shift (tau = 0.7,
    g = 1.0: the two predictions differ by 70 %)."""
    L, rho, tau, g = 64, 1.0, 0.7, 1.0
    rA, rB = inputs.phi_mode((4, L), rho, 1e-4)
    lat = sc.Lattice(0, (4, L), tau, tau, g, "f64", forcing=forcing).init(rA, rB).step(100)
    m = _fields(lat)
    a1 = _mode_amp(m[0] - m[1], 1)
    m = _fields(lat.step(1000))
    a2 = _mode_amp(m[0] - m[1], 1)
    k = 2 * np.pi / L
    rate = np.log(a1 / a2) / 1000.0
    gg = g if forcing == "guo" else tau * g / (tau - 0.5)
    theory = rho * (tau - 0.5) * (CS2 * (1 / rho - gg / 2) * k * k + gg / 4 * CS2 * CS2 * k ** 4)
    assert abs(rate / theory - 1) < 1e-2
