"""The free-energy two-population model (Sec. 2.2, Eqs. FE1 / FE2 with the
Eq. FEtau functional; lbm_model LBM_MODEL_FE) on the CUDA path, against the
FP64 oracle (oracle.OracleFE), through the C ABI.

Tolerances as in test_gpu_parity (FP64 1e-12 per field; FP32 1e-5 on the
densities, 1e-3 on u relative to max(max|u|, 1e-3)).  The FE model runs on the
kernels that choose the collision at run time (tile kinds 0 and 3, the
z-marching batch tiles) and on the TMA tile 34 (a compile-time FE instance);
all of them give bit-identical fields.  The workload recipe is a drop of
rho_A = 0.9 in rho_B = 0.14 (phi = +-0.76, the coexistence of g = 2.5 at
rho = 1.04), well inside |phi| < rho where the logarithm of the functional
lives.
"""
import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0
G_FE = 2.5


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


def _drop(shape, seed):
    return inputs.drop(shape, min(shape[-2:]) / 4.0, rho_hi=0.9, rho_lo=0.14, seed=seed)


def test_fe_drop_d2q9_f64(sc, oracle_mod):
    """64^2 drop, tau = 0.9, tau_g = 1.1, Gamma = 0.5, 500 steps: every field to 1e-12."""
    f = _drop((64, 64), 0)
    lat = sc.FELattice(0, (64, 64), 0.9, 1.1, G_FE, "f64", gamma=0.5).init(*f).step(500)
    o = oracle_mod.OracleFE(0, (64, 64), 0.9, 1.1, G_FE, gamma=0.5).init(*f).step(500)
    g = _fields(lat)
    a, b, u, p = o.moments()
    for name, x, y in zip(("rhoA", "rhoB", "u", "p"), g, (a, b, u[..., :2], p)):
        assert _rel(x, y, 1e-3 if name == "u" else 1e-300) < 1e-12, name
    d = lat.diagnostics()
    assert abs(d["mass_A"] + d["mass_B"] - (f[0] + f[1]).sum()) < 1e-10 * (f[0] + f[1]).sum()


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_fe_d3q19_ragged(sc, oracle_mod, precision, tol):
    shape = (28, 36, 44)
    f = _drop(shape, 21)
    lat = sc.FELattice(1, shape, 1.0, 0.8, G_FE, precision, gamma=0.7).init(*f).step(60)
    o = oracle_mod.OracleFE(1, shape, 1.0, 0.8, G_FE, gamma=0.7).init(*f).step(60)
    g = _fields(lat)
    a, b, u, _ = o.moments()
    assert _rel(g[0], a) < tol and _rel(g[1], b) < tol
    assert _rel(g[2], u, 1e-3) < (1e-3 if precision == "f32" else 1e-12)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_fe_every_launch_shape_bit_identical(sc, precision):
    shape = (40, 32, 70)
    f = _drop(shape, 12)
    probe = sc.FELattice(1, shape, 0.9, 1.1, G_FE, precision)
    tiles = [t for t in range(len(sc.TILES)) if probe.tile_fits(t)]
    assert set(sc.TILE_KIND[t] for t in tiles) <= {0, 3, 5} and (34 in tiles) == (precision == "f32")
    ref = None
    for tile in tiles:
        for z in (0, 40):
            got = _fields(sc.FELattice(1, shape, 0.9, 1.1, G_FE, precision).init(*f).set_tuning(tile, z).step(6))
            if ref is None:
                ref = got
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), (tile, z)


def test_fe_and_sc_lattices_in_one_batch(sc):
    """FE and SC lattices mixed in the z-marching batch tiles equal solo steps
    bitwise; the TMA batch tiles refuse a batch with an FE lattice."""
    mix = [((40, 20, 48), "fe"), ((17, 33, 70), "sc"), ((20, 16, 32), "fe"), ((9, 12, 128), "sc")]

    def make():
        out = []
        for k, (shape, m) in enumerate(mix):
            rA, rB = _drop(shape, k)
            if m == "fe":
                out.append(sc.FELattice(1, shape, 1.0, 0.9, G_FE, "f32", gamma=0.6).init(rA, rB))
            else:
                out.append(sc.Lattice(1, shape, 1.0, 1.0, 2.0, "f32").init(rA, rB))
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


def test_fe_matches_the_sc_spinodal_rate_on_gpu(sc):
    """The matching of Sec. 2.3 on the CUDA path (FP64): the FE model with g = g_tau
    and Gamma (tau_g - 1/2) = rho (tau - 1/2) decays a small phi mode at the rate
    of the SC linear theory, and so does the SC model itself."""
    L, rho, tau, tau_g, gt = 64, 1.0, 0.7, 1.0, 1.5
    k = 2 * np.pi / L
    theory = rho * (tau - 0.5) * (CS2 * (1 / rho - gt / 2) * k * k + gt / 4 * CS2 * CS2 * k ** 4)
    rA, rB = inputs.phi_mode((4, L), rho, 1e-4)
    lats = {"fe": sc.FELattice(0, (4, L), tau, tau_g, gt, "f64", gamma=rho * (tau - 0.5) / (tau_g - 0.5)),
            "sc": sc.Lattice(0, (4, L), tau, tau, gt * (tau - 0.5) / tau, "f64")}
    for name, lat in lats.items():
        m = _fields(lat.init(rA, rB).step(100))
        a1 = _mode_amp(m[0] - m[1], 1)
        m = _fields(lat.step(1000))
        a2 = _mode_amp(m[0] - m[1], 1)
        assert abs(np.log(a1 / a2) / 1000.0 / theory - 1) < 1e-2, name


def test_d2q9_batch_mixes_every_model_and_forcing(sc):
    """One D2Q9 batch (z-marching batch tiles) holding an SC lattice, a
    Kolmogorov-forced one, a Guo-forced one and an FE one, FP32 and FP64:
    bitwise equal to stepping each alone."""
    shapes = [(48, 64), (37, 50), (64, 40), (30, 72)]

    def make(prec):
        out = []
        for k, shape in enumerate(shapes):
            if k == 3:
                rA, rB = _drop(shape, k)
                out.append(sc.FELattice(0, shape, 0.9, 1.1, G_FE, prec, gamma=0.5).init(rA, rB))
                continue
            rA, rB = inputs.drop(shape, min(shape) / 4.0, seed=k)
            kw = [{}, {"body_A": 2e-5}, {"forcing": "guo", "body_A": -1e-5}][k]
            out.append(sc.Lattice(0, shape, 1.0, 0.8, 2.3, prec, **kw).init(rA, rB))
        return out
    for prec in ("f32", "f64"):
        solo = make(prec)
        for lat in solo:
            lat.step(17)
        ref = [_fields(lat) for lat in solo]
        tiles = [t for t in range(len(sc.BATCH_TILES)) if all(sc.batch_tile_fits(t, lat) for lat in solo)]
        assert tiles == [t for t in range(len(sc.BATCH_TILES)) if not sc.BATCH_TILE_TMA[t]]
        for tile in tiles:
            lats = make(prec)
            b = sc.Batch(lats, tile=tile)
            b.step(9).step(8)
            for k, lat in enumerate(lats):
                for x, y in zip(_fields(lat), ref[k]):
                    assert np.array_equal(x, y), (prec, tile, k)
            b.close()


def test_fe_laplace_batch_on_gpu(sc):
    """Five FE drops (R = 12..32 on 128^2, FP32) advanced as one ragged batch for
    6000 steps: the bulk pressure jump follows Laplace's law dP = sigma / R
    (R^2 > 0.999, intercept below 5 % of sigma / 8), as the oracle's FE model does."""
    L, radii = 128, (12, 16, 20, 26, 32)
    lats, fields = [], []
    for R in radii:
        rA, rB = inputs.drop((L, L), R, rho_hi=0.9, rho_lo=0.14, seed=0, noise=0.0)
        lats.append(sc.FELattice(0, (L, L), 1.0, 1.0, G_FE, "f32", gamma=1.0).init(rA, rB))
    b = sc.Batch(lats, tile=1)
    b.step(6000)
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    r = np.hypot(x - L / 2, y - L / 2)
    inv, dps = [], []
    for R, lat in zip(radii, lats):
        a, _, _, p = _fields(lat)
        rin, rout = a[r < R / 4].mean(), a[r > R + 8].mean()
        Req = np.sqrt((a - rout).sum() / (rin - rout) / np.pi)
        inv.append(1 / Req)
        dps.append(p[r < Req / 4].mean() - p[r > Req + 8].mean())
    b.close()
    A = np.vstack([inv, np.ones(len(inv))]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, np.array(dps), rcond=None)
    pred = A @ [slope, icpt]
    r2 = 1 - ((np.array(dps) - pred) ** 2).sum() / ((np.array(dps) - np.mean(dps)) ** 2).sum()
    assert slope > 0 and r2 > 0.999 and abs(icpt) < 0.05 * slope / 8, (slope, icpt, r2)
