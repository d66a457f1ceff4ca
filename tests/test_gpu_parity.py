"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative error per field = max|gpu - oracle| / max|oracle|; the
velocity is compared in the max norm relative to max(max|u_oracle|, 1e-3):
a pointwise relative error is meaningless near u = 0, and the velocity is a
difference of O(rho) population sums, so its round-off is absolute, about
1e-16 lattice units in FP64, whatever the flow speed):
  * FP64 GPU build: 1e-12 per field (after 1000 steps on the 64^2 drop);
  * FP32: 1e-5 on the densities, mass drift < 1e-6 (FP64 diagnostics).
Inputs are the seeded drop / slab recipes of paper_1112_5547_gb300.inputs.
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


def _rel(a, b, floor=1e-300):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


U_FLOOR = 1e-3


def _rel_field(name, a, b):
    return _rel(a, b, U_FLOOR if name == "u" else 1e-300)


def _gpu_fields(lat):
    rA, rB, u, p = lat.moments()
    import torch
    torch.cuda.synchronize()
    return [t.double().cpu().numpy() for t in (rA, rB, u, p)]


def _run_pair(sc, oracle_mod, lattice, shape, tau_A, tau_B, G, steps, precision, fields, u=None):
    rA, rB = fields
    lat = sc.Lattice(lattice, shape, tau_A, tau_B, G, precision).init(rA, rB, u).step(steps)
    g = _gpu_fields(lat)
    o = oracle_mod.OracleSC(lattice, shape, tau_A, tau_B, G).init(rA, rB, u).step(steps)
    a, b, uo, po = o.moments()
    D = 2 if lattice == 0 else 3
    return g, (a, b, uo[..., :D], po), lat


def test_cfg0_f64_1000_steps(sc, oracle_mod):
    """64^2 D2Q9 drop R=16, tau=1, G rho_tot = 2.4, +-1e-3 noise: FP64 to 1e-12 per field."""
    f = inputs.drop((64, 64), 16, centre=(32, 32), seed=0)
    g, o, _ = _run_pair(sc, oracle_mod, 0, (64, 64), 1.0, 1.0, G0, 1000, "f64", f)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-12, name


def test_cfg0_f32_1000_steps(sc, oracle_mod):
    f = inputs.drop((64, 64), 16, centre=(32, 32), seed=0)
    g, o, lat = _run_pair(sc, oracle_mod, 0, (64, 64), 1.0, 1.0, G0, 1000, "f32", f)
    assert _rel(g[0], o[0]) < 1e-5
    assert _rel(g[1], o[1]) < 1e-5
    d = lat.diagnostics()
    m0A, m0B = f[0].sum(), f[1].sum()
    assert abs(d["mass_A"] - m0A) / m0A < 1e-6
    assert abs(d["mass_B"] - m0B) / m0B < 1e-6


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_d3q19_ragged_tiles(sc, oracle_mod, precision, tol):
    """D3Q19 on 37 x 19 x 20: two x tiles, three y tiles, all ragged, several z chunks."""
    shape = (20, 19, 37)
    f = inputs.drop(shape, 6, centre=(14.0, 9.5, 8.0), seed=5)
    g, o, _ = _run_pair(sc, oracle_mod, 1, shape, 0.8, 1.2, 2.0, 200, precision, f)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        t = tol if name != "u" else (1e-12 if precision == "f64" else 1e-3)
        assert _rel_field(name, a, b) < t, name


def test_d2q9_ragged_f64(sc, oracle_mod):
    shape = (70, 100)
    f = inputs.drop(shape, 15, centre=(40.0, 30.0), seed=6)
    g, o, _ = _run_pair(sc, oracle_mod, 0, shape, 1.3, 0.7, 2.2, 300, "f64", f)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-12, name


@pytest.mark.parametrize("lattice,shape", [(0, (4, 4)), (0, (1, 5)), (1, (7, 3, 5)), (1, (1, 4, 6)), (1, (3, 1, 1))])
def test_tiny_and_degenerate_lattices(sc, oracle_mod, lattice, shape):
    """Lattices smaller than one tile, and one-node-thick periodic directions."""
    rng = np.random.default_rng(9)
    rA = 0.5 + 0.3 * rng.random(shape)
    rB = 0.5 + 0.3 * rng.random(shape)
    g, o, _ = _run_pair(sc, oracle_mod, lattice, shape, 0.9, 1.1, 1.5, 30, "f64", (rA, rB))
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-12, name


def test_moving_start_and_unequal_tau(sc, oracle_mod):
    shape = (12, 16, 18)
    f = inputs.drop(shape, 4, seed=8, noise=1e-2)
    rng = np.random.default_rng(3)
    u = rng.uniform(-0.03, 0.03, size=shape + (3,))
    g, o, _ = _run_pair(sc, oracle_mod, 1, shape, 0.6, 1.5, 1.7, 100, "f64", f, u=u)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-12, name


def test_zero_coupling_and_zero_steps(sc, oracle_mod):
    shape = (9, 33)
    f = inputs.drop(shape, 3, seed=1)
    g, o, _ = _run_pair(sc, oracle_mod, 0, shape, 1.0, 1.0, 0.0, 50, "f64", f)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-12, name
    g, o, _ = _run_pair(sc, oracle_mod, 0, shape, 1.0, 1.0, 1.0, 0, "f64", f)
    for name, a, b in zip(("rhoA", "rhoB", "u", "p"), g, o):
        assert _rel_field(name, a, b) < 1e-13, name


def test_translation_equivariance_bitwise_gpu(sc):
    """A shift that is not a multiple of the 32 x 8 tile moves tile seams relative to the
    drop; per-node arithmetic is fixed, so the result shifts bitwise."""
    shape = (24, 21, 45)
    f = inputs.drop(shape, 6, seed=2)
    roll = (5, 3, 11)
    a = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32").init(*f).step(40)
    b = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32").init(*(np.roll(x, roll, (0, 1, 2)) for x in f)).step(40)
    for x, y in zip(_gpu_fields(a), _gpu_fields(b)):
        assert np.array_equal(np.roll(x, roll, (0, 1, 2)), y)


def test_uniform_state_stays_uniform(sc):
    shape = (6, 10, 40)
    lat = sc.Lattice(1, shape, 0.8, 1.2, 2.0, "f32").init(np.full(shape, 0.7), np.full(shape, 0.4)).step(20)
    rA, rB, u, p = _gpu_fields(lat)
    assert np.abs(rA - 0.7).max() < 1e-6 and np.abs(rB - 0.4).max() < 1e-6
    assert np.abs(u).max() < 1e-7


def test_diagnostics_match_oracle_fields(sc, oracle_mod):
    shape = (48, 56)
    f = inputs.drop(shape, 12, centre=(28.0, 24.0), seed=4)
    lat = sc.Lattice(0, shape, 1.0, 1.0, G0, "f64").init(*f).step(200)
    win = sc.Window((28.0, 24.0), 3.0, 20.0)
    d = lat.diagnostics(win)
    o = oracle_mod.OracleSC(0, shape, 1.0, 1.0, G0).init(*f).step(200)
    a, b, u, p = o.moments()
    rho = a + b
    sp = np.sqrt((u ** 2).sum(-1))
    assert abs(d["mass_A"] - a.sum()) < 1e-10 * a.sum()
    assert abs(d["mass_B"] - b.sum()) < 1e-10 * b.sum()
    np.testing.assert_allclose(d["momentum"][:2], (u[..., :2] * rho[..., None]).sum((0, 1)), atol=1e-11)
    assert abs(d["max_speed"] - sp.max()) < 1e-12
    assert abs(d["kinetic_energy"] - 0.5 * (rho * sp ** 2).sum()) < 1e-12 * max(1.0, d["kinetic_energy"])
    assert d["min_rho_A"] == pytest.approx(a.min(), abs=1e-13)
    assert d["min_rho_B"] == pytest.approx(b.min(), abs=1e-13)
    r = inputs.radial_distance(shape, (28.0, 24.0))
    assert d["in_count"] == (r < 3.0).sum() and d["out_count"] == (r > 20.0).sum()
    assert d["in_p"] == pytest.approx(p[r < 3.0].sum(), rel=1e-12)
    assert d["out_rho_A"] == pytest.approx(a[r > 20.0].sum(), rel=1e-12)
    assert d["status"] == sc.LBM_OK


@pytest.mark.parametrize("shape,with_u", [((16, 20, 24), False), ((100, 12, 40), True), ((256, 8, 32), False)])
def test_run_host_equals_device_path(sc, shape, with_u):
    """lbm_sc_run_host (host buffers, copies inside) gives the device path's result bitwise,
    also when its copies overlap the kernels in z slabs (64 planes or more: 100 planes make
    4 slabs of whole 32-plane chunks and a ragged last one, 256 planes the full 8), with and
    without an initial velocity, and on two calls in a row."""
    import torch
    rA, rB = inputs.drop(shape, 5, seed=3, dtype=np.float32)
    u0 = (1e-3 * np.random.default_rng(4).standard_normal(shape + (3,))).astype(np.float32) if with_u else None
    dev = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32").init(rA, rB, u0).step(25)
    ref = _gpu_fields(dev)
    lat = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32")
    nbytes = sc.lbm_sc_host_staging_bytes(lat.params)
    staging = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    sp = (staging.data_ptr() + 255) // 256 * 256
    hA = torch.from_numpy(rA.reshape(-1)).pin_memory()
    hB = torch.from_numpy(rB.reshape(-1)).pin_memory()
    N = rA.size
    oA, oB, oP = (torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(3))
    oU = torch.empty(3 * N, dtype=torch.float32).pin_memory()
    hU = torch.from_numpy(np.ascontiguousarray(np.moveaxis(u0, -1, 0)).reshape(-1)).pin_memory() if with_u else None
    for _ in range(2):
        for t in (oA, oB, oP, oU):
            t.fill_(-1.0)
        sc.lbm_sc_run_host(lat.handle, sp, nbytes, hA.data_ptr(), hB.data_ptr(), hU.data_ptr() if with_u else None,
                           25, oA.data_ptr(), oB.data_ptr(), oU.data_ptr(), oP.data_ptr())
        assert np.array_equal(oA.numpy().reshape(shape), ref[0].astype(np.float32))
        assert np.array_equal(oB.numpy().reshape(shape), ref[1].astype(np.float32))
        assert np.array_equal(oU.numpy().reshape(3, -1).T.reshape(shape + (3,)), ref[2].astype(np.float32))
        assert np.array_equal(oP.numpy().reshape(shape), ref[3].astype(np.float32))


def test_run_host_with_library_host_buffers(sc):
    """lbm_sc_run_host on buffers of lbm_sc_host_alloc (driver-allocated, page-locked)
    gives the device path's result bitwise; the buffers arrive zero-filled and are
    usable to their last byte."""
    import torch
    shape = (72, 16, 40)
    rA, rB = inputs.drop(shape, 6, seed=5, dtype=np.float32)
    ref = _gpu_fields(sc.Lattice(1, shape, 1.0, 1.0, G0, "f32").init(rA, rB).step(12))
    lat = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32")
    nbytes = sc.lbm_sc_host_staging_bytes(lat.params)
    staging = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    sp = (staging.data_ptr() + 255) // 256 * 256
    N = rA.size
    bufs = [sc.HostBuffer(n) for n in (N, N, N, N, 3 * N, N)]
    hA, hB, oA, oB, oU, oP = (b.tensor for b in bufs)
    assert all(not t.any() for t in (hA, oU))
    hA.copy_(torch.from_numpy(rA.reshape(-1)))
    hB.copy_(torch.from_numpy(rB.reshape(-1)))
    sc.lbm_sc_run_host(lat.handle, sp, nbytes, hA.data_ptr(), hB.data_ptr(), None, 12, oA.data_ptr(),
                       oB.data_ptr(), oU.data_ptr(), oP.data_ptr())
    assert np.array_equal(oA.numpy().reshape(shape), ref[0].astype(np.float32))
    assert np.array_equal(oB.numpy().reshape(shape), ref[1].astype(np.float32))
    assert np.array_equal(oU.numpy().reshape(3, -1).T.reshape(shape + (3,)), ref[2].astype(np.float32))
    assert np.array_equal(oP.numpy().reshape(shape), ref[3].astype(np.float32))
    for b in bufs:
        b.close()
    big = sc.HostBuffer(3 * N + 5)  # not a whole number of granules
    big.tensor[-1] = 2.0
    assert big.tensor[-1] == 2.0 and not big.tensor[:-1].any()
    big.close()


def test_unstable_state_reported(sc):
    """A negative density in the initial fields is reported as LBM_ERR_UNSTABLE."""
    shape = (8, 8)
    rA = np.full(shape, 0.5)
    rA[3, 3] = -0.1
    lat = sc.Lattice(0, shape, 1.0, 1.0, 1.0, "f32").init(rA, np.full(shape, 0.5))
    d = lat.diagnostics(check=False)
    assert d["status"] == sc.LBM_ERR_UNSTABLE
    rA[3, 3] = np.nan
    lat = sc.Lattice(0, shape, 1.0, 1.0, 1.0, "f32").init(rA, np.full(shape, 0.5))
    d = lat.diagnostics(check=False)
    assert d["status"] == sc.LBM_ERR_UNSTABLE and d["nonfinite"] >= 1


@pytest.mark.parametrize("precision", ["f32", "bf16", "f64", "bf16_rest", "f16_rest"])
def test_every_launch_shape_is_bit_identical(sc, precision):
    """The step kernel's tile, kernel kind and z-chunk change only speed: all shapes agree bitwise."""
    shape = (40, 32, 70)  # 32 rows: the clustered TMA tiles (pairs and quads of y tiles) fit too
    f = inputs.drop(shape, 8, seed=12)
    ref = None
    probe = sc.Lattice(1, shape, 0.9, 1.1, G0, precision, 0.5, 0.5)
    tiles = [t for t in range(len(sc.TILES)) if probe.tile_fits(t)]
    assert any(sc.TILE_KIND[t] == 5 for t in tiles) == (precision == "f32")
    assert any(sc.TILE_KIND[t] == 6 for t in tiles) == (precision in ("bf16", "bf16_rest", "f16_rest"))
    for tile in tiles:
        for z in (0, 7, 40):
            lat = sc.Lattice(1, shape, 0.9, 1.1, G0, precision, 0.5, 0.5).init(*f).set_tuning(tile, z).step(6)
            got = _gpu_fields(lat)
            if ref is None:
                ref = got
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (tile, z)


def test_autotuner_restores_state(sc):
    from paper_1112_5547_gb300 import autotune
    shape = (32, 24, 40)
    f = inputs.drop(shape, 7, seed=13)
    a = sc.Lattice(1, shape, 1.0, 1.0, G0, "f32").init(*f).step(3)
    before = _gpu_fields(a)
    best, table = autotune.autotune(a, trial_steps=2, warmup_steps=2)
    assert len(table) == len(autotune.candidates(a))
    after = _gpu_fields(a)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    assert a.tuning() == (best[0], best[1])
