"""Ragged batch through the C ABI: many lattices of different sizes and
parameters advanced by one launch per step give bit-identical results to
stepping each lattice alone (which the parity tests hold against the oracle),
with and without CUDA-graph chunks, for every batch tile and storage type."""
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


# (shape, tau_A, tau_B, G): ragged sizes (partial tiles, nz below and above the
# z chunk), mixed relaxation times and couplings
MIX3 = [((40, 20, 24), 1.0, 1.0, G0), ((17, 33, 9), 0.8, 1.3, 2.0), ((64, 40, 36), 1.0, 1.0, G0),
        ((5, 7, 6), 1.0, 0.7, 2.5), ((33, 65, 31), 1.2, 1.2, 1.6)]
# lattices every TMA-fed batch tile takes (nx >= 64, ny >= 8), ragged in x and y
MIX3_TMA = [((40, 20, 64), 1.0, 1.0, G0), ((17, 33, 70), 0.8, 1.3, 2.0), ((64, 40, 96), 1.0, 1.0, G0),
            ((5, 8, 64), 1.0, 0.7, 2.5), ((33, 65, 65), 1.2, 1.2, 1.6)]
# TMA-fed tiles of both widths in one batch (tile 9: 64x4 for nx >= 64, else 32x8)
MIX3_MIXED = [((40, 20, 48), 1.0, 1.0, G0), ((17, 33, 70), 0.8, 1.3, 2.0), ((20, 16, 32), 1.1, 0.9, 2.2),
              ((33, 65, 65), 1.2, 1.2, 1.6), ((9, 8, 128), 1.0, 1.0, G0)]
# every lattice at least 32 x 12: the 384-thread batch tiles (10: 32x12; 11: 64x6 or 32x12 per lattice)
MIX3_TALL = [((40, 20, 48), 1.0, 1.0, G0), ((17, 33, 70), 0.8, 1.3, 2.0), ((20, 16, 32), 1.1, 0.9, 2.2),
             ((33, 65, 65), 1.2, 1.2, 1.6), ((9, 12, 128), 1.0, 1.0, G0)]
# batch tile 12 gives each lattice the best of 64x6, 48x8 and 32x12: one lattice of each
MIX3_SHAPE3 = [((12, 64, 64), 1.0, 1.0, G0), ((10, 40, 48), 0.8, 1.3, 2.0), ((9, 24, 32), 1.1, 0.9, 2.2),
               ((20, 17, 96), 1.2, 1.2, 1.6)]
MIX2 = [((64, 64), 1.0, 1.0, G0), ((37, 50), 0.8, 1.3, 2.0), ((7, 130), 1.0, 1.0, 2.2), ((96, 33), 1.1, 0.9, G0)]


def _fields(shape, k):
    return inputs.drop(shape, min(shape) / 4.0, seed=k)


def _make(sc, lattice, mix, precision):
    lats = []
    for k, (shape, tA, tB, G) in enumerate(mix):
        rA, rB = _fields(shape, k)
        lats.append(sc.Lattice(lattice, shape, tA, tB, G, precision).init(rA, rB))
    return lats


def _state(lat):
    import torch
    out = [t.cpu().numpy().copy() for t in lat.moments()]
    torch.cuda.synchronize()
    return out


def _assert_same(a, b, what):
    for x, y in zip(a, b):
        assert np.array_equal(x, y), what


@pytest.mark.parametrize("lattice,mix,precision", [(1, MIX3, "f32"), (0, MIX2, "f64"), (1, MIX3, "bf16"),
                                                   (0, MIX2, "f16"), (1, MIX3_TMA, "f32"),
                                                   (1, MIX3, "bf16_rest"), (0, MIX2, "f16_rest"),
                                                   (1, MIX3_TMA, "bf16_rest"), (1, MIX3_TMA, "f16_rest"),
                                                   (1, MIX3_MIXED, "f32"), (1, MIX3_TALL, "f32"),
                                                   (1, MIX3_SHAPE3, "f32")])
def test_batch_equals_solo(sc, lattice, mix, precision):
    steps = 13
    solo = _make(sc, lattice, mix, precision)
    for lat in solo:
        lat.step(steps)
    ref = [_state(lat) for lat in solo]
    tiles = [t for t in range(len(sc.BATCH_TILES)) if all(sc.batch_tile_fits(t, lat) for lat in solo)]
    if mix is MIX3_TMA and precision == "f32":
        # every FP32 tile of at most 8 rows (one lattice is 8 tall), and tile 12 (48x8 for it)
        assert tiles == [t for t in range(len(sc.BATCH_TILES)) if t != sc.BATCH_TILE_REST
                         and (sc.BATCH_TILES[t][1] <= 8 or t == sc.BATCH_TILE_SHAPE3)]
    if mix is MIX3_TMA and precision.endswith("_rest"):  # the z-marching tiles and the rest-offset TMA tile
        assert tiles == [t for t in range(len(sc.BATCH_TILES))
                         if not sc.BATCH_TILE_TMA[t] or t == sc.BATCH_TILE_REST]
    if mix is MIX3_SHAPE3:
        assert sc.BATCH_TILE_SHAPE3 in tiles
        assert sorted(sc.batch_shape3(shape[2], shape[1]) for shape, *_ in mix[:3]) == [0, 1, 2]
    if mix is MIX3_MIXED:
        assert 9 in tiles
    if mix is MIX3_TALL:
        assert 10 in tiles and 11 in tiles
    for tile in tiles:
        for zchunk in ((0, 8) if lattice == 1 else (0,)):
            lats = _make(sc, lattice, mix, precision)
            b = sc.Batch(lats, tile=tile, zchunk=zchunk)
            b.step(5).step(8)
            for k, lat in enumerate(lats):
                _assert_same(_state(lat), ref[k], (precision, tile, zchunk, k))
            b.close()


def test_batch_graph_chunks(sc):
    """Graph replay (chunks of 4 steps, both starting parities) equals direct launches."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        solo = _make(sc, 1, MIX3, "f32")
        for lat in solo:
            lat.step(23)
        ref = [_state(lat) for lat in solo]
        lats = _make(sc, 1, MIX3, "f32")
        b = sc.Batch(lats, tile=2, zchunk=16, graph_steps=4, stream=stream)
        b.step(7).step(9).step(7)  # 1 graph + 3; parity 1: 2 graphs + 1; parity 0: 1 graph + 3
        stream.synchronize()
        for k, lat in enumerate(lats):
            _assert_same(_state(lat), ref[k], k)
        # the TMA-fed kernel under graph replay
        solo = _make(sc, 1, MIX3_TMA, "f32")
        for lat in solo:
            lat.step(23)
        ref = [_state(lat) for lat in solo]
        for tile in (3, 6):  # persistent over the work counter; one CTA per item
            lats = _make(sc, 1, MIX3_TMA, "f32")
            b = sc.Batch(lats, tile=tile, zchunk=16, graph_steps=4, stream=stream)
            b.step(7).step(9).step(7)
            stream.synchronize()
            for k, lat in enumerate(lats):
                _assert_same(_state(lat), ref[k], ("tma", tile, k))


def test_batch_continues_solo_state(sc):
    """A batch built over lattices that already ran picks up their current buffers;
    after the batch, solo steps continue from the batch's state."""
    a = _make(sc, 1, MIX3[:3], "f32")
    b = _make(sc, 1, MIX3[:3], "f32")
    for lat in a:
        lat.step(10)
    a[0].step(1)  # odd parity on one lattice
    b[0].step(1)
    bt = sc.Batch(a, tile=0)
    bt.step(6)
    bt.close()
    for lat in a:
        lat.step(3)
    for lat in b:
        lat.step(19)
    for x, y in zip(a, b):
        _assert_same(_state(x), _state(y), "continued")


def test_batch_tma_timeout_word_clear(sc):
    """After TMA-fed batch steps every lattice's error word is clear (diagnostics
    report no expired wait)."""
    lats = _make(sc, 1, MIX3_TMA, "f32")
    sc.Batch(lats, tile=4, zchunk=8).step(6)
    for lat in lats:
        assert lat.diagnostics()["status"] == sc.LBM_OK


def test_batch_rejects_outside_step(sc):
    lats = _make(sc, 1, MIX3[:2], "f32")
    b = sc.Batch(lats)
    b.step(2)
    lats[1].step(1)
    with pytest.raises(sc.LbmError) as e:
        b.step(1)
    assert e.value.status == sc.LBM_ERR_INVALID_ARG


def test_batch_one_lattice_vs_oracle(sc, oracle_mod):
    """A batch of one ragged D3Q19 lattice against the FP64 oracle directly (FP32: 1e-5)."""
    shape, tA, tB, G = MIX3[1]
    rA, rB = _fields(shape, 1)
    lat = sc.Lattice(1, shape, tA, tB, G, "f32").init(rA, rB)
    sc.Batch([lat], tile=1, zchunk=4).step(40)
    g = _state(lat)
    o = oracle_mod.OracleSC(1, shape, tA, tB, G).init(rA, rB).step(40)
    a, bb, _, _ = o.moments()
    for x, y in ((g[0], a), (g[1], bb)):
        assert np.abs(x - y).max() / np.abs(y).max() < 1e-5


def test_batch_autotuner_restores_state(sc):
    """tune_batch times every candidate on the caller's lattices and puts their
    states back: afterwards they continue exactly as if never tuned."""
    import torch
    from paper_1112_5547_gb300 import autotune
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = _make(sc, 1, MIX3_TALL, "f32")
        b = _make(sc, 1, MIX3_TALL, "f32")
        for lat in a + b:
            lat.step(3)
        best, table = autotune.tune_batch(a, trial_steps=2, warmup_steps=2, stream=stream,
                                          cands=autotune.batch_candidates(a, zchunks=(0, 16), graph_steps=(0, 2)))
        assert len(table) >= 8 and best in [c for c, _ in table]
        for lat in a + b:
            lat.step(5)
        for x, y in zip(a, b):
            _assert_same(_state(x), _state(y), "restored")
