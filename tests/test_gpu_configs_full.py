"""The two long workloads at their full step counts against stored oracle results.

The FP64 oracle needs tens of minutes for them, so ``tests/golden/make_config_goldens.py``
(which calls only ``oracle/`` and the seeded input recipes) ran them once and
stored the observables and sampled fields; here the CUDA path runs the same
seeded inputs through the C ABI and is compared with those values.

* D2Q9 Laplace batch (Sec. 4.1): drops of R = 8 .. 40 on 256^2 and a flat
  interface on 256 x 64, FP32, 20000 steps, advanced as one ragged batch.
  Per drop: mass-equivalent radius, pressure jump and peak speed within 1e-3
  of the oracle's, the fitted sigma (dP = sigma / R) within 1e-3; the flat
  interface has no jump.  Each species' mass stays within 1e-6 over the
  20000 steps (FP32 at tau = 1; measured on GB300: at most 3.2e-8).  The
  densities on the rows and columns through the centres are held to 1.5e-4
  of the largest density, not the 1e-5 of 1000 steps (the 64^2 drop of
  test_gpu_parity.py): over 20000 steps of a dynamic interface FP32 rounding
  moves them by up to 6.3e-5 (measured).
* The ragged batch of 64 D3Q19 lattices (L from {32, 48, 64, 96, 128}),
  FP32, 2000 steps in the bench's launch shape: bitwise the same as the
  lattices stepped one at a time, each species' mass within 1e-6.
* D3Q19 drop R = 32 on 128^3, 5000 steps (the static drop in three
  dimensions): FP32 as above (observables 1e-3, the sampled rho_A 1e-5, mass
  drift 1e-6); the rest-offset 16-bit storages within 1 % on radius, pressure
  jump and peak speed; the reference-offset 16-bit storages are reported only
  (their offsets from one reference density per species are O(rho) in one of
  the two phases, so they miss the 1 % bar).
"""
import json
import os
import sys

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
if GOLDEN not in sys.path:
    sys.path.insert(0, GOLDEN)
import make_config_goldens as cfg  # noqa: E402  (recipes and observables; no oracle call)


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


def _rel(a, b):
    return abs(a / b - 1.0)


# FP32 bounds over the 20000 steps of the Laplace batch: the mass bar of the
# FP32 parity, and about twice the measured 6.3e-5 on the densities
DRIFT_20000 = 1e-6
ROWS_20000 = 1.5e-4


def test_laplace_batch_20000_steps_vs_oracle(sc):
    import torch
    gold = json.load(open(os.path.join(GOLDEN, "laplace_batch_256.json")))
    assert gold["steps"] == cfg.LAPLACE_STEPS
    stream = torch.cuda.Stream()
    cases = cfg.laplace_cases()
    with torch.cuda.stream(stream):
        lats = [sc.Lattice(0, shape, 1.0, 1.0, cfg.G0, "f32", stream=stream).init(
            *(x.astype(np.float32) for x in f)) for _, shape, f, _ in cases]
        m0 = [(d["mass_A"], d["mass_B"]) for d in (lat.diagnostics() for lat in lats)]
        b = sc.Batch(lats, tile=7, graph_steps=100, stream=stream)
        b.step(cfg.LAPLACE_STEPS)
        stream.synchronize()
        b.close()
        m1 = [(d["mass_A"], d["mass_B"]) for d in (lat.diagnostics() for lat in lats)]
        fields = [[t.double().cpu().numpy() for t in lat.moments()] for lat in lats]
    R, dP, report = [], [], {}
    for (name, shape, _, R0), (rA, rB, u, p), a0, a1 in zip(cases, fields, m0, m1):
        g = gold["cases"][name]
        ny, nx = shape
        scale = max(np.abs(np.array(g["row_rho_A"])).max(), 1e-3)
        r = {"drift": max(abs(a1[0] / a0[0] - 1), abs(a1[1] / a0[1] - 1)),
             "row": np.abs(rA[ny // 2] - np.array(g["row_rho_A"])).max() / scale}
        if R0 is None:
            r["flat_dP"] = cfg.slab_jump(p)
        else:
            r["col"] = np.abs(rA[:, nx // 2] - np.array(g["col_rho_A"])).max() / scale
            obs = cfg.observables(rA, p, u, R0)
            r["obs"] = [_rel(x, y) for x, y in zip(obs, (g["R"], g["dP"], g["umax"]))]
            R.append(obs[0])
            dP.append(obs[1])
        report[name] = r
    sigma, c0, r2 = cfg.laplace_fit(R, dP)
    print("laplace batch: sigma %.6f (oracle %.6f), r2 %.5f" % (sigma, gold["fit"]["sigma"], r2))
    for name, r in report.items():
        print("  %-9s %s" % (name, {k: (np.round(v, 9).tolist() if isinstance(v, list) else float("%.3e" % v))
                                     for k, v in r.items()}))
    for name, r in report.items():
        assert r["drift"] < DRIFT_20000, (name, r)
        assert r["row"] < ROWS_20000 and r.get("col", 0.0) < ROWS_20000, (name, r)
        if "obs" in r:
            assert max(r["obs"]) < 1e-3, (name, r)
    assert _rel(sigma, gold["fit"]["sigma"]) < 1e-3
    assert r2 > 0.99 and abs(c0) < 0.05 * max(dP)
    assert abs(report["slab"]["flat_dP"]) < 0.02 * max(dP)  # the flat interface carries no jump


@pytest.fixture(scope="module")
def drop3d_gold():
    return json.load(open(os.path.join(GOLDEN, "drop3d_128_5000.json")))


@pytest.mark.parametrize("precision,bar", [("f32", 1e-3), ("bf16_rest", 1e-2), ("f16_rest", 1e-2),
                                           ("bf16", None), ("f16", None)])
def test_drop3d_128_5000_steps_vs_oracle(sc, drop3d_gold, precision, bar):
    import torch
    g = drop3d_gold
    L, R0 = cfg.DROP3D_L, g["R0"]
    assert g["steps"] == cfg.DROP3D_STEPS
    f = cfg.drop3d_fields()
    ref = (1.0, 0.04) if precision in ("bf16", "f16") else (0.0, 0.0)
    lat = sc.Lattice(1, (L, L, L), 1.0, 1.0, cfg.G0, precision, *ref).init(*(x.astype(np.float32) for x in f))
    d0 = lat.diagnostics()
    lat.step(cfg.DROP3D_STEPS)
    d1 = lat.diagnostics()
    rA, rB, u, p = (t.double().cpu().numpy() for t in lat.moments())
    obs = cfg.observables(rA, p, u, R0)
    err = [_rel(x, y) for x, y in zip(obs, (g["R"], g["dP"], g["umax"]))]
    drift = max(abs(d1["mass_A"] / d0["mass_A"] - 1), abs(d1["mass_B"] / d0["mass_B"] - 1))
    print("drop3d %s: R %.3e dP %.3e umax %.3e, mass drift %.2e" % ((precision,) + tuple(err) + (drift,)))
    del lat
    torch.cuda.empty_cache()
    if bar is None:
        return  # reported only
    assert max(err) < bar, (precision, err)
    if precision == "f32":
        assert drift < 1e-6
        c = L // 2
        scale = max(abs(v) for v in g["line_x_rho_A"])
        for got, key in ((rA[c, c, :], "line_x_rho_A"), (rA[c, :, c], "line_y_rho_A"), (rA[:, c, c], "line_z_rho_A"),
                         (rB[c, c, :], "line_x_rho_B")):
            assert np.abs(got - np.array(g[key])).max() < 1e-5 * scale, key
        o = g["sub8_offset"]
        sub = rA[o::8, o::8, o::8].ravel()
        assert np.abs(sub - np.array(g["sub8_rho_A"])).max() < 1e-5 * scale


def test_drop3d_256_5000_steps_laplace_and_storage(sc, drop3d_gold):
    """The static drop at L = 256 (R0 = 64), 5000 steps, where the FP64 oracle
    would need hours: properties that hold at any size.  FP32 conserves each
    species' mass to 1e-6 and keeps the drop at its mass-equivalent radius
    (within 1 % of the oracle's R / R0 at L = 128); Laplace's law (Sec. 4.1,
    dP = 2 sigma / R in 3D) gives the same dP R as the oracle's 128^3 drop
    within 5 % (the law's curvature corrections differ between R = 32 and 64);
    the rest-offset 16-bit storages stay within 1 % of the FP32 run on R, dP
    and max|u|, the bar the 128^3 drop meets against the oracle.  Measured on
    GB300: R 63.95 (R / R0 0.6 % from the oracle's at 128^3), dP R 2.0 % below
    the 128^3 value, mass drift 2.7e-9; bf16 / f16 rest-offset within 0.42 % /
    0.095 % of FP32."""
    import torch
    g = drop3d_gold
    L, R0, steps = 256, 64.0, cfg.DROP3D_STEPS
    f = [x.astype(np.float32) for x in inputs_drop((L, L, L), R0)]
    obs, drift = {}, {}
    for precision in ("f32", "bf16_rest", "f16_rest"):
        lat = sc.Lattice(1, (L, L, L), 1.0, 1.0, cfg.G0, precision).init(*f)
        d0 = lat.diagnostics()
        lat.step(steps)
        d1 = lat.diagnostics()
        rA, rB, u, p = (t.double().cpu().numpy() for t in lat.moments())
        obs[precision] = cfg.observables(rA, p, u, R0)
        drift[precision] = max(abs(d1["mass_A"] / d0["mass_A"] - 1), abs(d1["mass_B"] / d0["mass_B"] - 1))
        del lat, rA, rB, u, p
        torch.cuda.empty_cache()
    R, dP, umax = obs["f32"]
    laplace = dP * R / (g["dP"] * g["R"])
    print("drop3d 256: R %.4f dP %.6e umax %.4e, dP R / (dP R at 128) %.5f, drift %s" % (R, dP, umax, laplace, drift))
    for precision in ("bf16_rest", "f16_rest"):
        print("  %s: %s" % (precision, [_rel(x, y) for x, y in zip(obs[precision], obs["f32"])]))
    assert drift["f32"] < 1e-6
    assert _rel(R / R0, g["R"] / g["R0"]) < 1e-2
    assert abs(laplace - 1.0) < 0.05
    for precision in ("bf16_rest", "f16_rest"):
        assert max(_rel(x, y) for x, y in zip(obs[precision], obs["f32"])) < 1e-2, precision


def inputs_drop(shape, R):
    from paper_1112_5547_gb300 import inputs
    return inputs.drop(shape, R, seed=2)


def test_ragged_batch_2000_steps_equals_solo(sc):
    """The 64 ragged lattices over 2000 steps, batched in the bench's launch
    shape (batch tile 12: 64x6 / 48x8 / 32x12 per lattice, one CTA per work
    item, 16-plane chunks, graph chunks of 8 steps) and stepped one at a time
    (each lattice in its default launch shape): the fields are bitwise equal,
    and every lattice keeps each species' mass within 1e-6.  About half of the
    recipe's draws (low tau with strong coupling) drive a density below zero
    within a few hundred steps, in the FP64 oracle as well; conservation and
    the batch-equals-solo identity hold for them too, so every lattice is
    checked and the unstable ones are counted."""
    import torch
    from paper_1112_5547_gb300 import inputs
    specs = inputs.ragged_drop_specs()
    steps = 2000
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        mk = lambda sp: sc.Lattice(1, sp["shape"], sp["tau_A"], sp["tau_B"], sp["G"], "f32", stream=stream).init(
            *inputs.spec_fields(sp, dtype=np.float32))
        ref, m0 = [], []
        for sp in specs:
            lat = mk(sp)
            d = lat.diagnostics(check=False)
            m0.append((d["mass_A"], d["mass_B"]))
            lat.step(steps)
            ref.append([t.cpu().numpy() for t in lat.moments()])
            lat.close()
        lats = [mk(sp) for sp in specs]
        b = sc.Batch(lats, tile=12, zchunk=16, graph_steps=8, stream=stream)
        b.step(steps)
        stream.synchronize()
        b.close()
        worst, unstable, diverged = 0.0, 0, 0
        for k, lat in enumerate(lats):
            for x, y in zip((t.cpu().numpy() for t in lat.moments()), ref[k]):
                assert np.array_equal(x, y, equal_nan=True), k
            d = lat.diagnostics(check=False)
            if d["nonfinite"] > 0:  # diverged: the identity above still holds, mass is not defined
                diverged += 1
                continue
            unstable += not (d["min_rho_A"] > 0 and d["min_rho_B"] > 0)
            worst = max(worst, abs(d["mass_A"] / m0[k][0] - 1), abs(d["mass_B"] / m0[k][1] - 1))
        print("ragged batch 2000 steps: bitwise equal to solo; worst mass drift %.2e over the %d finite lattices, "
              "%d of them with a non-positive density; %d diverged" % (worst, len(lats) - diverged, unstable,
                                                                       diverged))
        assert worst < 1e-6 and diverged < len(lats) // 2
    torch.cuda.empty_cache()
