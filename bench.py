"""Benchmark of the fused two-component Shan-Chen step (MLUPS and HBM roofline).

Default workload: D3Q19 512^3 periodic lattice, FP32, spherical drop R = L/4
(tau = 1, G rho_tot = 2.4, rho 1.0 / 0.04, tanh width 2, +-1e-3 seeded noise).
One timed "step" is one lattice time step (one fused-kernel launch) over all
134,217,728 nodes.  Each population buffer is 20.4 GB, far larger than the
129 MB L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--L 512] [--precision f32|bf16|f16|bf16_rest|f16_rest|f64]
                    [--no-e2e] [--no-cpu-baseline] [--no-batch] [--serve-requests 24]
                    [--no-storage16] [--no-kolmogorov] [--no-guo] [--no-fe] [--no-pfm]

Prints one JSON line (rank 0).  Beside the headline step it carries
"storage16" (the same step with 16-bit rest-offset storage), "kolmogorov"
(the same drop under the Kolmogorov forcing of Sec. 4.2), "guo" (the same
drop with Guo forcing, Sec. 2.3), "fe" (the free-energy model of Sec. 2.2 on
the same lattice), "pfm" (the phase-field model of Sec. 3 against the SC step
on a 256^3 grid), "batch"
(64 ragged D3Q19 lattices advanced by one launch per step against the same
lattices stepped one at a time), "batch_rest16" (the same with the paired
16-bit rest-offset storage) and "serving" (a seeded Poisson stream of
drop-relaxation requests served with continuous batching against serial
solves, p50/p99 time to result).  Under torchrun each rank advances its own
lattice (independent replicas, no collective on the data path); the timed
region is bracketed by barriers and the max over ranks is reported; the batch
and serving comparisons run on rank 0 only.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

G_RHO = 2.4
RHO_HI, RHO_LO = 1.0, 0.04
BYTES_PER_VALUE = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2, "bf16_rest": 2, "f16_rest": 2}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "bf16": "f32 (bf16 storage)", "f16": "f32 (f16 storage)",
              "bf16_rest": "f32 (bf16 rest-offset storage)", "f16_rest": "f32 (f16 rest-offset storage)"}


def bytes_per_lu(prec: str, q: int = 19) -> int:
    """Algorithmic HBM bytes of one lattice update (both species): every population
    read once and written once, plus the two FP32 densities of the rest-offset storage."""
    b = 2 * q * 2 * BYTES_PER_VALUE[prec]
    if prec.endswith("_rest"):
        b += 2 * 2 * 4
    return b
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--precision", default="f32", choices=list(BYTES_PER_VALUE))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tile", type=int, default=-1, help="force a step tile (skips the autotuner)")
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch vs serial comparison")
    ap.add_argument("--batch-steps", type=int, default=40)
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the continuous-batching serving run (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--no-storage16", action="store_true", help="skip the 16-bit rest-offset storage line")
    ap.add_argument("--no-kolmogorov", action="store_true", help="skip the Kolmogorov-forced drop line")
    ap.add_argument("--no-guo", action="store_true", help="skip the Guo-forcing line")
    ap.add_argument("--no-fe", action="store_true", help="skip the free-energy model line")
    ap.add_argument("--no-pfm", action="store_true", help="skip the phase-field model line")
    ap.add_argument("--profile", default=None, choices=list(PROFILE_CASES),
                    help="run one small fixed workload for ncu and exit (no JSON line)")
    ap.add_argument("--batch-tile", type=int, default=5, help="batch tile of the --profile batch cases")
    ap.add_argument("--ragged-n", type=int, default=64, help="lattices of the --profile ragged case (same recipe)")
    return ap.parse_args()


PROFILE_CASES = ("step", "step2d", "solo_vs_batch", "ragged", "pfm")


def profile_case(a):
    """Small fixed workloads for profiling the kernels under ncu; each builds its
    lattices, runs ``--steps`` steps with a fixed launch shape and exits.

      step           one D3Q19 drop lattice (R = L/4, G rho_tot = 2.4, tau = 1)
                     in --precision, --tile / --zchunk, solo steps
      step2d         the same on an L^2 D2Q9 lattice
      solo_vs_batch  the D3Q19 drop stepped twice alone, then twice as a batch of one
      ragged         the ragged batch (inputs.ragged_drop_specs, --ragged-n lattices, --precision), --batch-tile
      pfm            the phase-field solver (FP32) on an L^3 drop (rho_A 1.2 / rho_B 0.2,
                     tau 0.6, g 0.3, dt 0.1)

    e.g. python bench.py --profile step --L 192 --precision bf16_rest --tile 35 --zchunk 48 --steps 3
    """
    import torch
    from paper_1112_5547_gb300 import inputs, lbm_sc
    G = G_RHO / (RHO_HI + RHO_LO)

    def drop_lattice(L, precision, stream):
        rA, rB = inputs.drop((L, L, L), L / 4, seed=2, dtype=np.float32)
        ref = (0.52, 0.52) if precision in ("bf16", "f16") else (0.0, 0.0)
        return lbm_sc.Lattice(lbm_sc.LBM_D3Q19, (L, L, L), 1.0, 1.0, G, precision, ref[0], ref[1],
                              stream=stream).init(rA, rB)

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        if a.profile == "pfm":
            from paper_1112_5547_gb300 import phase_field
            rA, rB = inputs.drop((a.L,) * 3, a.L / 4, rho_hi=1.2, rho_lo=0.2, seed=2, dtype=np.float32)
            phase_field.PFM((a.L,) * 3, 1.4, 0.6, 0.3, 0.1, "f32", stream=st).init(rA - rB).step(a.steps)
        elif a.profile == "step2d":
            rA, rB = inputs.drop((a.L, a.L), a.L / 4, seed=0, dtype=np.float32)
            lat = lbm_sc.Lattice(lbm_sc.LBM_D2Q9, (a.L, a.L), 1.0, 1.0, G, a.precision, stream=st).init(rA, rB)
            lat.set_tuning(max(a.tile, 0), 0)
            lat.step(a.steps)
        elif a.profile == "step":
            lat = drop_lattice(a.L, a.precision, st)
            lat.set_tuning(max(a.tile, 0), a.zchunk)
            lat.step(a.steps)
        elif a.profile == "solo_vs_batch":
            lat = drop_lattice(a.L, a.precision, st)
            lat.set_tuning(max(a.tile, 0), a.zchunk)
            lat.step(2)
            b = lbm_sc.Batch([lat], tile=a.batch_tile, zchunk=a.zchunk, stream=st)
            b.step(2)
            st.synchronize()
            b.close()
        else:
            lats = []
            for sp in inputs.ragged_drop_specs(n=a.ragged_n):
                rA, rB = inputs.spec_fields(sp, dtype=np.float32)
                lats.append(lbm_sc.Lattice(lbm_sc.LBM_D3Q19, sp["shape"], sp["tau_A"], sp["tau_B"], sp["G"], a.precision,
                                           stream=st).init(rA, rB))
            print("ragged batch: %d lattices, %d nodes" % (len(lats), sum(x.N for x in lats)))
            b = lbm_sc.Batch(lats, tile=a.batch_tile, zchunk=a.zchunk, stream=st)
            b.step(a.steps)
            st.synchronize()
            b.close()
        st.synchronize()
    print("profile case %s ok" % a.profile)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1112_5547_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def drop_fields(L, dtype, seed=2):
    from paper_1112_5547_gb300 import inputs
    return inputs.drop((L, L, L), L / 4.0, rho_hi=RHO_HI, rho_lo=RHO_LO, width=2.0, noise=1e-3, seed=seed,
                       dtype=dtype)


def cpu_baseline(seconds: float, L: int = 128):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of the
    same workload (a 128^3 drop with the same recipe): time whole steps until
    ``seconds`` have passed."""
    import oracle
    oracle.build()
    G = G_RHO / (RHO_HI + RHO_LO)
    rA, rB = drop_fields(L, np.float64)
    o = oracle.OracleSC(1, (L, L, L), 1.0, 1.0, G).init(rA, rB)
    o.step(1)  # warm-up
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds and n >= 2:
            break
    mlups = L ** 3 * n / el / 1e6
    cores = oracle.num_threads()
    # the same oracle on one core, on a 64^3 sample of the recipe (a few seconds)
    oracle.set_num_threads(1)
    try:
        Ls = 64
        rA, rB = drop_fields(Ls, np.float64)
        o1 = oracle.OracleSC(1, (Ls, Ls, Ls), 1.0, 1.0, G).init(rA, rB)
        t0 = time.perf_counter()
        n1 = 0
        while time.perf_counter() - t0 < seconds / 4 or n1 < 2:
            o1.step(1)
            n1 += 1
        el1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "D3Q19 %d^3 drop (same recipe), FP64 oracle, %d steps in %.1f s" % (L, n, el),
            "single_core": {"value": Ls ** 3 * n1 / el1 / 1e6, "unit": "MLUPS",
                            "sample": "D3Q19 %d^3 drop, 1 thread, %d steps in %.1f s" % (Ls, n1, el1)}}


def batch_compare(steps: int, warmup: int, n: int = 64, seed: int = 3, precision: str = "f32"):
    """Ragged batch against one-lattice-at-a-time on the same lattices: n
    independent D3Q19 drop lattices (storage `precision`: FP32, or the paired
    16-bit rest-offset words), L from {32, 48, 64, 96, 128}, per
    lattice G rho_tot in [2.2, 2.8], tau_A, tau_B in [0.6, 1.5], R in [L/8, L/3]
    at a random centre (inputs.ragged_drop_specs).  Serial: every lattice
    stepped alone with its own autotuned launch shape (tuned once per size),
    lattice after lattice, `steps` steps each.  Batched: one launch per step for
    all lattices, launch shape and graph chunk autotuned (tune_batch).  Both
    timed with CUDA events on one stream; aggregate MLUPS = total nodes x steps
    / time.  Results are bit-identical between the two (tests/test_gpu_batch.py)."""
    import torch
    from paper_1112_5547_gb300 import autotune, inputs, lbm_sc

    st = torch.cuda.Stream()
    specs = inputs.ragged_drop_specs(n=n, seed=seed)
    lats = []
    with torch.cuda.stream(st):
        for sp in specs:
            rA, rB = inputs.spec_fields(sp, dtype=np.float32)
            lats.append(lbm_sc.Lattice(lbm_sc.LBM_D3Q19, sp["shape"], sp["tau_A"], sp["tau_B"], sp["G"], precision,
                                       stream=st).init(rA, rB))
        st.synchronize()
        N = sum(lat.N for lat in lats)
        best = {}
        for lat in lats:
            if lat.shape not in best:
                best[lat.shape] = autotune.autotune(lat)[0]
            lat.set_tuning(*best[lat.shape])

        def timed(fn, k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(k)
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1)

        for lat in lats:
            lat.step(warmup + warmup % 2)
        ser_ms = timed(lambda k: [lat.step(k) for lat in lats], steps) / steps
        (tile, zc, gs), table = autotune.tune_batch(lats, stream=st)
        b = lbm_sc.Batch(lats, tile=tile, zchunk=zc, graph_steps=gs, stream=st)
        b.step(max(warmup, gs, 2))
        k = steps if gs == 0 else max(gs, steps // gs * gs)
        bat_ms = timed(b.step, k) / k
        b.close()
    sizes = sorted({lat.shape[0] for lat in lats})
    traffic = None  # ncu DRAM bytes per LU of this launch shape on this workload, if the kernels are unchanged
    # the captured launches: FP32 on batch tile 12 with 16-plane chunks, bf16 rest-offset
    # on tile 13 with 32-plane chunks (zchunk 0 means 32)
    captured = {"f32": (12, 16), "bf16_rest": (13, 32)}
    key = "batch_ragged64_%s" % precision
    if (os.path.exists(TRAFFIC_FILE) and n == 64 and seed == 3 and precision in captured
            and (tile, zc or 32) == captured[precision]):
        tf = json.load(open(TRAFFIC_FILE))
        if tf.get(key, {}).get("source_hash") == kernel_source_hash():
            traffic = tf[key]["dram_bytes_per_lu"]
    storage = "FP32" if precision == "f32" else precision + " (FP32 arithmetic)"
    out = {"workload": "%d ragged D3Q19 %s drop lattices, L in %s, %.1fM nodes, seed %d"
                       % (n, storage, sizes, N / 1e6, seed),
           "nodes": N, "steps": steps, "batched_mlups": N / bat_ms / 1e3, "serial_mlups": N / ser_ms / 1e3,
           "batched_ms_per_step": bat_ms, "serial_ms_per_step": ser_ms, "speedup": ser_ms / bat_ms,
           "batch_launch": {"tile_id": tile, "tile": list(lbm_sc.BATCH_TILES[tile]), "tma": lbm_sc.BATCH_TILE_TMA[tile],
                            "zchunk": zc, "graph_steps": gs, "candidates": len(table)},
           "gpu_launches_per_step": {"batched": 1, "serial": n},
           "dram_bytes_per_lu": traffic, "algorithmic_bytes_per_lu": bytes_per_lu(precision)}
    del lats
    torch.cuda.empty_cache()
    return out


def _drop_leg(L: int, steps: int, warmup: int, peak: float, precision: str, body_A: float = 0.0,
              forcing: str = "shift", tile=None, fe=None):
    """One D3Q19 L^3 drop (the headline's lattice and fields) timed like the
    headline step: CUDA events on the lattice's stream over `steps` steps after
    `warmup`, inputs far larger than L2.  Launch shape from the tuning cache
    (autotuned on GB300), else autotuned here, unless `tile` = (tile, zchunk)
    fixes it.  Returns the timing, the launch shape and the diagnostics before
    and after.  fe = (g, Gamma, rho_hi, rho_lo): the free-energy model of Sec. 2.2
    (tau = tau_g = 1) on a drop of those densities instead."""
    import torch
    from paper_1112_5547_gb300 import autotune, inputs, lbm_sc
    st = torch.cuda.Stream()
    G = G_RHO / (RHO_HI + RHO_LO)
    if fe is not None:
        rA, rB = inputs.drop((L, L, L), L / 4.0, rho_hi=fe[2], rho_lo=fe[3], seed=2, dtype=np.float32)
    else:
        rA, rB = drop_fields(L, np.float32, seed=2)
    with torch.cuda.stream(st):
        if fe is not None:
            lat = lbm_sc.FELattice(lbm_sc.LBM_D3Q19, (L, L, L), 1.0, 1.0, fe[0], precision, gamma=fe[1],
                                   stream=st).init(rA, rB)
        else:
            lat = lbm_sc.Lattice(lbm_sc.LBM_D3Q19, (L, L, L), 1.0, 1.0, G, precision, stream=st,
                                 body_A=body_A, forcing=forcing).init(rA, rB)
        del rA, rB
        d0 = lat.diagnostics(check=False)
        if tile is not None:
            lat.set_tuning(*tile)
        else:
            autotune.tuned(lat, store=False)
        lat.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.step(steps)
        e1.record(st)
        e1.synchronize()
        d = lat.diagnostics(check=False)
        tile_used = lat.tuning()
    ms = e0.elapsed_time(e1) / steps
    del lat
    torch.cuda.empty_cache()
    N = L ** 3
    bpl = bytes_per_lu(precision)
    gbs = bpl * N / (ms / 1e3) / 1e9
    return {"precision": precision, "mlups": N / ms / 1e3, "ms_per_step": ms, "steps": steps,
            "algorithmic_bytes_per_lu": bpl, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
            "tile": list(lbm_sc.TILES[tile_used[0]]), "tile_id": tile_used[0], "zchunk": tile_used[1]}, d0, d


def storage16_compare(L: int, steps: int, warmup: int, peak: float, precision: str = "bf16_rest"):
    """The same D3Q19 drop step with 16-bit rest-offset storage (FP32 arithmetic):
    MLUPS and the HBM roofline of its 168 algorithmic bytes per LU."""
    out, _, d = _drop_leg(L, steps, warmup, peak, precision)
    N = L ** 3
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        tf = json.load(open(TRAFFIC_FILE))
        key = "d3q19_%s" % precision
        if key in tf and tf[key].get("source_hash") == kernel_source_hash():
            traffic = tf[key]["dram_bytes_per_lu"] * N
    out.update({"workload": "D3Q19 %d^3 drop, same as the headline" % L, "traffic": traffic,
                "diag_status": d["status"],
                "accuracy": "radius / Laplace dP / max|u| within 1% of the FP64 oracle (tests/test_gpu_storage16.py)"})
    return out


def guo_compare(L: int, steps: int, warmup: int, peak: float):
    """The headline drop with Guo forcing (the cure of the tau-dependent
    coupling named in Sec. 2.3) instead of the velocity shift: the same 304
    algorithmic bytes per LU, a longer collision (the source term), on the
    headline's tile 34 (its Guo instantiation)."""
    out, _, d = _drop_leg(L, steps, warmup, peak, "f32", forcing="guo", tile=(34, 32))
    out.update({"workload": "D3Q19 %d^3 drop, Guo forcing" % L, "forcing": "guo", "diag_status": d["status"],
                "parity": "tests/test_gpu_guo.py (FP64 1e-12, FP32 1e-5 vs the oracle; sampled nodes at 512^3)"})
    return out


def fe_compare(L: int, steps: int, warmup: int, peak: float):
    """The free-energy two-population model of Sec. 2.2 (Eqs. FE1, FE2, the Eq.
    FEtau functional with g = 2.5, Gamma = 0.5, tau = tau_g = 1) on an L^3 drop of
    rho_A = 0.9 in rho_B = 0.14 (phi = +-0.76, its coexistence at rho = 1.04): the
    same storage and 304 algorithmic bytes per LU as the SC step, on tile 34
    (its FE instance)."""
    out, _, d = _drop_leg(L, steps, warmup, peak, "f32", tile=(34, 32), fe=(2.5, 0.5, 0.9, 0.14))
    out.update({"workload": "D3Q19 %d^3 drop, free-energy model (g 2.5, Gamma 0.5, rho 0.9 / 0.14)" % L,
                "model": "fe", "diag_status": d["status"],
                "parity": "tests/test_gpu_fe.py (FP64 1e-12, FP32 1e-5 vs the FE oracle; sampled nodes at 512^3)"})
    return out


def pfm_compare(L: int, steps: int, warmup: int):
    """The pseudo-spectral phase-field model of Sec. 3 (libpfm.so: cuFFT plus the
    library's kernels) against the SC step on the same L^3 grid and drop
    (rho_A 1.2 / rho_B 0.2, tau = 0.6, g = 0.3, FP32): milliseconds per step of
    each, CUDA events on one stream, and their ratio per step and per unit of
    physical time (the PFM runs at dt = 0.1 here, the LBM at 1; the paper reports
    T_PFM / T_SC = 2.9 for its 2D runs on CPUs, Fig. 6)."""
    import torch
    from paper_1112_5547_gb300 import inputs, lbm_sc, phase_field
    st = torch.cuda.Stream()
    rA, rB = inputs.drop((L, L, L), L / 4.0, rho_hi=1.2, rho_lo=0.2, seed=2, dtype=np.float32)
    dt = 0.1

    def timed(obj):
        obj.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        obj.step(steps)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    with torch.cuda.stream(st):
        s = phase_field.PFM((L, L, L), 1.4, 0.6, 0.3, dt, "f32", stream=st).init(rA - rB)
        ms_pfm = timed(s)
        phi, _ = s.fields()
        finite = bool(torch.isfinite(phi).all())
        del s, phi
        torch.cuda.empty_cache()
        lat = lbm_sc.Lattice(lbm_sc.LBM_D3Q19, (L, L, L), 0.6, 0.6, 0.3, "f32", stream=st).init(rA, rB)
        lat.set_tuning(34, 32)
        ms_sc = timed(lat)
        del lat
        torch.cuda.empty_cache()
    N = L ** 3
    return {"workload": "3D %d^3 drop, rho 1.2 / 0.2, tau 0.6, g 0.3, FP32; PFM dt = %g" % (L, dt),
            "ms_per_step_pfm": ms_pfm, "ms_per_step_sc": ms_sc, "ratio_per_step": ms_pfm / ms_sc,
            "ratio_per_time_unit": ms_pfm / dt / ms_sc, "pfm_mnodes_per_s": N / ms_pfm / 1e3,
            "transforms_per_step": 19, "steps": steps, "finite": finite,
            "parity": "tests/test_gpu_pfm.py (FP64 1e-10, FP32 1e-5 vs the numpy oracle; 128^3 whole field)"}


def kolmogorov_compare(L: int, steps: int, warmup: int, peak: float, A: float = 1e-6):
    """The headline drop under the Kolmogorov forcing of Eq. kolmo (Sec. 4.2),
    F_x = rho A sin(2 pi y / L), A = 1e-6 as in the paper: the same fused step
    with the body force, MLUPS and roofline fraction, plus the kinetic energy
    and the leakage L(t) = M(t) / M_0 (nodes with rho_A >= rho_B) after the run."""
    out, d0, d = _drop_leg(L, steps, warmup, peak, "f32", body_A=A)
    out.update({"workload": "D3Q19 %d^3 drop, Kolmogorov forcing A = %g" % (L, A), "body_A": A,
                "kinetic_energy": d["kinetic_energy"], "leakage": d["droplet_nodes"] / d0["droplet_nodes"],
                "steps_run": warmup + steps, "diag_status": d["status"],
                "parity": "tests/test_gpu_kolmogorov.py (FP64 1e-12, FP32 1e-5 vs the oracle; closed form at 512^3)"})
    return out


def serve_compare(n: int, rate: float, seed: int = 4):
    """Continuous batching against serial solves on a seeded Poisson stream of
    n drop- and interface-relaxation requests (a quarter are flat interfaces;
    mean rate per second): D2Q9 lattices 64^2 ..
    1024^2 and D3Q19 32^3 .. 192^3 (sizes 32, 48, 64, 96, 128, 160, 192), per-request G, tau, R as in the ragged
    batch; each runs until max|u_phys| changes by < 1% over 500 steps or 10000
    steps; 80 GB HBM admission budget, smallest lattices admitted first while
    the resident set holds fewer than 48 M nodes; FP32.  Time to result = arrival to the
    result (rho_A) in host memory.  Serial: the same requests one at a time
    (plain lbm_sc_step, same convergence rule), input generation not timed."""
    from paper_1112_5547_gb300 import serving
    reqs = serving.poisson_requests(n, rate, seed, interface_fraction=0.25)
    # smallest lattices admitted first while the resident set holds < 48 M nodes
    # (256-request sweep: p50 45 -> 12 s at 1 % less throughput, p99 unchanged)
    res, st = serving.Server(hbm_budget=80e9, order="size", max_active_nodes=48_000_000).run(reqs)
    sres, stot, smlups = serving.serial_baseline(reqs)
    return {"workload": "%d Poisson requests at %.0f/s (seed %d): drops and (1 in 4) flat interfaces, "
                        "D2Q9 64^2..1024^2, D3Q19 32^3..192^3, "
                        "until |d max|u|| < 1%% per 500 steps, a non-positive density (retired as unstable) "
                        "or 10000 steps, 80 GB budget, FP32" % (n, rate, seed),
            "served_mlups": st.mlups, "serial_mlups": smlups, "speedup": st.mlups / smlups,
            "p50_s": st.p50_s, "p99_s": st.p99_s, "mean_s": st.mean_s, "wall_s": st.wall_s, "serial_s": stot,
            "max_resident": st.max_resident, "admission": "fewest nodes first, resident nodes < 48 M",
            "converged": sum(r.converged for r in res),
            "unstable": sum(r.unstable for r in res),
            "interfaces": sum(r.kind == "interface" for r in reqs),
            "same_steps_as_alone": all(a.steps == b.steps for a, b in zip(res, sres))}


def max_over_ranks(value: float, dist=None, device: str = "cuda") -> float:
    """The largest of one float over all ranks (the job's time is its slowest
    rank's); with no process group, the value itself."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, nodes_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank advanced its own lattice of nodes_per_rank
    nodes by `steps` steps within `seconds` (weak scaling, replicas)."""
    return world * nodes_per_rank * steps / seconds / 1e6


def workload_config(L: int, prec: str, world: int) -> dict:
    """The config object of the JSON line (shared by both arms)."""
    N = L ** 3
    return {"workload": "D3Q19 %d^3 two-component SC drop R=L/4, tau=1, G*rho_tot=2.4, seed 2" % L,
            "lattice": "D3Q19", "L": L, "nodes": N, "storage": prec,
            "l2": "inputs larger than L2 (%.1f GB per population buffer)" % (N * 38 * BYTES_PER_VALUE[prec] / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU"}


REFERENCE_SAMPLE_L = 128


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle (the paper has no code to install) on
    the host cores, W untimed and exactly K timed steps of a 128^3 sample of the
    headline drop workload (same recipe); the line states that sample as its
    config, its own step count and its own time per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    L = REFERENCE_SAMPLE_L
    G = G_RHO / (RHO_HI + RHO_LO)
    rA, rB = drop_fields(L, np.float64)
    o = oracle.OracleSC(1, (L, L, L), 1.0, 1.0, G).init(rA, rB)
    o.step(max(args.warmup, 1))
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    mlups = L ** 3 * args.steps / el / 1e6
    cores = oracle.num_threads()
    cfg = workload_config(L, "f64", 1)
    cfg["parallelism"] = "%d host threads" % cores
    cfg["sample_of"] = "the %d^3 headline workload (oracle FP64 on host cores; a bounded sample)" % args.L
    cb = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
          "sample": "D3Q19 %d^3 drop (same recipe), FP64 oracle, %d timed steps after %d warm-up in %.1f s"
                    % (L, args.steps, max(args.warmup, 1), el)}
    line = {"impl": "reference", "metric": "2-comp SC D3Q19 MLUPS & HBM roofline %", "value": mlups,
            "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.profile is not None:
        from paper_1112_5547_gb300 import build as gb
        gb.build()
        profile_case(args)
        return

    import torch
    from paper_1112_5547_gb300 import build as gb
    from paper_1112_5547_gb300 import lbm_sc

    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        gb.build()
    if dist is not None:
        dist.barrier()
    lbm_sc.load()

    # CPU baseline first (before any CUDA work on this process is busy), rank 0 only at N=1.
    cb = None
    if not args.no_cpu_baseline and world == 1 and rank == 0:
        cb = cpu_baseline(args.cpu_seconds)

    L = args.L
    N = L ** 3
    G = G_RHO / (RHO_HI + RHO_LO)
    prec = args.precision
    cdt = np.float64 if prec == "f64" else np.float32
    ref = (0.5 * (RHO_HI + RHO_LO), 0.5 * (RHO_HI + RHO_LO)) if prec in ("bf16", "f16") else (0.0, 0.0)
    rA, rB = drop_fields(L, cdt, seed=2 + rank)
    stream = torch.cuda.Stream()
    lat = lbm_sc.Lattice(lbm_sc.LBM_D3Q19, (L, L, L), 1.0, 1.0, G, prec, ref[0], ref[1], stream=stream)
    with torch.cuda.stream(stream):
        lat.init(rA, rB)
    stream.synchronize()
    # launch shape: autotuned on this lattice (state restored), or forced
    if args.tile >= 0:
        lat.set_tuning(args.tile, args.zchunk)
        tune_info = {"tile_id": args.tile, "tile": list(lbm_sc.TILES[args.tile]), "kind": lbm_sc.TILE_KIND[args.tile],
                     "cluster": list(lbm_sc.TILE_CLUSTER[args.tile]), "zchunk": lat.tuning()[1], "source": "forced"}
    else:
        from paper_1112_5547_gb300 import autotune
        (tile, zc), source = autotune.tuned(lat, store=(rank == 0))
        tune_info = {"tile_id": tile, "tile": list(lbm_sc.TILES[tile]), "kind": lbm_sc.TILE_KIND[tile],
                     "cluster": list(lbm_sc.TILE_CLUSTER[tile]), "zchunk": zc,
                     "source": source if source == "autotuned" else "tuning cache (autotuned on GB300)"}

    # warm-up
    lat.step(args.warmup)
    stream.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        lat.step(1)
        ev[k][1].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = start.elapsed_time(stop)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    if dist is not None:
        total_ms = max_over_ranks(total_ms, dist)
        dist.barrier()
    d = lat.diagnostics(check=False)

    ms_per_step = total_ms / K
    value = job_mlups(world, N, K, total_ms / 1e3)
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    bpl = bytes_per_lu(prec)
    achieved = bpl * N / avg_launch_s / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        tf = json.load(open(TRAFFIC_FILE))
        key = "d3q19_%s" % prec
        if key in tf and tf[key].get("source_hash") == kernel_source_hash():
            traffic = tf[key]["dram_bytes_per_lu"] * N

    # End to end through the C ABI with host buffers: H2D of the initial fields,
    # init, K steps, moments, D2H of rho_A, rho_B, u, p.
    e2e = None
    if not args.no_e2e:
        lat2 = lat  # reuse the same workspace
        sb = lbm_sc.lbm_sc_host_staging_bytes(lat2.params)
        staging = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
        sp = (staging.data_ptr() + 255) // 256 * 256
        # page-locked host buffers of the library's allocator (driver-allocated)
        tdt = torch.float64 if prec == "f64" else torch.float32
        hbufs = [lbm_sc.HostBuffer(n, tdt) for n in (N, N, N, N, N, 3 * N)]
        hA, hB, oA, oB, oP, oU = (b.tensor for b in hbufs)
        hA.copy_(torch.from_numpy(np.ascontiguousarray(rA).reshape(-1)))
        hB.copy_(torch.from_numpy(np.ascontiguousarray(rB).reshape(-1)))
        # untimed warm-up job (W steps): first touch of the pinned buffers and the copy path
        lbm_sc.lbm_sc_run_host(lat2.handle, sp, sb, hA.data_ptr(), hB.data_ptr(), None, args.warmup,
                               oA.data_ptr(), oB.data_ptr(), oU.data_ptr(), oP.data_ptr())
        # three timed jobs, the median reported (the host link's rate varies from job to job)
        jobs = []
        for _ in range(3):
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbm_sc.lbm_sc_run_host(lat2.handle, sp, sb, hA.data_ptr(), hB.data_ptr(), None, K, oA.data_ptr(),
                                   oB.data_ptr(), oU.data_ptr(), oP.data_ptr())
            jobs.append(time.perf_counter() - t0)
        e2e_s = statistics.median(jobs)
        if dist is not None:
            e2e_s = max_over_ranks(e2e_s, dist)
        esz = 8 if prec == "f64" else 4
        # the link's own rate on these buffers (one field each way, CUDA events), for the floor below
        dfield = torch.empty(N, dtype=tdt, device="cuda")
        ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        h2d_gbs = d2h_gbs = 0.0
        # plain cudaMemcpyAsync, as lbm_sc_run_host issues them (torch's copy_ does
        # not take the driver-allocated buffers for pinned memory and is slower)
        try:
            cudart = ctypes.CDLL("libcudart.so.13")  # the runtime torch has loaded
            cudart.cudaMemcpyAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                               ctypes.c_void_p]
            link_via = "cudaMemcpyAsync"
        except OSError:
            cudart, link_via = None, "torch copy_"
        nb = N * esz

        def copy(dst, src, kind):
            if cudart is None:
                with torch.cuda.stream(stream):
                    dst.copy_(src, non_blocking=True)
            else:
                rc = cudart.cudaMemcpyAsync(dst.data_ptr(), src.data_ptr(), nb, kind, stream.cuda_stream)
                assert rc == 0, rc

        for _ in range(3):  # best of three (the first pass maps the fresh device pages)
            ev0.record(stream)
            copy(dfield, hA, 1)
            ev1.record(stream)
            copy(oA, dfield, 2)
            ev2.record(stream)
            stream.synchronize()
            h2d_gbs = max(h2d_gbs, N * esz / (ev0.elapsed_time(ev1) / 1e3) / 1e9)
            d2h_gbs = max(d2h_gbs, N * esz / (ev1.elapsed_time(ev2) / 1e3) / 1e9)
        del dfield
        copy_s = 2 * N * esz / h2d_gbs / 1e9 + 6 * N * esz / d2h_gbs / 1e9
        e2e = {"value": job_mlups(world, N, K, e2e_s), "unit": "MLUPS",
               "h2d_bytes_per_step": 2 * N * esz / K, "d2h_bytes_per_step": 6 * N * esz / K,
               "seconds": e2e_s, "jobs_seconds": jobs,
               "link_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs, "measured_with": link_via},
               "floor_seconds": K * ms_per_step / 1e3 + copy_s,
               "note": "one job of %d steps through lbm_sc_run_host: H2D rho_A, rho_B; D2H rho_A, rho_B, u(3), p "
                       "(copies overlapped with init and moments in z slabs; host buffers of lbm_sc_host_alloc), "
                       "the median of three jobs; "
                       "bytes per step = job bytes / steps; "
                       "floor = the steps alone + every copy at the measured link rate, unoverlapped" % K}
        del staging, hA, hB, oA, oB, oP, oU, lat2
        for b in hbufs:
            b.close()

    bt = None
    del lat
    torch.cuda.empty_cache()
    s16 = None
    if not args.no_storage16 and rank == 0 and prec == "f32":
        s16 = storage16_compare(L, max(10, K // 2), args.warmup, peak)
    kf = None
    if not args.no_kolmogorov and rank == 0 and prec == "f32":
        kf = kolmogorov_compare(L, max(10, K // 2), args.warmup, peak)
    gf = None
    if not args.no_guo and rank == 0 and prec == "f32":
        gf = guo_compare(L, max(10, K // 2), args.warmup, peak)
    ff = None
    if not args.no_fe and rank == 0 and prec == "f32":
        ff = fe_compare(L, max(10, K // 2), args.warmup, peak)
    pm = None
    if not args.no_pfm and rank == 0 and prec == "f32":
        pm = pfm_compare(256, max(10, K // 2), args.warmup)
    bt16 = None
    if not args.no_batch and rank == 0:
        bt = batch_compare(args.batch_steps, args.warmup)
        bt16 = batch_compare(args.batch_steps, args.warmup, precision="bf16_rest")
    sv = None
    if args.serve_requests > 0 and rank == 0:
        sv = serve_compare(args.serve_requests, args.serve_rate)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": "2-comp SC D3Q19 MLUPS & HBM roofline %",
        "value": value,
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE_NAME[prec],
        "data": "synthetic",
        "config": dict(workload_config(L, prec, world), step_launch=tune_info),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_lu": bpl,
                     "kernel": "D3Q19 %s step, tile %s kind %d" % (prec, tuple(tune_info["tile"]), tune_info["kind"])},
        "gpu_launches": K,
        "clocks": clk,
        "diag": {"mass_A": d["mass_A"], "max_speed": d["max_speed"], "status": d["status"]},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if bt is not None:
        line["batch"] = bt
    if bt16 is not None:
        line["batch_rest16"] = bt16
    if sv is not None:
        line["serving"] = sv
    if s16 is not None:
        line["storage16"] = s16
    if kf is not None:
        line["kolmogorov"] = kf
    if gf is not None:
        line["guo"] = gf
    if ff is not None:
        line["fe"] = ff
    if pm is not None:
        line["pfm"] = pm
    if cb is not None:
        line["cpu_baseline"] = cb
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
