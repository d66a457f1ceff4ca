"""Continuous-batching server for drop-relaxation runs.

Requests (a drop of component A in B on a periodic D2Q9 or D3Q19 lattice, with
their own size, G, tau_A, tau_B and radius) arrive over time.  The server
keeps every admitted lattice's populations resident in device memory, admits
waiting requests in arrival order while their workspace fits the HBM budget,
and advances all resident lattices together: one ragged batch per lattice kind
(lbm_sc_batch_*: one kernel launch per step for the whole batch), in chunks of
``chunk`` steps.  Every ``check_every`` steps of a request's own age its peak
speed max|u_phys| is read (FP64 diagnostics, enqueued for all due requests and
read back with one synchronisation); a request is done when that peak changed
by less than ``tol`` times its value at the previous check, or after
``max_steps`` steps.  A finished request's density field is copied to host
memory (the result), its memory released and the batch rebuilt without it,
so requests that arrived meanwhile take its place at the next chunk boundary.

Because a batched step is bit-identical to a solo step, a request's result
(fields and step count) is the same alone and in any mix.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import inputs, lbm_sc

# Doubles in one lbm_sc_diag record (the rows of the device diagnostics array).
DIAG_DOUBLES = ctypes.sizeof(lbm_sc.lbm_sc_diag) // 8


def max_speed_of(row) -> float:
    """max|u_phys| of one lbm_sc_diag record held as DIAG_DOUBLES doubles."""
    return check_of(row)[0]


def check_of(row):
    """(max|u_phys|, unstable) of one lbm_sc_diag record held as DIAG_DOUBLES
    doubles; unstable: a non-finite value, or a species density that is no
    longer positive anywhere (the state the diagnostics call LBM_ERR_UNSTABLE)."""
    d = lbm_sc.lbm_sc_diag.from_buffer_copy(np.ascontiguousarray(row, dtype=np.float64).tobytes())
    unstable = d.nonfinite > 0 or not (d.min_rho_A > 0 and d.min_rho_B > 0)
    return float(d.max_speed), bool(unstable)


@dataclass
class Request:
    rid: int
    lattice: int          # lbm_sc.LBM_D2Q9 or LBM_D3Q19
    shape: tuple          # numpy order: (ny, nx) or (nz, ny, nx)
    G: float
    tau_A: float
    tau_B: float
    R: float
    centre: tuple         # (cx, cy[, cz]) node units
    seed: int
    arrival: float = 0.0  # seconds after the start of the run
    precision: str = "f32"
    kind: str = "drop"    # "drop" (radius R) or "interface" (a slab of half-width R: two flat interfaces)

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    def fields(self):
        """Initial (rho_A, rho_B) in FP32: the drop recipe of paper_1112_5547_gb300.inputs,
        or its slab recipe (interfaces normal to x, centred at the request's centre x)."""
        if self.kind == "interface":
            return inputs.slab(self.shape, self.R, centre_x=self.centre[0], seed=self.seed, dtype=np.float32)
        return inputs.drop(self.shape, self.R, centre=self.centre, seed=self.seed, dtype=np.float32)


def poisson_requests(n: int, rate: float = 50.0, seed: int = 4, d3_fraction: float = 0.5,
                     sizes2=(64, 128, 256, 512, 1024), sizes3=(32, 48, 64, 96, 128, 160, 192),
                     precision: str = "f32", interface_fraction: float = 0.0) -> List[Request]:
    """n requests with exponential inter-arrival times of mean 1/rate (seeded).

    Each is D3Q19 with probability d3_fraction, else D2Q9; the edge L is drawn
    uniformly from sizes3 / sizes2, G rho_tot uniformly in [2.2, 2.8], tau_A,
    tau_B uniformly in [0.6, 1.5], the drop radius uniformly in [L/8, L/3] at a
    uniformly random centre (the ragged-batch recipe of inputs.ragged_drop_specs).
    With probability interface_fraction a request relaxes a flat interface
    instead (a slab of half-width R); with 0 the stream is the drops-only one
    (no extra random draws).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out, t = [], 0.0
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        d3 = bool(rng.uniform() < d3_fraction)
        sizes = sizes3 if d3 else sizes2
        L = int(sizes[int(rng.integers(len(sizes)))])
        dim = 3 if d3 else 2
        g_rho = float(rng.uniform(2.2, 2.8))
        tau_A = float(rng.uniform(0.6, 1.5))
        tau_B = float(rng.uniform(0.6, 1.5))
        R = float(rng.uniform(L / 8.0, L / 3.0))
        centre = tuple(float(c) for c in rng.uniform(0.0, L, size=dim))
        kind = "interface" if interface_fraction > 0 and rng.uniform() < interface_fraction else "drop"
        out.append(Request(k, lbm_sc.LBM_D3Q19 if d3 else lbm_sc.LBM_D2Q9, (L,) * dim, g_rho / inputs.RHO_TOT,
                           tau_A, tau_B, R, centre, int(seed) * 1000003 + k, t, precision, kind))
    return out


@dataclass
class Result:
    rid: int
    nodes: int
    steps: int
    converged: bool
    arrival: float
    admitted: float
    done: float
    umax: float
    rhoA: Optional[np.ndarray] = None
    unstable: bool = False  # retired at a check that saw a non-positive density or a non-finite value

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    req: Request
    lat: "lbm_sc.Lattice"
    nbytes: int
    admitted: float
    steps: int = 0
    last_umax: Optional[float] = None


@dataclass
class ServeStats:
    wall_s: float
    lattice_updates: float
    mlups: float
    p50_s: float
    p99_s: float
    mean_s: float
    max_resident: int
    chunks: int
    rebuilds: int
    extra: Dict = field(default_factory=dict)


def _percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else float("nan")


class Server:
    """Continuous batching over resident lattices (see the module docstring)."""

    def __init__(self, hbm_budget: float = 80e9, chunk: int = 100, check_every: int = 500, tol: float = 0.01,
                 max_steps: int = 10000, graph_steps: int = 0, keep_fields: bool = False, device="cuda",
                 prep_workers: int = 4, max_active_nodes: Optional[int] = None, order: str = "arrival"):
        """max_active_nodes: admit a waiting request only while the resident
        lattices hold fewer nodes than this (besides the HBM budget), so that the
        GPU is kept full without sharing it among every queued request: earlier
        requests then finish sooner.  None: the HBM budget alone decides.
        order: which waiting request is admitted next, "arrival" (first come,
        first served) or "size" (fewest nodes first, a shortest-job-first proxy:
        the step count to convergence is not known in advance)."""
        if order not in ("arrival", "size"):
            raise ValueError("order must be 'arrival' or 'size'")
        self.order = order
        import torch
        if check_every % chunk:
            raise ValueError("chunk must divide check_every")
        self.torch = torch
        self.budget = float(hbm_budget) - self.RESERVE_BYTES  # the lattices' and their batches' share
        self.max_active_nodes = max_active_nodes
        self.chunk = int(chunk)
        self.check_every = int(check_every)
        self.tol = float(tol)
        self.max_steps = int(max_steps)
        self.graph_steps = int(graph_steps)
        self.keep_fields = keep_fields
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.prep_workers = prep_workers
        self._diag = None

    # -- helpers -------------------------------------------------------------
    # Device memory the server holds besides the lattices' own workspaces, kept
    # out of the HBM budget: the diagnostics rows of one check (one lbm_sc_diag
    # per due request), the batches' CUDA graphs and allocator rounding.
    RESERVE_BYTES = 64 << 20
    # A lattice's share of its batch workspace: its descriptor (both parities,
    # two tensor maps and two argument blocks, under 2 KiB) and its work items
    # (16 bytes each), at most one per 32 x 4 column tile and plane (every batch
    # tile is at least that large, every z chunk at least one plane).
    BATCH_DESCRIPTOR_BYTES = 2048

    @staticmethod
    def batch_share(req: Request) -> int:
        """Upper bound of the bytes a request adds to its batch's workspace."""
        ny, nx = req.shape[-2], req.shape[-1]
        nz = req.shape[0] if len(req.shape) == 3 else 1
        items = -(-nx // 32) * -(-ny // 4) * nz
        return Server.BATCH_DESCRIPTOR_BYTES + 16 * items

    @staticmethod
    def footprint(req: Request) -> int:
        """Device bytes a resident request holds: its workspace (two population
        buffers and diagnostics scratch) and its share of the batch workspace."""
        p = lbm_sc.make_params(req.lattice, req.shape, req.tau_A, req.tau_B, req.G, req.precision)
        return int(lbm_sc.lbm_sc_workspace_bytes(p)) + Server.batch_share(req)

    @staticmethod
    def batch_shape(lats):
        """(tile, zchunk) of a batch: the TMA-fed tiles with one CTA per work item and
        16-plane chunks when every lattice takes them (D3Q19, FP32): 384-thread
        64x6 / 32x12 per lattice (at least 32 x 12), else 32x8 (at least 32 x 8);
        for the rest-offset 16-bit storages the 32x8 TMA tile (at least 32 x 8);
        otherwise the persistent 32 x 4 z-marching one (the fastest on ragged D2Q9
        batches: 28 GLUPS on 32 lattices of 64^2 .. 1024^2 against 21 one at a time)."""
        for tile in (11, 5, lbm_sc.BATCH_TILE_REST):
            if all(lbm_sc.batch_tile_fits(tile, lat) for lat in lats):
                # 32-plane chunks on the rest-offset tile (20.3 against 19.6 GLUPS with 16
                # on the 64 ragged lattices), 16 on the FP32 ones
                return tile, 32 if tile == lbm_sc.BATCH_TILE_REST else 16
        return 1, 0

    def _check(self, slots: List[_Slot]):
        """(max|u_phys|, unstable) of each slot's current state, one synchronisation for all."""
        torch = self.torch
        n = len(slots)
        width = DIAG_DOUBLES
        if self._diag is None or self._diag.shape[0] < n:
            self._diag = torch.empty((max(n, 64), width), dtype=torch.float64, device=self.device)
        assert self._diag.shape[1] * 8 == ctypes.sizeof(lbm_sc.lbm_sc_diag)
        for k, s in enumerate(slots):
            eb, q, px, py, gx, gy, ptr = lbm_sc.lbm_sc_layout(s.lat.handle)
            lbm_sc.lbm_sc_diagnostics_noalloc(s.lat.params, ptr, None, self._diag[k].data_ptr(),
                                              self.stream.cuda_stream)
        host = self._diag[:n].cpu().numpy()  # on the current stream, which is self.stream
        return [check_of(host[k]) for k in range(n)]

    def _admit(self, req: Request, f, now: float) -> _Slot:
        with self.torch.cuda.stream(self.stream):
            lat = lbm_sc.Lattice(req.lattice, req.shape, req.tau_A, req.tau_B, req.G, req.precision,
                                 device=self.device, stream=self.stream)
            lat.init(f[0], f[1])
        return _Slot(req, lat, lat.workspace_bytes + self.batch_share(req), now)

    def _retire(self, s: _Slot, now, converged: bool, umax: float, unstable: bool = False) -> Result:
        """Copy the result (the density field of component A) to host memory,
        release the lattice; ``now()`` after the copy is the completion time."""
        with self.torch.cuda.stream(self.stream):
            rho = s.lat.moments()[0].cpu().numpy()  # synchronises the stream
        done = now()
        s.lat.close()
        return Result(s.req.rid, s.req.nodes, s.steps, converged, s.req.arrival, s.admitted, done, umax,
                      rho if self.keep_fields else None, unstable)

    # -- the serving loop ----------------------------------------------------
    def run(self, requests: List[Request], clock=time.perf_counter):
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        prep: Dict[int, cf.Future] = {}
        resident: List[_Slot] = []
        results: List[Result] = []
        used = 0
        batches: Dict[int, lbm_sc.Batch] = {}
        dirty = True
        chunks = rebuilds = max_res = 0
        lu = 0.0
        pool = cf.ThreadPoolExecutor(max_workers=self.prep_workers)
        t0 = clock()
        with torch.cuda.stream(self.stream):
            while pending or waiting or resident:
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    r = pending.popleft()
                    waiting.append(r)
                    prep[r.rid] = pool.submit(r.fields)
                # admission: arrival (or size) order, while the head of the queue fits
                if self.order == "size" and len(waiting) > 1:
                    waiting = deque(sorted(waiting, key=lambda r: (r.nodes, r.arrival)))
                while (waiting and used + self.footprint(waiting[0]) <= self.budget
                       and (self.max_active_nodes is None or not resident
                            or sum(x.req.nodes for x in resident) + waiting[0].nodes <= self.max_active_nodes)):
                    r = waiting.popleft()
                    s = self._admit(r, prep.pop(r.rid).result(), clock() - t0)
                    resident.append(s)
                    used += s.nbytes
                    dirty = True
                if waiting and not resident and used + self.footprint(waiting[0]) > self.budget:
                    raise RuntimeError("request %d does not fit the HBM budget" % waiting[0].rid)
                if not resident:
                    if pending:
                        time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                    continue
                max_res = max(max_res, len(resident))
                if dirty:
                    for b in batches.values():
                        b.close()
                    batches = {}
                    # one batch per lattice kind and storage precision (a batch holds one of each)
                    for key in sorted({(s.req.lattice, s.req.precision) for s in resident}):
                        lats = [s.lat for s in resident if (s.req.lattice, s.req.precision) == key]
                        tile, zc = self.batch_shape(lats)
                        batches[key] = lbm_sc.Batch(lats, tile=tile, zchunk=zc, graph_steps=self.graph_steps,
                                                    stream=self.stream)
                    rebuilds += 1
                    dirty = False
                for b in batches.values():
                    b.step(self.chunk)
                chunks += 1
                for s in resident:
                    s.steps += self.chunk
                    lu += float(s.req.nodes) * self.chunk
                due = [s for s in resident if s.steps % self.check_every == 0]
                if due:
                    checks = self._check(due)
                    for s, (u, bad) in zip(due, checks):
                        conv = (not bad and s.last_umax is not None
                                and abs(u - s.last_umax) < self.tol * max(s.last_umax, 1e-300))
                        if conv or bad or s.steps >= self.max_steps:
                            results.append(self._retire(s, lambda: clock() - t0, conv, u, bad))
                            resident.remove(s)
                            used -= s.nbytes
                            dirty = True
                        else:
                            s.last_umax = u
            self.stream.synchronize()
        wall = clock() - t0
        pool.shutdown()
        for b in batches.values():
            b.close()
        lat_s = [r.latency for r in results]
        stats = ServeStats(wall, lu, lu / wall / 1e6, _percentile(lat_s, 50), _percentile(lat_s, 99),
                           float(np.mean(lat_s)) if lat_s else float("nan"), max_res, chunks, rebuilds)
        return sorted(results, key=lambda r: r.rid), stats


def solve_alone(req: Request, chunk: int = 100, check_every: int = 500, tol: float = 0.01, max_steps: int = 10000,
                keep_fields: bool = False, stream=None, fields=None, clock=time.perf_counter):
    """One request on its own (plain lbm_sc_step, same convergence rule): the
    one-at-a-time baseline.  Returns (Result, seconds spent on the device path)."""
    import torch
    stream = stream if stream is not None else torch.cuda.Stream()
    f = fields if fields is not None else req.fields()
    with torch.cuda.stream(stream):
        t0 = clock()
        lat = lbm_sc.Lattice(req.lattice, req.shape, req.tau_A, req.tau_B, req.G, req.precision, stream=stream)
        lat.init(f[0], f[1])
        steps, last, conv, bad, u = 0, None, False, False, float("nan")
        diag = torch.empty(DIAG_DOUBLES, dtype=torch.float64, device="cuda")
        while True:
            lat.step(chunk)
            steps += chunk
            if steps % check_every == 0:
                eb, q, px, py, gx, gy, ptr = lbm_sc.lbm_sc_layout(lat.handle)
                lbm_sc.lbm_sc_diagnostics_noalloc(lat.params, ptr, None, diag.data_ptr(), stream.cuda_stream)
                u, bad = check_of(diag.cpu().numpy())
                conv = not bad and last is not None and abs(u - last) < tol * max(last, 1e-300)
                if conv or bad or steps >= max_steps:
                    break
                last = u
        rho = lat.moments()[0].cpu().numpy()
        t1 = clock()
        lat.close()
    return Result(req.rid, req.nodes, steps, conv, 0.0, 0.0, t1 - t0, u, rho if keep_fields else None, bad), t1 - t0


def serial_baseline(requests: List[Request], **kw):
    """Every request solved alone, one after another (input generation not
    timed).  Returns (results, total device-path seconds, MLUPS)."""
    total, lu, res = 0.0, 0.0, []
    for r in requests:
        f = r.fields()
        out, dt = solve_alone(r, fields=f, **kw)
        total += dt
        lu += float(r.nodes) * out.steps
        res.append(out)
    return res, total, lu / total / 1e6 if total > 0 else float("nan")


def main(argv=None):
    """Serve a seeded Poisson stream at one or more arrival rates, then solve the
    same requests one at a time, and print one JSON line per rate."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rate", type=str, default="50", help="arrival rate(s) per second, comma-separated")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--hbm-budget-gb", type=float, default=80.0)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--max-steps", type=int, default=10000)
    ap.add_argument("--no-serial", action="store_true")
    ap.add_argument("--order", type=str, default="arrival", help="admission order(s): arrival, size")
    ap.add_argument("--max-active-mnodes", type=str, default="none",
                    help="cap(s) on resident lattice nodes, millions, comma-separated ('none': HBM budget only)")
    a = ap.parse_args(argv)
    rates = [float(r) for r in a.rate.split(",")]
    caps = [None if c.strip().lower() == "none" else int(float(c) * 1e6) for c in a.max_active_mnodes.split(",")]
    serial = None
    orders = a.order.split(",")
    for rate, cap, order in [(r, c, o) for r in rates for c in caps for o in orders]:
        reqs = poisson_requests(a.requests, rate, a.seed, precision=a.precision)
        srv = Server(hbm_budget=a.hbm_budget_gb * 1e9, chunk=a.chunk, max_steps=a.max_steps, max_active_nodes=cap,
                     order=order)
        res, st = srv.run(reqs)
        out = {"requests": len(reqs), "rate_per_s": rate, "seed": a.seed, "precision": a.precision,
               "max_active_nodes": cap, "order": order,
               "served_mlups": st.mlups, "wall_s": st.wall_s, "p50_s": st.p50_s, "p99_s": st.p99_s,
               "mean_s": st.mean_s, "max_resident": st.max_resident, "chunks": st.chunks, "rebuilds": st.rebuilds,
               "converged": sum(r.converged for r in res), "unstable": sum(r.unstable for r in res),
               "steps_total": sum(r.steps for r in res),
               "lattice_updates": st.lattice_updates}
        if not a.no_serial:
            if serial is None:  # the same requests (arrival times do not matter one at a time)
                serial = serial_baseline(reqs, chunk=a.chunk, max_steps=a.max_steps)
            sres, stot, smlups = serial
            out.update({"serial_mlups": smlups, "serial_s": stot, "speedup": st.mlups / smlups,
                        "same_steps": all(x.steps == y.steps for x, y in zip(res, sres))})
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
