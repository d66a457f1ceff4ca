"""Autotuner of the step kernel's launch shape (CTA tile and z-chunk length).

Every candidate shape computes bit-identical results, so tuning only changes
speed.  Candidates are timed on the caller's own lattice with CUDA events on
its stream; the population buffer is saved before and restored after, and each
trial runs an even number of steps so the ping-pong buffers end where they
started.  For batches, ``tune_batch`` times whole batched steps.
"""
from __future__ import annotations

from typing import Iterable, List, Optional, Sequence, Tuple

from . import lbm_sc


def candidates(lattice: "lbm_sc.Lattice") -> List[Tuple[int, int]]:
    """(tile, zchunk) pairs worth timing for this lattice (zchunk 0 = automatic)."""
    tiles = [t for t in range(len(lbm_sc.TILES)) if lattice.tile_fits(t)]
    if lattice.lattice == lbm_sc.LBM_D2Q9:
        return [(t, 0) for t in tiles]
    nz = lattice.shape[0]
    zs = sorted({0} | {z for z in (32, 64, 128, 256) if z < nz} | {nz})
    return [(t, z) for t in tiles for z in zs]


def _time_steps(lattice, nsteps: int) -> float:
    import torch
    st = lattice.stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    lattice.step(nsteps)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / nsteps


def autotune(lattice: "lbm_sc.Lattice", trial_steps: int = 4, warmup_steps: int = 2,
             cands: Optional[Iterable[Tuple[int, int]]] = None, restore: bool = True):
    """Time each candidate, apply the fastest, return (best, table).

    table: list of ((tile, zchunk_requested), zchunk_used, ms_per_step).
    """
    if (trial_steps + warmup_steps) % 2:
        trial_steps += 1
    saved = lattice.state().clone() if restore else None
    table = []
    for tile, z in (cands if cands is not None else candidates(lattice)):
        lattice.set_tuning(tile, z)
        lattice.step(warmup_steps)
        ms = _time_steps(lattice, trial_steps)
        table.append(((tile, z), lattice.tuning()[1], ms))
    best = min(table, key=lambda r: r[2])
    lattice.set_tuning(best[0][0], best[1])
    if saved is not None:
        lattice.state().copy_(saved)
        lattice.stream.synchronize()
    return (best[0][0], best[1]), table


def format_table(table: Sequence) -> str:
    rows = ["id tile  kind stages cluster  zchunk  ms/step"]
    for (tile, _), zc, ms in sorted(table, key=lambda r: r[2]):
        tx, ty = lbm_sc.TILES[tile]
        cx, cy = lbm_sc.TILE_CLUSTER[tile]
        rows.append("%2d %2dx%-2d k%d s%d c%dx%d  %6d  %.4f" % (tile, tx, ty, lbm_sc.TILE_KIND[tile],
                                                            lbm_sc.TILE_STAGES[tile], cx, cy, zc, ms))
    return "\n".join(rows)


# ---- ragged batch ---------------------------------------------------------------
def batch_candidates(lattices, zchunks=(0, 16, 32, 64), graph_steps=(0, 8, 32)):
    """(tile, zchunk, graph_steps) triples for a batch (zchunk only for D3Q19)."""
    zs = zchunks if lattices[0].lattice == lbm_sc.LBM_D3Q19 else (0,)
    tiles = [t for t in range(len(lbm_sc.BATCH_TILES)) if all(lbm_sc.batch_tile_fits(t, lat) for lat in lattices)]
    return [(t, z, g) for t in tiles for z in zs for g in graph_steps]


def tune_batch(lattices, trial_steps: int = 8, warmup_steps: int = 2, cands=None, stream=None,
               restore: bool = True):
    """Time whole batched steps for each (tile, zchunk, graph_steps) candidate on
    the caller's lattices (states saved and restored; even step counts) and
    return (best, table) with table rows ((tile, zchunk, graph_steps), ms_per_step).
    Graph chunks only take effect on a non-default stream."""
    import torch
    if (trial_steps + warmup_steps) % 2:
        trial_steps += 1
    stream = stream if stream is not None else lattices[0].stream
    saved = [lat.state().clone() for lat in lattices] if restore else None
    table = []
    for tile, z, g in (cands if cands is not None else batch_candidates(lattices)):
        if g and trial_steps % g:
            continue
        b = lbm_sc.Batch(lattices, tile=tile, zchunk=z, graph_steps=g, stream=stream)
        b.step(max(warmup_steps, g))  # the first chunk captures the graph
        if max(warmup_steps, g) % 2:
            b.step(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(trial_steps)
        e1.record(stream)
        e1.synchronize()
        b.close()
        table.append(((tile, z, g), e0.elapsed_time(e1) / trial_steps))
    best = min(table, key=lambda r: r[1])
    if saved is not None:
        for lat, sv in zip(lattices, saved):
            lat.state().copy_(sv)
        stream.synchronize()
    return best[0], table


# ---- tuning cache --------------------------------------------------------------
CACHE_PATH = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                        "tuning_cache.json")


def cache_key(lattice: "lbm_sc.Lattice") -> str:
    prec = {v: k for k, v in lbm_sc.PRECISIONS.items()}[lattice.params.precision]
    kind = "D2Q9" if lattice.lattice == lbm_sc.LBM_D2Q9 else "D3Q19"
    key = "%s/%s/%s" % (kind, prec, "x".join(str(s) for s in reversed(lattice.shape)))
    # the collision changes the best shape: separate entries for Guo forcing and the FE model
    if lattice.params.model == lbm_sc.LBM_MODEL_FE:
        return key + "/fe"
    return key + "/guo" if lattice.params.forcing == lbm_sc.LBM_FORCING_GUO else key


def tuned(lattice: "lbm_sc.Lattice", path: str = CACHE_PATH, store: bool = True, **kw):
    """Apply the cached launch shape for this lattice kind, precision and size, or
    autotune (state restored) and remember the winner.  Returns ((tile, zchunk), source)."""
    import json
    import os
    key = cache_key(lattice)
    cache = {}
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
    if key in cache:
        tile, zc = cache[key]["tile"], cache[key]["zchunk"]
        if lattice.tile_fits(tile):
            lattice.set_tuning(tile, zc)
            return (tile, lattice.tuning()[1]), "cache"
    best, table = autotune(lattice, **kw)
    if store:
        cache[key] = {"tile": best[0], "zchunk": best[1], "ms_per_step": min(r[2] for r in table),
                      "candidates": len(table)}
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return best, "autotuned"
