"""Launch-schedule autotuner for batched smoothing.

Three knobs shape how a batch's levels are launched:
  * ``fused_max_merges``: a sequence's level with at most this many combinations runs as a
    fused single-launch level (one thread-block cluster per combination, FP32 cross term);
    larger levels go through the split kernels (column/row terms, the tensor-core or
    CUDA-core tile sums, the row CDF with the draws);
  * ``max_merges_per_launch``: the chunk of combinations per launch (workspace size versus
    launch count; larger chunks are searched for the fused tensor-core kernel);
  * ``tc_fused`` (tensor-core precisions, N <= 512, d <= 4): the other levels run either as
    one persistent warp-specialised kernel per chunk (operand rows, tcgen05 cross term,
    exponentials, row CDF and draws of a combination on one SM) or as the split kernels;
  * ``tile_cols`` (the tile shape of the row tile sums: 32 or 64 columns per tile, at most 64
    tiles per row; the fused tensor-core kernel takes 32): fewer, wider tiles halve the tile sums written
    and read, and double the columns the draws recompute.
The chunk size and ``tc_fused`` never change a result, and the fused small levels and the
split path are bit-identical with the FP32 cross term (with a tensor-core cross term the
fused small levels differ by that precision's rounding).  The tile width changes the
sampler's random streams per stage (the same law, other draws), not the weights.

``tune_batch`` times every candidate on the device for one batch shape (two timed
runs each, after one warm-up) and returns the fastest; results are cached per shape in
``~/.cache/dsmc_gb300/autotune.json`` (the cache is optional: a read-only home only skips
it)."""
from __future__ import annotations

import hashlib
import json
import os
from typing import Optional

import numpy as np

from . import workloads as W

FUSED_CANDIDATES = (-1, 8, 32, 128)
CHUNK_CANDIDATES = (1024, 4096, 16384)
# the fused tensor-core kernel keeps a combination's intermediates in shared memory, so its
# chunks can be larger (fewer launches, each with its pipeline fill and drain); the workspace
# still sizes the split path's per-combination arrays by the chunk (13 GB at 131072, N = 512)
TC_CHUNK_CANDIDATES = (16384, 65536, 131072)
TC_FUSED_CANDIDATES = (-1, 1)
TILE_CANDIDATES = (32, 64)


def tc_fused_eligible(model: W.SSM, N: int, compute: int) -> bool:
    """Whether the fused tensor-core level kernel applies: BF16 / TF32 cross term, N <= 512,
    padded state dimension <= 4."""
    D = 1
    while D < model.d:
        D *= 2
    return compute != 0 and N <= 512 and D <= 4
_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dsmc_gb300", "autotune.json")


def shape_key(model: W.SSM, Ks, N: int, compute: int, device_name: str) -> str:
    Ks = np.sort(np.asarray(Ks, np.int64))
    h = hashlib.sha1(Ks.tobytes()).hexdigest()[:16]
    return f"{device_name}|kind{model.kind}|d{model.d}|N{N}|c{compute}|n{len(Ks)}|K{h}"


def _load_cache() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict):
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        tmp = _CACHE + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, _CACHE)
    except OSError:
        pass


def candidates(model: W.SSM, N: int, compute: int, fused=FUSED_CANDIDATES, chunks=CHUNK_CANDIDATES,
               tc=TC_FUSED_CANDIDATES, tiles=TILE_CANDIDATES, tc_chunks=TC_CHUNK_CANDIDATES):
    """The (fused_max_merges, max_merges_per_launch, tc_fused, tile_cols) schedules searched
    for this shape: the fused tensor-core kernel where eligible (32-column tiles only), the
    64-column tiles where they give at most 64 tiles per row."""
    tcs = tuple(tc) if tc_fused_eligible(model, N, compute) else (-1,)
    out = []
    for tcf in tcs:
        for tile in tiles:
            if tile != 32 and (tcf > 0 or (N + tile - 1) // tile > 64):
                continue
            if tile == 32 and (N + 31) // 32 > 64:
                continue
            for fm in fused:
                for mc in (tc_chunks if tcf > 0 else chunks):
                    out.append((fm, mc, tcf, tile))
    return out


def tune_batch(model: W.SSM, Ks, N: int, ys, compute: int, use_cache: bool = True,
               fused=FUSED_CANDIDATES, chunks=CHUNK_CANDIDATES, tc=TC_FUSED_CANDIDATES,
               tiles=TILE_CANDIDATES, tc_chunks=TC_CHUNK_CANDIDATES) -> dict:
    """The fastest (fused_max_merges, max_merges_per_launch, tc_fused, tile_cols) for this
    batch shape, with the timings of every candidate (ms per batched smoothing)."""
    import torch

    from . import dsmc
    dev_name = torch.cuda.get_device_name()
    key = shape_key(model, Ks, N, compute, dev_name) + "|tc|tile|tcchunk"
    cands = candidates(model, N, compute, fused, chunks, tc, tiles, tc_chunks)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    timings = {}
    best = None
    yd = [torch.as_tensor(np.asarray(y, np.float32), device="cuda") for y in ys]
    for fm, mc, tcf, tile in cands:
        b = dsmc.BatchSmoother(model, Ks, N, compute=compute, fused_max_merges=fm,
                               max_merges_per_launch=mc, tc_fused=tcf, tile_cols=tile)
        b.set_inputs(yd)
        b.prepare()
        b.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            b.run()
        e1.record()
        torch.cuda.synchronize()
        if b.status() != 0:
            raise RuntimeError(f"autotune candidate ({fm}, {mc}, {tcf}, {tile}): device status {b.status()}")
        ms = e0.elapsed_time(e1) / 2
        timings[f"{fm},{mc},{tcf},{tile}"] = ms
        if best is None or ms < best[4]:
            best = (fm, mc, tcf, tile, ms)
        del b
        torch.cuda.empty_cache()
    out = {"fused_max_merges": best[0], "max_merges_per_launch": best[1], "tc_fused": best[2],
           "tile_cols": best[3], "ms": best[4], "timings": timings}
    if use_cache:
        cache[key] = out
        _store_cache(cache)
    return out
