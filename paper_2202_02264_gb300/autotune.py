"""Launch-schedule autotuner for batched smoothing.

Three knobs shape how a batch's levels are launched:
  * ``fused_max_merges``: a sequence's level with at most this many combinations runs as a
    fused single-launch level (one thread-block cluster per combination, FP32 cross term);
    larger levels go through the split kernels (column/row terms, the tensor-core or
    CUDA-core tile sums, the row CDF with the draws);
  * ``max_merges_per_launch``: the chunk of combinations per launch (workspace size versus
    launch count);
  * ``tc_fused`` (tensor-core precisions, N <= 512, d <= 4): the other levels run either as
    one persistent warp-specialised kernel per chunk (operand rows, tcgen05 cross term,
    exponentials, row CDF and draws of a combination on one SM) or as the split kernels.
None changes what is computed for a given choice of path: the chunk size and ``tc_fused``
never change a result, and the fused small levels and the split path are bit-identical with
the FP32 cross term (with a tensor-core cross term the fused small levels differ by that
precision's rounding).

``tune_batch`` times every candidate pair on the device for one batch shape (two timed
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
TC_FUSED_CANDIDATES = (-1, 1)


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


def tune_batch(model: W.SSM, Ks, N: int, ys, compute: int, use_cache: bool = True,
               fused=FUSED_CANDIDATES, chunks=CHUNK_CANDIDATES, tc=TC_FUSED_CANDIDATES) -> dict:
    """The fastest (fused_max_merges, max_merges_per_launch, tc_fused) for this batch shape,
    with the timings of every candidate (ms per batched smoothing)."""
    import torch

    from . import dsmc
    dev_name = torch.cuda.get_device_name()
    key = shape_key(model, Ks, N, compute, dev_name) + "|tc"
    tcs = tuple(tc) if tc_fused_eligible(model, N, compute) else (-1,)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    timings = {}
    best = None
    yd = [torch.as_tensor(np.asarray(y, np.float32), device="cuda") for y in ys]
    for tcf in tcs:
        for fm in fused:
            for mc in chunks:
                b = dsmc.BatchSmoother(model, Ks, N, compute=compute, fused_max_merges=fm,
                                       max_merges_per_launch=mc, tc_fused=tcf)
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
                    raise RuntimeError(f"autotune candidate ({fm}, {mc}, {tcf}): device status {b.status()}")
                ms = e0.elapsed_time(e1) / 2
                timings[f"{fm},{mc},{tcf}"] = ms
                if best is None or ms < best[3]:
                    best = (fm, mc, tcf, ms)
                del b
                torch.cuda.empty_cache()
    out = {"fused_max_merges": best[0], "max_merges_per_launch": best[1], "tc_fused": best[2], "ms": best[3],
           "timings": timings}
    if use_cache:
        cache[key] = out
        _store_cache(cache)
    return out
