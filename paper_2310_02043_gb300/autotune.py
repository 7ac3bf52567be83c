"""Launch-shape autotuner for the tracing kernels.

Times a caller-supplied unit of work (one forward + adjoint step, one batch
step) under each candidate launch shape — threads per block, resident blocks
per SM, and whether the BVH is staged in shared memory or read through L1 —
with CUDA events, keeps the fastest, and caches the choice per workload key
in a JSON file so later runs skip the search.
"""
from __future__ import annotations

import json
import os
import statistics

# (threads per block (0: the bound of the kernel the BVH selects, 1024 when it
# is staged and when nodes come through L1), blocks per SM (0: as many as
# fit), shared-memory node budget in bytes (0: nodes through L1; the library
# stages the triangles with the nodes where that costs no resident block));
# every field is set explicitly.
CANDIDATES = (
    (0, 0, 200 * 1024), (0, 0, 0),
    (512, 0, 200 * 1024), (512, 0, 0),
    (384, 0, 200 * 1024), (384, 0, 0),
    (256, 0, 200 * 1024), (256, 0, 0),
)


def _time_ms(run, repeats: int, timer):
    vals = []
    for _ in range(repeats):
        vals.append(timer(run))
    return statistics.median(vals)


def cuda_timer(run):
    """Milliseconds of `run()` measured with CUDA events on the current stream."""
    import torch
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    run()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def tune(tracer, run, key: str, candidates=CANDIDATES, repeats: int = 3, cache_path: str | None = None,
         timer=cuda_timer):
    """Pick the fastest launch shape for `run` (a callable issuing the work on
    the tracer) and apply it. Returns (shape, {shape: ms}). A shape that the
    library refuses (it does not fit an SM) is skipped."""
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            shape = tuple(cache[key]["shape"])
            tracer.set_launch(*shape)
            return shape, {tuple(json.loads(k)): v for k, v in cache[key]["ms"].items()}
    results = {}
    for shape in candidates:
        try:
            tracer.set_launch(*shape)
            run()                                   # warm-up (and graph capture, if any)
        except RuntimeError:
            continue
        results[tuple(shape)] = _time_ms(run, repeats, timer)
    if not results:
        raise RuntimeError("no candidate launch shape ran")
    best = min(results, key=results.get)
    tracer.set_launch(*best)
    if cache_path:
        cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        cache[key] = {"shape": list(best), "ms": {json.dumps(list(k)): v for k, v in results.items()}}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, results


def workload_key(device_name: str, n_tri: int, n_texels: int, photons: int, hits: int, n_designs: int = 1) -> str:
    return f"{device_name}|tri{n_tri}|tex{n_texels}|ph{photons}|hits{hits}|d{n_designs}"
