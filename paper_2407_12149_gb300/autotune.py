"""Run-time choice of a batch's kernel settings, with a cache.

Three settings change how a cycle runs but not what it computes:
  coarse_max_n  grids with n <= coarse_max_n run inside the shared-memory coarse
                kernel (one CTA per chain, barrier-latency bound), the larger ones in
                per-depth launches;
  band_min_n    of the 9-point grids below the finest (FP32), those with
                n >= band_min_n run in the streaming band kernels, the others in the
                tile kernels (bitwise identical states);
  coarse_threads threads per CTA of the coarse kernel (0: by the chain count; the
                kernel's arithmetic does not depend on it).
Which values are fastest depends on the chain count and the grid sizes, so each
candidate's captured V-cycle is timed with CUDA events over back-to-back cycles
(states resident on the device) and the fastest kept.  band_min_n and coarse_threads
candidates are timed on one handle (mgmc_set_band_min_n, mgmc_set_coarse_threads);
coarse_max_n candidates each need their own handle.  The choice is stored in a JSON
cache keyed by (dim, grid sizes, precision, chain count) and applied when a
BatchSampler is created with that cache and without explicit settings
(mgmc.BatchSampler -> mgmc_create_batch, then mgmc_set_coarse_threads).
"""
from __future__ import annotations

import json
import os
from collections import Counter
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

# a band threshold above every grid: the tile kernels only
TILES_ONLY = 1 << 20
DEFAULTS = {"coarse_max_n": 31, "band_min_n": 0, "coarse_threads": 0}
COARSE_THREADS = (0, 128, 256, 512, 1024)


def pick_fastest(timings: Dict[int, float]) -> int:
    """The candidate with the smallest time; on equal times the smaller value."""
    if not timings:
        raise ValueError("no candidate was timed")
    return min(timings, key=lambda c: (timings[c], c))


def cache_key(problems: Sequence, precision: str) -> str:
    """'2d|fp32|c=32|1023x32' : dimension, precision, chain count and the multiset of
    finest grid sizes (chain order does not matter)."""
    dims = {p.dim for p in problems}
    if len(dims) != 1:
        raise ValueError("a batch has one dimension")
    sizes = Counter(int(p.n) for p in problems)
    sz = ",".join(f"{n}x{k}" for n, k in sorted(sizes.items()))
    return f"{dims.pop()}d|{precision}|c={len(problems)}|{sz}"


def default_cache_path() -> str:
    return os.environ.get("MGMC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mgmc_gb300", "tune.json"))


class TuneCache:
    """JSON file of {key: {"coarse_max_n": int, "band_min_n": int, "coarse_threads": int,
    "ms": {...}}}."""

    def __init__(self, path: Optional[str] = None):
        self.path = path or default_cache_path()
        self.entries: Dict[str, dict] = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                data = json.load(f)
            if isinstance(data, dict):
                self.entries = data

    def get(self, key: str) -> Optional[dict]:
        e = self.entries.get(key)
        if not isinstance(e, dict):
            return None
        out = {}
        for k in DEFAULTS:
            if k in e:
                v = int(e[k])
                if v < 0:
                    return None
                out[k] = v
        return out or None

    def put(self, key: str, settings: dict, timings: Optional[dict] = None) -> None:
        e = dict(self.entries.get(key, {}))
        for k, v in settings.items():
            if k not in DEFAULTS:
                raise KeyError(k)
            e[k] = int(v)
        if timings:
            e.setdefault("ms", {}).update({str(k): float(v) for k, v in timings.items()})
        self.entries[key] = e

    def save(self) -> None:
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def resolve_settings(problems: Sequence, precision: str, coarse_max_n: Optional[int] = None,
                     band_min_n: Optional[int] = None, cache: Optional[TuneCache] = None,
                     coarse_threads: Optional[int] = None) -> dict:
    """Explicit values win; otherwise the cached choice for this batch; otherwise the
    library defaults."""
    out = dict(DEFAULTS)
    if cache is not None:
        got = cache.get(cache_key(problems, precision))
        if got:
            out.update(got)
    if coarse_max_n is not None:
        out["coarse_max_n"] = int(coarse_max_n)
    if band_min_n is not None:
        out["band_min_n"] = int(band_min_n)
    if coarse_threads is not None:
        out["coarse_threads"] = int(coarse_threads)
    return out


def band_candidates(problems: Sequence, coarse_max_n: int) -> list:
    """The thresholds that give different splits: each grid size below the finest and
    above coarse_max_n (from there on the band kernels), and the tiles only."""
    sizes = set()
    for p in problems:
        n = (p.n - 1) // 2
        while n > coarse_max_n:
            sizes.add(n)
            n = (n - 1) // 2
    return sorted(sizes) + [TILES_ONLY]


def time_cycles(sampler, cycles: int = 20, warm: int = 3, seed: int = 1, device: int = 0) -> float:
    """Milliseconds per V-cycle of a BatchSampler whose states are resident (CUDA events
    on the current stream around `cycles` back-to-back cycles after `warm` untimed ones)."""
    import torch
    sampler.sample(None, warm, seed)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sampler.sample(None, cycles, seed, step_offset=warm)
    e1.record(stream)
    torch.cuda.synchronize(device)
    return e0.elapsed_time(e1) / cycles


def tune_band_min_n(sampler, candidates: Iterable[int], timer: Optional[Callable[[object], float]] = None
                    ) -> Tuple[int, Dict[int, float]]:
    """(best band_min_n, {candidate: ms per cycle}) timed on one handle; the handle is left
    at the best value.  `timer(sampler)` replaces the GPU timing (tests)."""
    cands = sorted({int(c) for c in candidates})
    if not cands or cands[0] < 0:
        raise ValueError("band_min_n candidates must be >= 0")
    timer = timer or time_cycles
    timings = {}
    for c in cands:
        sampler.set_band_min_n(c)
        timings[c] = float(timer(sampler))
    best = pick_fastest(timings)
    sampler.set_band_min_n(best)
    return best, timings


def tune_coarse_threads(sampler, candidates: Iterable[int] = COARSE_THREADS,
                        timer: Optional[Callable[[object], float]] = None) -> Tuple[int, Dict[int, float]]:
    """(best thread count, {candidate: ms per cycle}) of the coarse kernel, timed on one
    handle, which is left at the best value."""
    cands = sorted({int(c) for c in candidates})
    if not cands or cands[0] < 0:
        raise ValueError("coarse thread candidates must be >= 0")
    timer = timer or time_cycles
    timings = {}
    for c in cands:
        sampler.set_coarse_threads(c)
        timings[c] = float(timer(sampler))
    best = pick_fastest(timings)
    sampler.set_coarse_threads(best)
    return best, timings


def time_batch_cycle(problems: Sequence, coarse_max_n: int, precision: str = "fp32", cycles: int = 20,
                     warm: int = 3, device: int = 0, seed: int = 1, band_min_n: int = 0) -> float:
    """Milliseconds per V-cycle of a new batch with this coarse threshold."""
    from .mgmc import BatchSampler
    s = BatchSampler(problems, precision=precision, coarse_max_n=coarse_max_n, band_min_n=band_min_n,
                     device=device)
    try:
        s.sample(s.zeros(), 1, seed)
        return time_cycles(s, cycles=cycles, warm=warm, seed=seed, device=device)
    finally:
        s.close()


def autotune_coarse_max_n(problems: Sequence, precision: str = "fp32", candidates: Iterable[int] = (15, 31, 63),
                          cycles: int = 20, warm: int = 3, device: int = 0,
                          timer: Optional[Callable[[Sequence, int], float]] = None) -> Tuple[int, Dict[int, float]]:
    """(best threshold, {threshold: ms per cycle}) over the candidates (positive, each
    timed on its own handle).  `timer(problems, threshold)` replaces the GPU timing (tests)."""
    cands = sorted({int(c) for c in candidates})
    if not cands or cands[0] < 1:
        raise ValueError("candidates must be positive grid sizes")
    if timer is None:
        def timer(ps, c):
            return time_batch_cycle(ps, c, precision=precision, cycles=cycles, warm=warm, device=device)
    timings = {c: float(timer(problems, c)) for c in cands}
    return pick_fastest(timings), timings


def autotune(problems: Sequence, precision: str = "fp32", coarse_candidates: Iterable[int] = (31,),
             cache: Optional[TuneCache] = None, cycles: int = 20, warm: int = 3, device: int = 0,
             make_sampler: Optional[Callable] = None, timer: Optional[Callable[[object], float]] = None) -> dict:
    """Time every coarse_max_n candidate (its own handle) and, on each, every band
    threshold and then every coarse thread count (same handle); store the fastest
    combination in the cache (if given) and return {"coarse_max_n", "band_min_n",
    "coarse_threads", "ms": {...}}.  make_sampler(problems, c)
    and timer(sampler) replace the GPU parts (tests)."""
    if make_sampler is None:
        from .mgmc import BatchSampler

        def make_sampler(ps, c):
            s = BatchSampler(ps, precision=precision, coarse_max_n=c, device=device)
            s.sample(s.zeros(), 1, 1)
            return s
    if timer is None:
        def timer(s):
            return time_cycles(s, cycles=cycles, warm=warm, device=device)
    best, all_ms = None, {}
    for c in sorted({int(c) for c in coarse_candidates}):
        s = make_sampler(problems, c)
        try:
            b, ms = tune_band_min_n(s, band_candidates(problems, c), timer=timer)
            t, tms = tune_coarse_threads(s, timer=timer)
        finally:
            s.close()
        for k, v in ms.items():
            all_ms[f"{c}/band {k}"] = v
        for k, v in tms.items():
            all_ms[f"{c}/threads {k}"] = v
        if best is None or tms[t] < best[3]:
            best = (c, b, t, tms[t])
    out = {"coarse_max_n": best[0], "band_min_n": best[1], "coarse_threads": best[2], "ms": all_ms}
    if cache is not None:
        cache.put(cache_key(problems, precision),
                  {"coarse_max_n": best[0], "band_min_n": best[1], "coarse_threads": best[2]}, all_ms)
        cache.save()
    return out
