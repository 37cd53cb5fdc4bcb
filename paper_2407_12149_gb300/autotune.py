"""Run-time choice of a batch's coarse-grid threshold (mgmc_config.coarse_max_n).

Grids with n <= threshold run inside the shared-memory coarse kernel (one CTA per
chain, barrier-latency bound); the larger ones in the persistent tile launches (one
forward and one backward launch plus two low-rank launches per grid depth).  Which
split is faster depends on the chain count and the grid sizes, so each candidate's
captured V-cycle is timed with CUDA events over back-to-back cycles (states resident
on the device) and the fastest is kept.  The arithmetic of a cycle does not depend
on the threshold beyond the rounding of the FP32 coarse grids' sweeps.
"""
from __future__ import annotations

from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple


def pick_fastest(timings: Dict[int, float]) -> int:
    """The candidate with the smallest time; on equal times the smaller threshold
    (fewer grids held in shared memory)."""
    if not timings:
        raise ValueError("no candidate was timed")
    return min(timings, key=lambda c: (timings[c], c))


def time_batch_cycle(problems: Sequence, coarse_max_n: int, precision: str = "fp32", cycles: int = 20,
                     warm: int = 3, device: int = 0, seed: int = 1) -> float:
    """Milliseconds per V-cycle of the batch with this threshold (CUDA events on the
    current stream around `cycles` back-to-back cycles after `warm` untimed ones)."""
    import torch
    from .mgmc import BatchSampler
    s = BatchSampler(problems, precision=precision, coarse_max_n=coarse_max_n, device=device)
    try:
        xs = s.zeros()
        s.sample(xs, warm, seed)
        stream = torch.cuda.current_stream(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.sample(None, cycles, seed, step_offset=warm)
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / cycles
    finally:
        s.close()


def autotune_coarse_max_n(problems: Sequence, precision: str = "fp32", candidates: Iterable[int] = (15, 31, 63),
                          cycles: int = 20, warm: int = 3, device: int = 0,
                          timer: Optional[Callable[[Sequence, int], float]] = None) -> Tuple[int, Dict[int, float]]:
    """(best threshold, {threshold: ms per cycle}) over the candidates (positive, each
    timed once).  `timer(problems, threshold)` replaces the GPU timing (tests)."""
    cands = sorted({int(c) for c in candidates})
    if not cands or cands[0] < 1:
        raise ValueError("candidates must be positive grid sizes")
    if timer is None:
        def timer(ps, c):
            return time_batch_cycle(ps, c, precision=precision, cycles=cycles, warm=warm, device=device)
    timings = {c: float(timer(problems, c)) for c in cands}
    return pick_fastest(timings), timings
