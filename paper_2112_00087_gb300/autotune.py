"""Launch-shape autotuner for the persistent batched solver.

The persistent engine reads five launch-shape knobs from the environment at every solve:
``HELM_PERSIST_BLOCKS_PER_SM`` (resident blocks per SM, i.e. the register budget),
``HELM_TILE_ROWS`` (minimum rows per tile, i.e. how many per-tile reductions a phase pays),
``HELM_TILES_PER_BLOCK`` (about how many tiles per resident block a system with more than 4,096
rows per block is cut into, never below 4,096 rows, i.e. how finely the dynamic scheduler can
balance its tiles),
``HELM_PREFETCH`` (how many block rows ahead each thread of the double-word SpMV prefetches its
matrix parts into L2) and ``HELM_PF_CHUNKS`` (how many 256-row chunks ahead one thread per
block bulk-prefetches the vectors of the double-word update phases into L2). ``autotune``
searches them coordinate by coordinate for a caller-supplied workload: the caller passes a
function that runs one solve under the current environment and returns its time in seconds
(for example CUDA-event time of ``helm_solve_batch``), and gets back the fastest setting found,
which ``apply`` installs for later solves of the process.

The search is plain coordinate descent from the library defaults: each knob in turn is set to
each of its candidate values with the others held, the best value is kept (a new value only when
it is more than 0.5 % faster), and passes repeat
until a pass changes nothing (or ``max_passes``). Every candidate is timed ``reps`` times and
scored by its minimum.
"""
from __future__ import annotations

import os
from typing import Callable, Dict, List, Optional, Sequence, Tuple

DEFAULTS: Dict[str, int] = {"HELM_PERSIST_BLOCKS_PER_SM": 2, "HELM_TILE_ROWS": 4096, "HELM_TILES_PER_BLOCK": 2,
                            "HELM_PREFETCH": 1, "HELM_PF_CHUNKS": 2}
SPACE: Dict[str, Sequence[int]] = {
    "HELM_PERSIST_BLOCKS_PER_SM": (1, 2, 3),
    "HELM_TILE_ROWS": (512, 2048, 4096, 8192),
    "HELM_TILES_PER_BLOCK": (1, 2, 4),
    "HELM_PREFETCH": (0, 1, 2),
    "HELM_PF_CHUNKS": (0, 1, 2, 4),
}


# Knobs of the standalone kernels (read at every call): lanes per row of the CSR product for
# complex128 and complex64, and the partial sums per SM of helm_reduce.
KERNEL_DEFAULTS: Dict[str, int] = {"HELM_SPMV_LANES_C128": 4, "HELM_SPMV_LANES_C64": 8, "HELM_REDUCE_PARTS_PER_SM": 1}
KERNEL_SPACE: Dict[str, Sequence[int]] = {
    "HELM_SPMV_LANES_C128": (2, 4, 8, 16),
    "HELM_SPMV_LANES_C64": (2, 4, 8, 16),
    "HELM_REDUCE_PARTS_PER_SM": (1, 2, 4, 8, 16),
}


def apply(config: Dict[str, int]) -> None:
    """Install a setting for the solves that follow in this process."""
    for k, v in config.items():
        os.environ[k] = str(int(v))


def _timed(run: Callable[[], float], config: Dict[str, int], reps: int) -> float:
    saved = {k: os.environ.get(k) for k in config}
    try:
        apply(config)
        return min(float(run()) for _ in range(reps))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def autotune(run: Callable[[], float], space: Optional[Dict[str, Sequence[int]]] = None,
             start: Optional[Dict[str, int]] = None, reps: int = 1, max_passes: int = 3,
             min_gain: float = 0.005) -> Tuple[Dict[str, int], List[Tuple[Dict[str, int], float]]]:
    """Coordinate-descent search over `space` (default SPACE) from `start` (default DEFAULTS).

    run() executes one solve under the current environment and returns its time in seconds.
    A candidate replaces the current best only when it is faster by more than the fraction
    `min_gain` (timing noise, or a knob that does not change the workload, moves nothing).
    Returns (best setting, [(setting, time) for every setting timed, in order]). The process
    environment is left as it was; call apply(best) to use the result."""
    space = dict(SPACE if space is None else space)
    best = dict(DEFAULTS if start is None else start)
    for k in space:
        best.setdefault(k, space[k][0])
    seen: Dict[Tuple[Tuple[str, int], ...], float] = {}
    log: List[Tuple[Dict[str, int], float]] = []

    def score(cfg: Dict[str, int]) -> float:
        key = tuple(sorted(cfg.items()))
        if key not in seen:
            seen[key] = _timed(run, cfg, reps)
            log.append((dict(cfg), seen[key]))
        return seen[key]

    best_t = score(best)
    for _ in range(max_passes):
        changed = False
        for knob, values in space.items():
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best)
                cand[knob] = v
                t = score(cand)
                if t < best_t * (1.0 - min_gain):
                    best, best_t, changed = cand, t, True
        if not changed:
            break
    return best, log
