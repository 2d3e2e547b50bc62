"""Autotuner of the search kernel's launch-time knob.

The search kernel walks the octree with unions of source neurons that are adjacent
in Morton order (``search_group`` in relearn_params). By default each warp's 32
sources are cut into pieces wherever two neighbours do not share a cell of some
cut depth, and each piece walks one union; the cut depth follows the share of
neurons that search. A fixed width (32, 8, or every lane alone) or another cut depth
can be forced. The best choice depends on the workload (cluster sizes, density,
sigma relative to the domain). Results never depend on the choice, only the time
does, so the tuner simply times each candidate on the caller's own update and keeps
the fastest.

The tuner runs trials through a caller-supplied function that performs one
update with the given ``search_group`` and returns the search kernel's device
milliseconds (e.g. from ``relearn_collect_search_times`` after an update with
``FLAG_TIMING``); the caller restores its state between trials.
"""
from __future__ import annotations

from typing import Callable, Dict, Iterable, Tuple

# 0 = the library's default; 1 / 8 / 32 = one fixed width for every warp;
# 1000 + 100 * d = per-warp unions cut at the boundaries of depth-d cells.
DEFAULT_CANDIDATES = (0, 1, 8, 32, 1200, 1300, 1500, 1600)


def tune(trial: Callable[[int], float], candidates: Iterable[int] = DEFAULT_CANDIDATES,
         repeats: int = 2) -> Tuple[int, Dict[int, float]]:
    """Time every candidate ``repeats`` times (the minimum counts) and return
    (best candidate, {candidate: ms})."""
    table: Dict[int, float] = {}
    for c in candidates:
        table[int(c)] = min(float(trial(int(c))) for _ in range(max(repeats, 1)))
    best = min(table, key=table.get)
    return best, table
