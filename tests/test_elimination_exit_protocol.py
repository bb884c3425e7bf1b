"""Invariant of the register-tiled element elimination's early warp exit (CPU).

Tile pairs (ti, k) -- tiles (ti, 2k) and (ti, 2k + 1), the second present when
2k + 1 <= ti -- are numbered column pair by column pair (k ascending, then ti
from 2k to R - 1).  A thread's exit step is 4k + 2 (one tile) or 4k + 4 (two
tiles), capped at the number of pair steps; a warp leaves the pivot loop at the
maximum over its threads, and the loop barrier of step q counts the warps whose
exit step is >= q.  These tests restate the loop body's work conditions
(publish the pivot columns, record the pivot, update a live tile) and check,
for every block size the register-tiled path accepts (<= 124 rows) and every
pair count, that no thread has work at or after its warp's exit step, that
the numbering is a bijection, and that the pivot recorder of every step
belongs to a warp still in the loop."""
import math

import pytest


def tile_pair(t, R):
    k = int(((R + 1) - math.sqrt((R + 1) ** 2 - 4 * t)) / 2)
    while k > 0 and k * (R + 1 - k) > t:
        k -= 1
    while (k + 1) * (R - k) <= t:
        k += 1
    return 2 * k + (t - k * (R + 1 - k)), k


def exit_step(ti, k, npairs):
    return min(npairs, 4 * k + 4 if 2 * k + 1 <= ti else 4 * k + 2)


def has_work(ti, k, q, ext):
    c0, c1 = 2 * q, 2 * q + 1
    tq = c0 >> 2
    for h in range(2 if 2 * k + 1 <= ti else 1):
        tj = 2 * k + h
        if tj == tq and any(c0 <= 4 * ti + u < ext for u in range(4)):
            return True                      # publishes rows of the pivot columns
        if ti == tq and tj == tq:
            return True                      # owns the diagonal tile: records the pivot
        if 4 * ti + 3 > c1 and 4 * tj + 3 > c1:
            return True                      # a live row and a live column: update
    return False


@pytest.mark.parametrize("ext", list(range(2, 125, 7)) + [100, 120, 124])
def test_no_work_after_exit(ext):
    R = (ext + 3) // 4
    npr = (R + 1) * (R + 1) // 4
    nt = max(64, (npr + 31) // 32 * 32)
    pairs = [tile_pair(t, R) for t in range(npr)]
    assert len(set(pairs)) == npr and all(2 * k <= ti < R for ti, k in pairs)
    for npairs in range(0, ext // 2 + 1):
        exits = [exit_step(ti, k, npairs) for ti, k in pairs] + [0] * (nt - npr)
        wexit = [max(exits[32 * w:32 * w + 32]) for w in range(nt // 32)]
        for t, (ti, k) in enumerate(pairs):
            for q in range(wexit[t // 32], npairs):
                assert not has_work(ti, k, q, ext), (ext, npairs, t, q)
        for q in range(npairs):
            tq = (2 * q) >> 2
            owners = [t for t, (ti, k) in enumerate(pairs)
                      if ti == tq and (2 * k == tq or (2 * k + 1 <= ti and 2 * k + 1 == tq))]
            assert len(owners) == 1 and wexit[owners[0] // 32] > q
            # barrier of step q: warps with exit > q wait, exit == q arrive
            assert 32 * sum(e >= q for e in wexit) >= 32
