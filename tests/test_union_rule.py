"""CPU check of the union by jumps used by the pass-2 gathers (the union of closed intervals,
Sec. 3.3).

The kernels unite a column's intervals without sorting them: a run starts at the least left
end not yet covered, its right end is raised to the largest right end among the intervals
that start at or below it until it no longer rises (touching intervals join), and the next
run starts at the least left end beyond it.  This test compares that procedure with the
sort-and-sweep union on random interval sets (nested, touching, zero-length, repeated).
"""
import numpy as np


def _sorted_union(iv):
    out = []
    for a, b in sorted(iv):
        if out and a <= out[-1][1]:
            out[-1][1] = max(out[-1][1], b)
        else:
            out.append([a, b])
    return [tuple(x) for x in out]


def _jump_union(iv):
    runs = []
    if not iv:
        return runs
    lo = min(a for a, _ in iv)
    hi = lo
    while True:
        mx = max(b for a, b in iv if a <= hi)
        if mx > hi:
            hi = mx
            continue
        runs.append((lo, hi))
        later = [a for a, _ in iv if a > hi]
        if not later:
            return runs
        lo = hi = min(later)


def test_jump_union_matches_sorted_union():
    rng = np.random.default_rng(9)
    for trial in range(2000):
        n = int(rng.integers(0, 40))
        iv = []
        for _ in range(n):
            a = int(rng.integers(0, 60))
            iv.append((a, a + int(rng.integers(0, 6))))
        assert _jump_union(iv) == _sorted_union(iv), (trial, iv)
