"""The pass-1 window kernel's two ways of putting a tile's events in height order, modelled
on the CPU with the kernel's own index arithmetic (pass1l.cuh):

* p1l_merge_level: the sources' sorted runs merged pairwise, level by level; every thread
  takes a fixed range of output positions, finds the pair holding its first output by a
  binary search over the run bounds and its split of the pair by a binary search along the
  merge path, then merges.  Checked: every output position written once, every read inside
  its pair, the result sorted and a permutation of the input, for any run lengths (empty
  runs included), thread counts and counts of runs.
* the bitonic network with every comparator pointing the same way (each merge stage starts
  by comparing an element with its mirror in the block), positions past the E events being a
  virtual +inf that no comparator moves: sorted for every E, not only powers of two, without
  touching a position >= E.
"""
import random

import pytest


def merge_level(ks, ps, kd, pd, bo, e0, nr, w, o0, o1, written):
    def bnd(r):
        return bo[min(r, nr)] - e0
    np_ = (nr + 2 * w - 1) // (2 * w)
    lo, hi = 0, np_ - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if bnd(2 * w * mid) <= o0:
            lo = mid
        else:
            hi = mid - 1
    o, p = o0, lo
    while o < o1 and p < np_:
        a0, a1, a2 = bnd(2 * w * p), bnd(2 * w * p + w), bnd(2 * w * p + 2 * w)
        if o >= a2:
            p += 1
            continue
        nL, nR, k = a1 - a0, a2 - a1, o - a0
        i0, i1 = max(0, k - nR), min(k, nL)
        while i0 < i1:
            mid = (i0 + i1) >> 1
            assert 0 <= mid < nL and 0 <= k - 1 - mid < nR
            if ks[a0 + mid] <= ks[a1 + k - 1 - mid]:
                i0 = mid + 1
            else:
                i1 = mid
        i, j = i0, k - i0
        oe = min(o1, a2)
        while o < oe:
            left = j >= nR or (i < nL and ks[a0 + i] <= ks[a1 + j])
            src = a0 + i if left else a1 + j
            assert a0 <= src < a2
            assert not written[o]
            written[o] = True
            kd[o], pd[o] = ks[src], ps[src]
            i, j = (i + 1, j) if left else (i, j + 1)
            o += 1
        p += 1


def merge_sort(lens, threads, rng):
    e0 = rng.randint(0, 40)
    bo = [e0]
    for n in lens:
        bo.append(bo[-1] + n)
    nr, E = len(lens), bo[-1] - e0
    ks, ps = [], []
    for r, n in enumerate(lens):
        ks += sorted(rng.choice([rng.randint(0, 9), rng.randint(0, 10 ** 6)]) for _ in range(n))
        ps += [r] * n
    a = (ks[:], ps[:])
    w = 1
    while w < nr:
        b = ([None] * E, [None] * E)
        written = [False] * E
        per = (E + threads - 1) // threads
        for t in range(threads):
            o0 = min(E, t * per)
            merge_level(a[0], a[1], b[0], b[1], bo, e0, nr, w, o0, min(E, o0 + per), written)
        assert all(written)
        a, w = b, 2 * w
    return ks, ps, a


@pytest.mark.parametrize("seed", range(6))
def test_merge_path_levels(seed):
    rng = random.Random(seed)
    for _ in range(150):
        nr = rng.choice([1, 2, 3, rng.randint(1, 40), rng.randint(100, 300)])
        lens = [rng.choice([0, 0, 1, 2, 7, rng.randint(0, 60)]) for _ in range(nr)]
        threads = rng.choice([1, 7, 32, 64, 256])
        ks, ps, (ok, op) = merge_sort(lens, threads, rng)
        assert ok == sorted(ks)
        assert sorted(zip(ok, op)) == sorted(zip(ks, ps))


def bitonic_virtual(a, threads):
    E = len(a)
    n2 = 1
    while n2 < E:
        n2 <<= 1
    a = a[:]
    k = 2
    while k <= n2:
        jj = k >> 1
        while jj > 0:
            for tid in range(threads):
                for p in range(tid, n2 >> 1, threads):
                    if jj == (k >> 1):  # the flip: t against its mirror in the block of k
                        i = p & (jj - 1)
                        t = (p >> (jj.bit_length() - 1)) * k + i
                        x = t - i + (k - 1 - i)
                    else:
                        t = ((p & ~(jj - 1)) << 1) | (p & (jj - 1))
                        x = t | jj
                    assert t < x
                    if x < E:
                        if a[t] > a[x]:
                            a[t], a[x] = a[x], a[t]
            jj >>= 1
        k <<= 1
    return a


@pytest.mark.parametrize("seed", range(4))
def test_bitonic_with_virtual_padding(seed):
    rng = random.Random(100 + seed)
    for E in list(range(0, 40)) + [rng.randint(40, 700) for _ in range(20)]:
        a = [rng.randint(0, 30) for _ in range(E)]
        assert bitonic_virtual(a, rng.choice([1, 3, 32])) == sorted(a), E
