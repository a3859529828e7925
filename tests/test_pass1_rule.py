"""CPU check of the per-height rule the pass-1 kernels use (Sec. 3.3, the extrusion along x).

For one output column, every source column d spacings away contributes closed segments with
label d.  At an endpoint height v the label is P(v) = min{d : a segment of distance d
contains v}; on the open interval between consecutive endpoint heights it is O = min{d : a
segment contains the interval}.  The kernels do not evaluate P(v) per event: they apply all
events of one height (in any order, as XOR toggles of the open set) and take

    P(v) = min(O_below, O_above, g),  g = min{d : a source has an event at v},

emitting a point piece exactly when g < min(O_below, O_above).  This test compares that rule
with the definition on random segment sets (zero-length segments, shared endpoints and
touching segments included), with the events of each height shuffled.
"""
import numpy as np

NO = 10 ** 9


def _by_definition(segs):
    """P(v) at every endpoint height and O on every open interval, from the segments."""
    hs = sorted({h for a, b, _ in segs for h in (a, b)})
    P = {v: min([d for a, b, d in segs if a <= v <= b], default=NO) for v in hs}
    O = []
    for lo, hi in zip(hs, hs[1:]):
        mid = (lo + hi) / 2
        O.append(min([d for a, b, d in segs if a < mid < b], default=NO))
    return hs, P, O


def _by_events(segs, rng):
    """The kernels' walk: events sorted by height (order within a height shuffled), XOR
    toggles of the open set, each height closed when the next one comes."""
    ev = [(a, q) for q, (a, b, d) in enumerate(segs)] + [(b, q) for q, (a, b, d) in enumerate(segs)]
    rng.shuffle(ev)
    ev.sort(key=lambda e: e[0])  # stable: heights sorted, order within a height random
    open_set = set()
    Om = NO
    out = {}  # height -> (label below, label above, point label or None)
    i = 0
    while i < len(ev):
        v = ev[i][0]
        gmin = NO
        while i < len(ev) and ev[i][0] == v:
            q = ev[i][1]
            open_set ^= {q}
            gmin = min(gmin, segs[q][2])
            i += 1
        Ok = min([segs[q][2] for q in open_set], default=NO)
        pt = gmin < min(Om, Ok)
        out[v] = (Om, Ok, gmin if pt else None)
        Om = Ok
    return out


def test_point_rule_matches_definition():
    rng = np.random.default_rng(5)
    for trial in range(400):
        segs = []
        for d in range(int(rng.integers(1, 6))):  # distances 0 .. 4, both sides
            for _ in range(int(rng.integers(0, 3))):
                for _ in range(int(rng.integers(1, 4))):
                    a = int(rng.integers(0, 12))
                    b = a + int(rng.integers(0, 4))  # zero length allowed
                    segs.append((a, b, d))
        if not segs:
            continue
        hs, P, O = _by_definition(segs)
        got = _by_events(segs, rng)
        assert sorted(got) == hs
        for k, v in enumerate(hs):
            below = O[k - 1] if k > 0 else NO
            above = O[k] if k < len(O) else NO
            om, ok, pt = got[v]
            assert (om, ok) == (below, above), (trial, v)
            # the point exists exactly where the height's label is below both neighbours,
            # and carries that label
            assert P[v] <= min(below, above)  # the sources open around v contain it
            want_pt = P[v] < min(below, above)
            assert (pt is not None) == want_pt, (trial, v, segs)
            if want_pt:
                assert pt == P[v], (trial, v)
            else:
                assert P[v] == min(below, above), (trial, v)


def _by_events_lazy(segs, rng):
    """The same walk with the window kernel's lazy close: a height is closed only when one of
    its events came from a source within the label below it (d <= O_below); otherwise the
    labels and the missing point are taken as unchanged without looking."""
    ev = [(a, q) for q, (a, b, d) in enumerate(segs)] + [(b, q) for q, (a, b, d) in enumerate(segs)]
    rng.shuffle(ev)
    ev.sort(key=lambda e: e[0])
    open_set = set()
    Om = NO
    out = {}
    i = 0
    while i < len(ev):
        v = ev[i][0]
        gmin, dirty = NO, False
        while i < len(ev) and ev[i][0] == v:
            q = ev[i][1]
            open_set ^= {q}
            d = segs[q][2]
            if d <= Om:
                dirty = True
                gmin = min(gmin, d)
            i += 1
        if not dirty:
            out[v] = (Om, Om, None)
            continue
        Ok = min([segs[q][2] for q in open_set], default=NO)
        pt = gmin < min(Om, Ok)
        out[v] = (Om, Ok, gmin if pt else None)
        Om = Ok
    return out


def test_lazy_close_changes_nothing():
    """The lazy close gives the same labels and points at every height as closing every
    height (so skipping the closes of heights no lane needs is exact)."""
    rng = np.random.default_rng(9)
    for trial in range(600):
        segs = []
        for d in range(int(rng.integers(1, 8))):
            for _ in range(int(rng.integers(0, 3))):
                for _ in range(int(rng.integers(1, 4))):
                    a = int(rng.integers(0, 14))
                    segs.append((a, a + int(rng.integers(0, 4)), d))
        if not segs:
            continue
        seed = int(rng.integers(1 << 30))
        eager = _by_events(segs, np.random.default_rng(seed))
        lazy = _by_events_lazy(segs, np.random.default_rng(seed))
        assert eager == lazy, (trial, segs)
