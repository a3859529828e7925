"""GPU parity at the sizes the benchmark times: the 2048 x 2048 grid of 1000 primitives
(nested hollow spheres, thin plates, spheres, boxes, shells; up to 58 segments a column),
offset by k = 64 spacings, in the launch configuration the benchmark uses (one call through
the C ABI, library-owned scratch).  The oracle computes sampled output columns one by one:
2000 random ones, one full row and one full column, compared element by element with the
tolerances of the small-grid tests (FP64 1e-10, FP32 endpoints 4e-6, counts identical except
where the oracle's gap is below the mode's threshold).  These sizes take the paths the small
grids do not reach: the 16384-event pass-1 tiles of the densest windows and the gather
buckets learnt for a 129-column window.
"""
import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 4e-6
GAP64 = 1e-9
K = 64.0


@pytest.fixture(scope="module")
def grids():
    g64 = shapes.config3()
    return {"fp64": g64, "fp32": shapes.to_float32(g64)}


def _cols(n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.choice(n * n, 2000, replace=False),
                                     np.arange(n) + 777 * n, np.arange(n) * n + 1301]))


def _check(off, z, ref, cols, f32, what):
    tol = TOL32 if f32 else TOL64
    for t, c in enumerate(cols):
        got = np.asarray(z[off[c]:off[c + 1]], np.float64)
        exp = ref.column(t)
        if got.shape != exp.shape:
            gaps = exp[1:, 0] - exp[:-1, 1]
            if f32:
                scale = np.maximum(np.maximum(np.abs(exp[1:, 0]), np.abs(exp[:-1, 1])), 1.0)
                ok = gaps.size > 0 and np.min(gaps / scale) < 2.0 ** -23
            else:
                ok = gaps.size > 0 and np.min(gaps) < GAP64
            assert ok, f"{what}: count mismatch at column {c}: {got.shape} vs {exp.shape}"
            continue
        if exp.size:
            err = float(np.max(np.abs(got - exp)))
            assert err <= tol, f"{what}: column {c} endpoint error {err}"


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_2048_k64_sampled(grids, mode, op):
    import torch
    import paper_1804_08968_gb300 as dx
    g = grids[mode]
    f32 = mode == "fp32"
    dg = dx.Grid.from_synth(g, dtype=torch.float32 if f32 else torch.float64)
    ctx = dx.Context(0)
    out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, K)
    torch.cuda.synchronize()
    st = ctx.stats()
    off, z = out.to_host()
    del out, dg
    torch.cuda.empty_cache()
    cols = _cols(g.nx, 5 if op == "dilate" else 6)
    if op == "erode":
        cols = cols[::3]  # the erosion oracle is the slower one
    ref = (oracle.dilate if op == "dilate" else oracle.erode)(g, K, cols=cols)
    _check(off, z, ref, cols, f32, f"2048^2 k=64 {op} {mode}")
    assert st[0] == g.nseg and st[3] == off[-1]
