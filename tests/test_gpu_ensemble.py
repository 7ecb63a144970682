"""Ensemble of uneven boxes: the persistent, graph-captured path against
stepping each box alone (same device bodies, the same per-box CFL step).

The bodies are inlined into a different kernel, so the compiler's choice of
fused multiply-adds may differ: the two agree to the FP32 rounding of the
deviations (the mixed form's own error, bar 1e-5 of each field's change),
not bit for bit.  Runs of the ensemble itself are reproducible bit for bit
with any launch shape, and the autotuner leaves the state untouched."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def _boxes():
    dims = [(16, 24, 32), (24, 16, 20), (32, 32, 16), (20, 20, 24)]
    return [W.stratified_box(nx, ny, nz, seed=100 + i, amp=3e-2, beta=1e3, mach_heat=3e-2)
            for i, (nx, ny, nz) in enumerate(dims)]


def _alone(P, pr, nsteps):
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(nsteps)
    st = g.get_state()
    g.close()
    return st


def _same(a, b):
    for k in ("cons", "bx", "by", "bz"):
        assert np.array_equal(a[k], b[k]), k


def _close(pr, a, b):
    """L1 of (a - b) against the change over the run: per field for rho and E,
    per vector for momentum and B (their transverse parts start at zero)."""
    for v in (0, 4):
        change = np.abs(b["cons"][v] - pr.cons[v]).sum()
        assert np.abs(a["cons"][v] - b["cons"][v]).sum() <= 1e-5 * change, v
    change = np.abs(b["cons"][1:4] - pr.cons[1:4]).sum()
    assert np.abs(a["cons"][1:4] - b["cons"][1:4]).sum() <= 1e-5 * change, "momentum"
    change = sum(np.abs(b[k] - getattr(pr, k)).sum() for k in ("bx", "by", "bz"))
    assert sum(np.abs(a[k] - b[k]).sum() for k in ("bx", "by", "bz")) <= 1e-5 * change, "B"


@pytest.mark.parametrize("graph", [True, False])
def test_ensemble_equals_boxes_alone(P, graph):
    probs = _boxes()
    ref = [_alone(P, pr, 4) for pr in probs]
    E = P.Ensemble(probs, use_graph=graph)
    E.load()
    E.step(4)
    E.check()
    info = E.info()
    assert info["nbox"] == len(probs) and info["launches_per_step"] == 3
    assert info["graph"] == (1 if graph else 0)
    for g, r, pr in zip(E.grids, ref, probs):
        _close(pr, g.get_state(), r)
    E.close()


def test_launch_shapes_and_autotune(P):
    probs = _boxes()
    E = P.Ensemble(probs)
    E.load()
    E.step(3)
    ref = [g.get_state() for g in E.grids]
    E.load()
    res = E.autotune(trial_steps=1)
    assert len(res) >= 2 and all(r["ms_per_step"] > 0 for r in res)
    info = E.info()
    best = min(res, key=lambda r: r["ms_per_step"])
    assert (info["block"], info["blocks_per_sm"]) == (best["block"], best["blocks_per_sm"])
    E.step(3)
    for g, r in zip(E.grids, ref):     # the autotuner restored the initial state
        _same(g.get_state(), r)
    # any other co-resident shape gives the same bits
    E.load()
    E.set_shape(128, 1)
    E.step(3)
    for g, r in zip(E.grids, ref):
        _same(g.get_state(), r)
    E.close()


def test_ensemble_rejects_unsupported_boxes(P):
    """Only mixed-form, ideal-gas boxes without species join an ensemble."""
    import ctypes as C
    pr = W.stratified_box(16, 16, 16)
    d, keep = P.make_desc(pr, precision="fp64")
    descs = (P.GridDesc * 1)(d)
    h = C.c_void_p()
    with pytest.raises(P.PhlError):
        P._check(P.lib().phl_ensemble_create(descs, 1, 1, C.byref(h)))
