"""Ensemble of uneven boxes: the persistent, graph-captured path against
stepping each box alone (same device bodies, the same per-box CFL step).

The bodies are inlined into a different kernel, so the compiler's choice of
fused multiply-adds may differ: the two agree to the FP32 rounding of the
deviations (the mixed form's own error, bar 1e-5 of each field's change),
not bit for bit.  Runs of the ensemble itself are reproducible bit for bit
with any launch shape (the phase bodies are the same code in both launch
modes), and the autotuner leaves the state untouched."""
import numpy as np
import pytest

import oracle as O
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


def _deviation_l1(pr, a, b):
    """The mixed form's measure: relative L1 of the deviations from the
    background (rho - rho_hat, E - E_hat; momentum and B as vector fields with
    zero background)."""
    nz = pr.n[2]
    rho_hat = pr.bg["rho_c"][3:3 + nz][:, None, None]
    e_hat = pr.bg["p_c"][3:3 + nz][:, None, None] / (pr.gamma - 1.0)
    rel = lambda x, y: np.abs(x - y).sum() / np.abs(y).sum()
    return {"rho": rel(a["cons"][0] - rho_hat, b["cons"][0] - rho_hat),
            "m": rel(a["cons"][1:4], b["cons"][1:4]),
            "E": rel(a["cons"][4] - e_hat, b["cons"][4] - e_hat),
            "B": (sum(np.abs(a[k] - b[k]).sum() for k in ("bx", "by", "bz")) /
                  sum(np.abs(b[k]).sum() for k in ("bx", "by", "bz")))}


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_ensemble_boxes_match_the_oracle(P, mode):
    """Every box of a four-box ensemble, in each launch mode, against the CPU
    oracle stepping the same box alone (each side with its own CFL step: the
    mixed form's FP32 step differs by ~1e-7 relative), at the mixed form's
    bar of 1e-5 per field."""
    probs = _boxes()
    E = P.Ensemble(probs)
    E.load()
    E.set_shape(288 if mode == 3 else 256, 1 if mode == 0 else 0, mode=mode, streams=4 if mode == 2 else 0)
    if mode == 3:
        assert E.info()["launches_per_step"] == 3
    nsteps = 4
    E.step(nsteps)
    E.check()
    for g, pr in zip(E.grids, probs):
        ref, _, _ = O.Oracle(pr).run(nsteps)
        l1 = _deviation_l1(pr, g.get_state(), ref)
        print(pr.n, {k: f"{v:.2e}" for k, v in l1.items()})
        for k, v in l1.items():
            assert v <= 1e-5, (pr.n, k, v)
    E.close()


def test_launch_shapes_and_autotune(P):
    probs = _boxes()
    E = P.Ensemble(probs)

    def run(mode, blk, bps, streams=0):
        E.load()
        E.set_shape(blk, bps, mode=mode, streams=streams)
        E.step(3)
        return [g.get_state() for g in E.grids]

    # the same kernels give the same bits with any launch shape
    ref = {0: run(0, 256, 1), 1: run(1, 256, 0), 2: run(2, 256, 0, 4), 3: run(3, 288, 0)}
    for mode, blk, bps, ns in ((0, 128, 1, 0), (0, 128, 2, 0), (1, 128, 0, 0), (2, 256, 0, 1), (2, 256, 0, 3),
                               (3, 288, 0, 0)):
        for a, r in zip(run(mode, blk, bps, ns), ref[mode]):
            _same(a, r)
    # mode 2 runs each box's own per-kernel step: bit for bit the box alone
    for a, pr in zip(ref[2], probs):
        _same(a, _alone(P, pr, 3))
    # the launch modes inline the same bodies into different kernels
    for m in (1, 2):
        for a, r, pr in zip(ref[0], ref[m], probs):
            _close(pr, a, r)
    # the persistent fused kernel runs the fused tile body of the per-box chains
    for a, r, pr in zip(ref[3], ref[2], probs):
        _close(pr, a, r)
    E.load()
    res = E.autotune(trial_steps=1)
    assert len(res) >= 3 and all(r["ms_per_step"] > 0 for r in res)
    assert {r["mode"] for r in res} == {0, 1, 2, 3}
    info = E.info()
    best = min(res, key=lambda r: r["ms_per_step"])
    assert (info["mode"], info["block"], info["blocks_per_sm"], info["streams"]) == (
        best["mode"], best["block"], best["blocks_per_sm"], best["streams"])
    E.step(3)   # from the loaded state, which the autotuner restored
    after = [g.get_state() for g in E.grids]
    for a, r in zip(after, run(info["mode"], info["block"], info["blocks_per_sm"], info["streams"])):
        _same(a, r)
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
