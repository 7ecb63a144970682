"""Parity at the benchmark's full size: the stratified box at 256^3, one SSP-RK3
step of the FP64 form in the configuration bench.py times, checked cell by
cell on sampled sub-volumes against the oracle.

The oracle cannot afford the whole box, but one RK3 step only couples a cell
to neighbours within a bounded radius (per stage: PLM two cells, Contact-CT
one more, the shock flags' raw +-1 and 5-wide dilation): 12 cells per step.
So the oracle steps a sub-box of half-width 18 around each sample with the
GPU's dt, outflow sides where the sub-box cuts the domain (reflecting walls
kept where it reaches them), and the central 9^3 cells, 14 cells from any cut,
must agree with the GPU to 1e-11 of each field's scale.  (The sub-volume
method itself is checked on the CPU in test_subbox_locality.py.)
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from subbox import sub_problem

pytestmark = pytest.mark.gpu

N = 256
H = 18          # half-width of the oracle's sub-box
C = 4           # compared cells: |offset| <= C


@pytest.fixture(scope="module")
def full_step():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    pr = W.stratified_box(N, N, N)
    g = P.Grid(pr, precision="fp64")
    g.load()
    dt = g.compute_dt()
    g.step(1, dt)
    st = g.get_state()
    g.close()
    return pr, dt, st


@pytest.mark.parametrize("c", [(128, 128, 128), (3, 250, 100), (77, 5, 2), (200, 131, 253), (255, 0, 20)])
def test_full_size_step_on_sampled_subvolumes(full_step, c):
    pr, dt, st = full_step
    q, (ix, iy, iz) = sub_problem(pr, c, H)
    out, _, _ = O.Oracle(q).run(1, dt_fixed=dt)
    # centre cells in sub-box coordinates
    cx = cy = H
    cz = c[2] - iz[0]
    sx, sy = slice(cx - C, cx + C + 1), slice(cy - C, cy + C + 1)
    sz = slice(max(0, cz - C), min(iz.size, cz + C + 1))
    # the compared cells are at least 14 cells from every cut of the sub-box
    zmargin_lo = cz - C if iz[0] > 0 else 99
    zmargin_hi = (iz.size - 1) - (cz + C) if iz[-1] < pr.n[2] - 1 else 99
    assert min(H - C, zmargin_lo, zmargin_hi) >= 14
    gx, gy, gz = ix[sx], iy[sy], iz[sz]
    # rho and E per field; the momentum against rho c_s (the box starts at rest
    # in pressure equilibrium: after one step its horizontal momentum is the
    # rounding residue of the pressure balance, ~1e-9 rho c_s, on both sides)
    rho_cs = np.abs(pr.cons[0]).max() * np.sqrt(pr.gamma * (pr.gamma - 1.0) * np.abs(pr.cons[4]).max()
                                                  / np.abs(pr.cons[0]).min())
    for v in range(5):
        a = st["cons"][v][np.ix_(gz, gy, gx)]
        b = out["cons"][v][sz, sy, sx]
        scale = rho_cs if v in (1, 2, 3) else max(np.abs(pr.cons[v]).max(), np.abs(st["cons"][v]).max())
        assert np.abs(a - b).max() <= 1e-11 * scale, (v, np.abs(a - b).max() / scale)
    # face fields of the compared cells (their lower faces)
    for k in ("bx", "by", "bz"):
        a = st[k][np.ix_(gz, gy, gx)]
        b = out[k][sz, sy, sx]
        scale = np.abs(st["bx"]).max()
        assert np.abs(a - b).max() <= 1e-11 * scale, (k, np.abs(a - b).max() / scale)


@pytest.fixture(scope="module")
def full_step_mixed():
    """The mixed form as bench.py times it (fused tile kernel, default launch
    shape), one SSP-RK3 step at the FP64 form's dt."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    pr = W.stratified_box(N, N, N)
    g = P.Grid(pr, precision="fp64")
    g.load()
    dt = g.compute_dt()
    g.close()
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(1, dt)
    st = g.get_state()
    g.close()
    return pr, dt, st


@pytest.mark.parametrize("c", [(128, 128, 128), (3, 250, 100), (77, 5, 2), (200, 131, 253)])
def test_full_size_mixed_step_on_sampled_subvolumes(full_step_mixed, c):
    """The mixed form against the oracle on the compared cells: relative L1 of
    the deviation from the background <= 1e-5 (the mixed form's bar) for rho,
    E and B_x; the momentum, born from the buoyancy of the density noise in
    this first step, as one vector field (zero background) at the same bar."""
    pr, dt, st = full_step_mixed
    q, (ix, iy, iz) = sub_problem(pr, c, H)
    out, _, _ = O.Oracle(q).run(1, dt_fixed=dt)
    cx = cy = H
    cz = c[2] - iz[0]
    sx, sy = slice(cx - C, cx + C + 1), slice(cy - C, cy + C + 1)
    sz = slice(max(0, cz - C), min(iz.size, cz + C + 1))
    gx, gy, gz = ix[sx], iy[sy], iz[sz]
    kz = gz[:, None, None] + 3
    hats = {0: pr.bg["rho_c"][kz], 4: pr.bg["p_c"][kz] / (pr.gamma - 1.0)}
    for v in (0, 4):
        a = st["cons"][v][np.ix_(gz, gy, gx)] - hats[v]
        b = out["cons"][v][sz, sy, sx] - hats[v]
        rel = np.abs(a - b).sum() / np.abs(b).sum()
        assert rel <= 1e-5, (v, rel)
    a = np.stack([st["cons"][v][np.ix_(gz, gy, gx)] for v in (1, 2, 3)])
    b = np.stack([out["cons"][v][sz, sy, sx] for v in (1, 2, 3)])
    rel = np.abs(a - b).sum() / np.abs(b).sum()
    print("full-size mixed step, momentum L1:", f"{rel:.2e}")
    assert rel <= 1e-5, ("momentum", rel)
    a = st["bx"][np.ix_(gz, gy, gx)]
    b = out["bx"][sz, sy, sx]
    assert np.abs(a - b).sum() / np.abs(b).sum() <= 1e-5
