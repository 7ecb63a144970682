"""The sub-volume method behind the full-size GPU parity test, checked on the
CPU: one oracle RK3 step of a 48^3 stratified box and oracle steps of
sub-boxes of half-width 18 around sampled cells agree on the central 9^3
cells (up to the rounding of the sub-box's cell size)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from subbox import sub_problem

H, C = 18, 4


@pytest.fixture(scope="module")
def full():
    pr = W.stratified_box(48, 48, 48, amp=3e-2, beta=1e3, mach_heat=3e-2)
    o = O.Oracle(pr)
    dt = o.dt()
    st, _, _ = o.run(1, dt_fixed=dt)
    return pr, dt, st


@pytest.mark.parametrize("c", [(24, 24, 24), (3, 45, 20), (10, 5, 2), (40, 31, 45), (47, 0, 10)])
def test_subbox_step_equals_full_step_in_the_centre(full, c):
    pr, dt, st = full
    q, (ix, iy, iz) = sub_problem(pr, c, H)
    out, _, _ = O.Oracle(q).run(1, dt_fixed=dt)
    cz = c[2] - iz[0]
    sx = sy = slice(H - C, H + C + 1)
    sz = slice(max(0, cz - C), min(iz.size, cz + C + 1))
    gx, gy, gz = ix[sx], iy[sy], iz[sz]
    for v in range(5):
        a, b = st["cons"][v][np.ix_(gz, gy, gx)], out["cons"][v][sz, sy, sx]
        scale = max(np.abs(pr.cons[v]).max(), np.abs(st["cons"][v]).max())
        assert np.abs(a - b).max() <= 1e-15 * scale, v
    for k in ("bx", "by", "bz"):
        a, b = st[k][np.ix_(gz, gy, gx)], out[k][sz, sy, sx]
        assert np.abs(a - b).max() <= 1e-15 * np.abs(pr.bx).max(), k
