"""Checkpoint/resume, run-to-run determinism and the failure path of the
fused tile kernel's bounded wait.

* Resume: a run interrupted by phl_get_state / phl_set_state (U, face B, and T
  for the stellar EOS -- the Newton guess) continues bit for bit as the
  uninterrupted run; the CFL step is recomputed on the device from the state.
* Determinism: two independent runs of the same problem are bit-identical
  (no atomics touch the state; reductions are order-independent maxima).
* Bounded wait: the tile kernel's TMA barrier is made to wait for bytes that
  never arrive (phl_test_tile_wait_timeout); every wait gives up after its
  limit, the host reads PHL_ETIMEOUT, and the same context then steps
  normally -- no GPU fault, trap or hang is involved.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def _same(a, b):
    for k in ("cons", "bx", "by", "bz"):
        assert np.array_equal(a[k], b[k]), k
    if a.get("T") is not None:
        assert np.array_equal(a["T"], b["T"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_is_bitwise(P, precision):
    pr = W.stratified_box(20, 17, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    g = P.Grid(pr, precision=precision)
    g.load()
    g.step(6)
    whole = g.get_state()
    g.close()
    a = P.Grid(pr, precision=precision)
    a.load()
    a.step(3)
    mid = a.get_state()
    a.close()
    b = P.Grid(pr, precision=precision)
    b.set_state(mid["cons"], mid["bx"], mid["by"], mid["bz"])
    b.step(3)
    _same(b.get_state(), whole)
    b.close()


def test_resume_stellar_keeps_newton_guess(P):
    """The mixed stellar state includes T and the inversion record (each
    inversion's first guess): restoring both with the state makes the
    resumed run bit-identical; without the record the inversions start
    plainly and agree to the rounding of the FP32 deviations (a last-bit
    change of P can flip the rounding of its FP32 deviation)."""
    table = P.EosTable()
    pr = W.stellar_box(10, 9, 16)
    def run(g, n):
        g.step(n)
        return g.get_state()
    g = P.Grid(pr, precision="mixed", eos_table=table)
    g.load()
    whole = run(g, 4)
    g.close()
    a = P.Grid(pr, precision="mixed", eos_table=table)
    a.load()
    mid = run(a, 2)
    rec = a.get_eos_record()
    a.close()
    b = P.Grid(pr, precision="mixed", eos_table=table)
    b.set_state(mid["cons"], mid["bx"], mid["by"], mid["bz"], mid["T"])
    b.set_eos_record(rec)
    _same(run(b, 2), whole)
    b.close()
    c = P.Grid(pr, precision="mixed", eos_table=table)
    c.set_state(mid["cons"], mid["bx"], mid["by"], mid["bz"], mid["T"])
    plain = run(c, 2)
    c.close()
    for k in ("cons", "bx", "by", "bz"):
        scale = np.abs(whole[k]).max()
        assert np.abs(plain[k] - whole[k]).max() <= 1e-6 * scale, k
    table.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_runs_are_deterministic(P, precision):
    pr = W.stratified_box(24, 24, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    out = []
    for _ in range(2):
        g = P.Grid(pr, precision=precision)
        g.load()
        g.step(5)
        out.append(g.get_state())
        g.close()
    _same(out[0], out[1])


def test_tile_wait_timeout_is_reported_and_recoverable(P):
    pr = W.stratified_box(8, 8, 8, amp=3e-2, beta=1e3, mach_heat=3e-2)   # one tile
    ref = P.Grid(pr, precision="mixed")
    ref.load()
    ref.step(2, 1e-4)
    want = ref.get_state()
    ref.close()
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.test_tile_wait_timeout(True)
    g.step(1, 1e-4)
    with pytest.raises(P.PhlError) as e:
        g.check()
    assert "PHL_ETIMEOUT" in str(e.value)
    g.test_tile_wait_timeout(False)
    g.load()                      # reload: clears the error bits
    g.step(2, 1e-4)
    _same(g.get_state(), want)
    g.close()
