"""The allocation-free CFL step (phl_cfl_dt_noalloc) against phl_compute_dt.

phl_cfl_dt_noalloc serves callers that cannot let a library allocate device
memory (their own pool owns it, or their loop must not pay the synchronisation
of cudaMalloc/cudaFree).  Its scratch is a library-owned __device__ array that
every call reuses, so the test calls it twice in a row on different states and
checks each result against the allocating entry point.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative; both compute the same CFL sum, rounding may differ


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def _dev(pr):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(getattr(pr, k))).cuda() for k in ("cons", "bx", "by", "bz")]


def test_noalloc_dt_matches_compute_dt_on_two_calls(P):
    import torch
    a = W.stratified_box(48, 40, 56, amp=2e-2)
    b = W.orszag_tang(96)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for pr in (a, b):
        g = P.Grid(pr)
        g.load()
        ref = g.compute_dt()
        cons, bx, by, bz = _dev(pr)
        out.fill_(-1.0)
        P.cfl_dt_noalloc(g, cons, bx, by, bz, out)
        torch.cuda.synchronize()
        got = out.item()
        g.close()
        assert abs(got - ref) <= TOL * ref, (pr.name, got, ref)


def test_noalloc_rejects_grids_beyond_its_scratch(P):
    import torch
    pr = W.orszag_tang(16)
    g = P.Grid(pr)
    cons, bx, by, bz = _dev(pr)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = P.GridDesc.from_buffer_copy(g.desc)
    d.n[0], d.n[1], d.n[2] = 1024, 1024, 128          # 2^27 cells > 2^26 maximum
    # through the C entry point itself (the binding would already refuse the
    # small arrays for this descriptor)
    import ctypes
    st = P.lib().phl_cfl_dt_noalloc(ctypes.byref(d), cons.data_ptr(), bx.data_ptr(), by.data_ptr(),
                                    bz.data_ptr(), out.data_ptr(), None)
    assert st == 1 and "too many cells" in P.lib().phl_last_error().decode()
    # a factor beyond the maximum on its own, and a product that would
    # overflow a 64-bit count, are refused the same way
    for n in ((2 ** 31 - 1, 1, 1), (2 ** 30, 2 ** 30, 2 ** 30)):
        d.n[0], d.n[1], d.n[2] = n
        st = P.lib().phl_cfl_dt_noalloc(ctypes.byref(d), cons.data_ptr(), bx.data_ptr(), by.data_ptr(),
                                        bz.data_ptr(), out.data_ptr(), None)
        assert st == 1 and "too many cells" in P.lib().phl_last_error().decode()
    g.close()


def test_noalloc_on_a_stream_matches_compute_dt(P):
    """The same call queued on a side stream (its handle passed through the
    C ABI), synchronised on that stream only."""
    import torch
    pr = W.stratified_box(40, 32, 48, amp=3e-2)
    g = P.Grid(pr)
    g.load()
    ref = g.compute_dt()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        cons, bx, by, bz = _dev(pr)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    s.synchronize()
    P.cfl_dt_noalloc(g, cons, bx, by, bz, out, stream=s.cuda_stream)
    s.synchronize()
    got = out.item()
    g.close()
    assert abs(got - ref) <= TOL * ref, (got, ref)


@pytest.mark.parametrize("bad", ["nan", "negative_pressure", "zero_density"])
def test_noalloc_marks_a_bad_state_with_zero(P, bad):
    """One cell without a sound speed makes dt_out exactly 0 (the call has no
    error word of its own); phl_compute_dt reports the same state as an
    error."""
    import torch
    pr = W.orszag_tang(32)
    k = (0, 7, 9)
    if bad == "nan":
        pr.cons[(4,) + k] = np.nan
    elif bad == "negative_pressure":
        pr.cons[(4,) + k] = 1e-3 * pr.cons[(4,) + k] - 1.0   # internal energy < 0
    else:
        pr.cons[(0,) + k] = 0.0
    cons, bx, by, bz = _dev(pr)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    g = P.Grid(pr)
    P.cfl_dt_noalloc(g, cons, bx, by, bz, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    with pytest.raises(P.PhlError):
        g.load()
        g.compute_dt()
    g.close()


def test_noalloc_rejects_host_memory(P):
    """Host arrays are refused by the binding and, passed as raw pointers,
    by the C entry point itself (PHL_EINVAL) before anything is launched."""
    import ctypes
    import torch
    pr = W.orszag_tang(16)
    g = P.Grid(pr)
    cons, bx, by, bz = _dev(pr)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PhlError):
        P.cfl_dt_noalloc(g, pr.cons, bx, by, bz, out)            # numpy array
    with pytest.raises(P.PhlError):
        P.cfl_dt_noalloc(g, cons.float(), bx, by, bz, out)       # float32 tensor
    host = np.ascontiguousarray(pr.cons)
    st = P.lib().phl_cfl_dt_noalloc(ctypes.byref(g.desc), host.ctypes.data, bx.data_ptr(), by.data_ptr(),
                                    bz.data_ptr(), out.data_ptr(), None)
    assert st == 1 and "not device memory" in P.lib().phl_last_error().decode()
    g.close()
