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
    with pytest.raises(P.PhlError) as e:
        P.cfl_dt_noalloc(d, cons, bx, by, bz, out)
    assert e.value.status == 1 and "too many cells" in str(e.value)
    g.close()
