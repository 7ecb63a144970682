"""Device functions of the stage vs the oracle's, one face at a time."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def _states(rng, n, mag=True):
    g = 5.0 / 3.0
    w = np.zeros((n, 9))
    w[:, 0] = rng.uniform(0.3, 2.0, n)
    w[:, 1:4] = rng.normal(size=(n, 3))
    if mag:
        w[:, 4:6] = rng.normal(size=(n, 2))
    w[:, 6] = rng.uniform(0.1, 2.0, n)
    w[:, 7] = g
    w[:, 8] = g
    return w


@pytest.mark.parametrize("solver", ["lhlld", "hlld", "hll"])
def test_riemann_fp64_matches_oracle(P, solver):
    rng = np.random.default_rng(21)
    n = 4000
    wl, wr = _states(rng, n), _states(rng, n)
    # a quarter of the faces near rest / low Mach, a quarter with tiny B_n
    wl[: n // 4, 1:4] *= 1e-3
    wr[: n // 4, 1:4] *= 1e-3
    bn = rng.normal(size=n)
    bn[n // 4: n // 2] *= 1e-6
    f = P.riemann_batch(wl, wr, bn, solver=solver)
    for t in range(n):
        ref = O.riemann(wl[t], wr[t], bn[t], solver)
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(f[t] - ref).max() <= 1e-12 * scale, (t, f[t], ref)


def test_riemann_deviation_form_matches_full_form(P):
    """With a background, the device returns F(W_hat + dW) - F(W_hat, W_hat)."""
    rng = np.random.default_rng(8)
    n = 2000
    g = 5.0 / 3.0
    bg = np.zeros((n, 4))
    bg[:, 0] = rng.uniform(0.1, 1.0, n)
    bg[:, 1] = rng.uniform(0.01, 1.0, n)
    bg[:, 2:] = g
    dl, dr = _states(rng, n) * 1e-2, _states(rng, n) * 1e-2
    for d in (dl, dr):
        d[:, 7:9] = 0.0
    bn = rng.normal(size=n) * 1e-2
    f = P.riemann_batch(dl, dr, bn, bg=bg, solver="lhlld")
    for t in range(n):
        full_l, full_r = dl[t].copy(), dr[t].copy()
        for w in (full_l, full_r):
            w[0] += bg[t, 0]
            w[6] += bg[t, 1]
            w[7] = w[8] = g
        wb = np.array([bg[t, 0], 0, 0, 0, 0, 0, bg[t, 1], g, g])
        ref = O.riemann(full_l, full_r, bn[t], "lhlld") - O.riemann(wb, wb, 0.0, "lhlld")
        assert np.abs(f[t] - ref).max() <= 1e-12 * max(bg[t, 1], 1e-3), (t, f[t], ref)


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 0, 1)])
def test_orszag_tang_in_other_planes_gpu(P, perm):
    q = W.permute_axes(W.orszag_tang(48), list(perm))
    g = P.Grid(q)
    g.load()
    g.step(20, 2e-3)
    st = g.get_state()
    g.close()
    ref, _, _ = O.Oracle(q).run(20, dt_fixed=2e-3)
    for v in range(5):
        e = np.abs(st["cons"][v] - ref["cons"][v]).max() / max(np.abs(ref["cons"][v]).max(), 1e-300)
        assert e < 1e-12, (v, e)
    for k in ("bx", "by", "bz"):
        e = np.abs(st[k] - ref[k]).max() / max(np.abs(ref[k]).max(), 1e-300)
        assert e < 1e-12, (k, e)


def test_periodic_3d_box_one_step(P):
    pr = W.stratified_box(16, 12, 20, amp=2e-2)
    pr.bc = ((0, 0), (0, 0), (0, 0))
    pr.g = (0.0, 0.0, 0.0)
    pr.bg, pr.heat = None, None
    rng = np.random.default_rng(3)
    pr.cons[1:4] += 1e-2 * rng.standard_normal(pr.cons[1:4].shape)
    g = P.Grid(pr)
    g.load()
    g.step(1, 1e-3)
    st = g.get_state()
    g.close()
    ref, _, _ = O.Oracle(pr).run(1, dt_fixed=1e-3)
    for k in ("bx", "by", "bz"):
        d = np.abs(st[k] - ref[k]).max()
        assert d <= 1e-15, (k, d)


@pytest.mark.parametrize("k", [0, -20, 37, -80])
def test_scaled_conversions_match_ieee(P, k):
    """d2f_scaled / f2d_scaled, the mixed form's FP64 <-> FP32 boundary with a
    power-of-two unit folded into the exponent: x * 2^k rounded to nearest
    FP32 (IEEE ties-to-even and the kernel's ties-away agree off exact ties,
    which random doubles never hit), subnormal results flushed to zero,
    overflow to inf, NaN kept; the way back is exact."""
    rng = np.random.default_rng(100 + k)
    scale = 2.0 ** -k
    x = np.concatenate([
        rng.standard_normal(20000) * scale * 10.0 ** rng.uniform(-30, 30, 20000),
        np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan]) * scale,
        np.array([1e-50, -1e-45, 2.0 ** -130, 2.0 ** 129, -2.0 ** 200]) * scale,
    ])
    f, back = P.convert_batch(x, k)
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        ref = (x * 2.0 ** k).astype(np.float32)
    tiny = np.abs(ref) < np.float32(2.0 ** -126)
    ref = np.where(tiny, np.copysign(np.float32(0.0), ref), ref)
    nan = np.isnan(x)
    assert np.all(np.isnan(f[nan]))
    assert np.array_equal(f[~nan], ref[~nan])
    assert np.array_equal(np.signbit(f[~nan]), np.signbit(ref[~nan]))
    with np.errstate(over="ignore"):
        expect_back = f.astype(np.float64) * 2.0 ** -k
    assert np.array_equal(back[~nan], expect_back[~nan])
