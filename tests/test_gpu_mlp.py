"""The temperature-guess network on the device vs the CPU oracle, and what it
gains the EOS inversion.

* FP32 forward/backward kernels: loss and gradient against the oracle's FP64
  backpropagation with the same weights.
* BF16 tensor-core inference against the oracle's forward pass with the
  weights rounded to BF16.
* Training on device-generated EOS samples; Newton iterations from the
  network's guess vs a cold guess; converged T unchanged (1e-12).
* A stellar box stepped with and without the network: same state to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

NIN, NH = 3, 64
A, Z = W.STELLAR_A, W.STELLAR_Z


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


@pytest.fixture(scope="module")
def table(P):
    return P.EosTable()


@pytest.fixture(scope="module")
def trained(P, table):
    m = P.Mlp(seed=11)
    st = m.train(table, nsamples=2_000_000, epochs=4, batch=1024, lr=1e-2, seed=99)
    return m, st


def _random_weights(seed, scale=0.4):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * rng.standard_normal(NH * NIN + NH + NH * NH + NH + NH + 1)).astype(np.float32)


def _bf16(a):
    """Round float32 to the nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32)


def _bf16_weights(w):
    """Weight matrices representable in BF16 (the training forward pass uses
    them rounded as inference does), biases left in FP32."""
    w = w.copy()
    o_b1, o_w2, o_b2, o_w3 = NH * NIN, NH * NIN + NH, NH * NIN + NH + NH * NH, NH * NIN + 2 * NH + NH * NH
    w[:o_b1] = _bf16(w[:o_b1])
    w[o_w2:o_b2] = _bf16(w[o_w2:o_b2])
    w[o_w3:o_w3 + NH] = _bf16(w[o_w3:o_w3 + NH])
    return w


def test_fp32_gradient_matches_oracle_backprop(P):
    m = P.Mlp(seed=5)
    w = _bf16_weights(_random_weights(1))
    m.set_weights(w)
    rng = np.random.Generator(np.random.PCG64(2))
    n = 5000
    x = rng.uniform(-1, 1, size=(n, NIN)).astype(np.float32)
    t = rng.uniform(-1, 1, size=n).astype(np.float32)
    loss, g = m.loss_grad(x, t)
    lo, go = O.mlp_loss_grad(w.astype(np.float64), NIN, NH, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    # per parameter block, relative to the block's largest gradient
    offs = [0, NH * NIN, NH * NIN + NH, NH * NIN + NH + NH * NH, NH * NIN + 2 * NH + NH * NH,
            NH * NIN + 3 * NH + NH * NH, w.size]
    for a, b in zip(offs[:-1], offs[1:]):
        err = np.abs(g[a:b] - go[a:b]).max() / np.abs(go[a:b]).max()
        assert err <= 1e-4, (a, b, err)


def test_bf16_tensor_core_forward_vs_oracle(P):
    m = P.Mlp(seed=5)
    w = _random_weights(3, scale=0.3)
    m.set_weights(w)
    rng = np.random.Generator(np.random.PCG64(4))
    n = 4099                      # several warps and a ragged tail
    x = rng.uniform(-1, 1, size=(n, NIN)).astype(np.float32)
    y = m.forward(x)
    yo = O.mlp_forward(_bf16_weights(w).astype(np.float64), NIN, NH, x.astype(np.float64))
    scale = max(1.0, np.abs(yo).max())
    # weights rounded to BF16 on both sides; activations carried as BF16 hi + lo
    # pairs (~2^-17 relative); tanh is the hardware approximation (~2^-11)
    assert np.abs(y - yo).max() <= 5e-3 * scale, np.abs(y - yo).max()
    assert np.abs(y - yo).mean() <= 1e-3 * scale, np.abs(y - yo).mean()


def test_training_converges(trained):
    _, st = trained
    assert np.isfinite(st["final_loss"])
    # log10 T within a few hundredths on held-out samples: a few per cent in T
    assert st["val_rms_log10T"] < 0.02, st
    assert st["val_max_log10T"] < 0.2, st


def _samples(table, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lr = rng.uniform(5.0, 7.0, n)
    lt = rng.uniform(8.0, np.log10(3e9), n)
    x0 = rng.uniform(0.0, 1.0, n)
    ot = O.EosTable()
    cfg = O.stellar_cfg(A, Z, ot)
    rho, T = 10 ** lr, 10 ** lt
    r = [O.eos_rt(cfg, rho[i], T[i], [x0[i], 1 - x0[i]]) for i in range(n)]
    e = np.array([q["e"] for q in r])
    cond = np.array([max(1.0, q["e"] / (q["cv"] * T[i])) for i, q in enumerate(r)])
    abar = 1.0 / (x0 / A[0] + (1 - x0) / A[1])
    ye = x0 * Z[0] / A[0] + (1 - x0) * Z[1] / A[1]
    return rho, e, x0, abar, ye, T, cond


def test_network_guess_saves_newton_iterations(P, table, trained):
    m, _ = trained
    rho, e, x0, abar, ye, T, cond = _samples(table, 2000, 7)
    g_mlp = m.guess_T(table, rho, e, x0)
    assert np.abs(np.log10(g_mlp / T)).mean() < 0.05
    cold = np.full_like(rho, 1e9)
    r_mlp = P.eos(table, rho, e, abar, ye, g_mlp)
    r_cold = P.eos(table, rho, e, abar, ye, cold)
    assert (r_mlp["iters"] > 0).all() and (r_cold["iters"] > 0).all()
    # the criterion: the converged temperature does not depend on the guess, to
    # 1e-12 or the rounding floor of e amplified by e / (c_v T) (degenerate
    # electrons), whichever is larger
    assert (np.abs(r_mlp["T"] / r_cold["T"] - 1) <= np.maximum(1e-12, 2e-14 * cond)).all()
    it_mlp, it_cold = r_mlp["iters"].mean(), r_cold["iters"].mean()
    print(f"\nNewton iterations per inversion: network guess {it_mlp:.2f}, cold guess (1e9 K) {it_cold:.2f}")
    assert it_mlp < it_cold


def test_grid_with_network_guess_matches_plain_newton(P, table, trained):
    m, _ = trained
    pr = W.stellar_box(16, 16, 32, amp=3e-2, beta=1e3, mach_heat=3e-2, vel_amp=1e-2)
    out = []
    for net, mode in ((None, 0), (m, 1), (m, 2)):
        g = P.Grid(pr, eos_table=table, mlp=net, mlp_mode=mode)
        g.load()
        g.step(5)
        st = g.get_state()
        st["iters"] = g.stats()["newton_iters"]
        g.close()
        out.append(st)
    a = out[0]
    for b in out[1:]:
        for v in range(a["cons"].shape[0]):
            e = np.abs(a["cons"][v] - b["cons"][v]).max() / np.abs(a["cons"][v]).max()
            assert e <= 1e-12, (v, e)
        for k in ("bx", "by", "bz"):
            e = np.abs(a[k] - b[k]).max() / np.abs(a[k]).max()
            assert e <= 1e-12, (k, e)
        assert np.abs(a["T"] / b["T"] - 1).max() <= 1e-12
    print(f"\nNewton iterations over 5 steps: previous-T guess {a['iters']}, network guess first "
          f"{out[1]['iters']}, network only without a previous T {out[2]['iters']}")
    # with previous temperatures available everywhere, mode 2 is plain Newton
    assert out[2]["iters"] == a["iters"]


def test_cold_start_from_conserved_state(P, table, trained):
    """A stellar state loaded from conserved variables without temperatures:
    the first inversions start from the network's guess (or the table's
    mid-range T without it); same converged state, fewer iterations."""
    m, _ = trained
    ot = O.EosTable()
    pr = O.prepare_stellar(W.stellar_box(16, 16, 32, amp=3e-2, beta=1e3, mach_heat=3e-2, vel_amp=1e-2), ot)
    out = []
    for net in (None, m):
        g = P.Grid(pr, eos_table=table, mlp=net, mlp_mode=2)
        g.set_state(np.ascontiguousarray(pr.cons), np.ascontiguousarray(pr.bx), np.ascontiguousarray(pr.by),
                    np.ascontiguousarray(pr.bz), None)
        g.step(1)
        st = g.get_state()
        st["iters"] = g.stats()["newton_iters"]
        g.close()
        out.append(st)
    a, b = out
    for v in range(a["cons"].shape[0]):
        e = np.abs(a["cons"][v] - b["cons"][v]).max() / np.abs(a["cons"][v]).max()
        assert e <= 1e-12, (v, e)
    assert np.abs(a["T"] / b["T"] - 1).max() <= 1e-12
    print(f"\nNewton iterations, first step from conserved state: mid-table guess {a['iters']}, "
          f"network guess {b['iters']}")
    assert b["iters"] < a["iters"]
