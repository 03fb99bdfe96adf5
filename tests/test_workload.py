"""The seeded input module both sides read (paper_2105_06975_gb300/workload.py):
deterministic draws, the shapes and ranges each workload's recipe states, and
the batched workload's window mix."""
import numpy as np
import pytest

from paper_2105_06975_gb300 import workload as W


def same_draws(a, b):
    if a.bump_center != b.bump_center:
        return False
    for name in ("obs_idx", "z_b", "z_q", "z_r", "x0_pert", "rhs_probe"):
        if not np.array_equal(getattr(a, name), getattr(b, name)):
            return False
    return a.extra.keys() == b.extra.keys() and all(np.array_equal(a.extra[k], b.extra[k]) for k in a.extra)


@pytest.mark.parametrize("w", [W.TINY, W.small(W.SCALE, s=128, N=5, p=40), W.small(W.L96, s=40, N=4, p=20),
                               W.HEAT.with_(s=64, N=3, p=16, msoar_b=(0.4, 0.6, 6), msoar_q=(0.2, 0.5, 7))])
def test_draws_are_deterministic_and_shaped(w):
    a, b, c = W.draws(w, 3), W.draws(w, 3), W.draws(w, 4)
    assert same_draws(a, b) and not same_draws(a, c)
    assert a.obs_idx.dtype == np.int32 and a.obs_idx.shape == (w.p,)
    assert np.all(np.diff(a.obs_idx) > 0) and a.obs_idx[0] >= 0 and a.obs_idx[-1] < w.s
    assert a.z_b.shape == (w.s,) and a.z_q.shape == (w.N, w.s) and a.z_r.shape == (w.N + 1, w.p)
    assert a.rhs_probe.shape == (w.n,) and 0.0 <= a.bump_center < 1.0
    if w.obs == "even":
        assert np.array_equal(a.obs_idx, np.arange(w.p) * (w.s // w.p))


def test_heat_draws_and_block_sizes():
    w = W.HEAT.with_(s=64, N=3, p=16)
    d = W.draws(w, 0)
    assert d.extra["psi"].shape == (2,) and np.all((0 <= d.extra["psi"]) & (d.extra["psi"] < 0.5))
    nb = len(W.block_sizes(w.p, w.r_blocks))
    assert d.extra["pcorr_on"].shape == (nb * (nb - 1) // 2,) and d.extra["r_u"].shape == (w.p, w.p)
    for p, k in [(16, 8), (17, 8), (5, 8), (12500, 8), (7, 1)]:
        b = W.block_sizes(p, k)
        assert b.sum() == p and b.min() >= 1 and b.max() - b.min() <= 1 and len(b) == min(k, p)
    assert W.HEAT.n == (2 * 50000 + 12500) * 6


def test_batch_windows_mix():
    """Config 3's windows: s = 4 U{32..512}, N = U{8..96}, p = s/2 or s/4,
    advection-diffusion or Lorenz-96 (dt = 1e-4) by a fair coin; seeds
    1000 m + w; the same list for the same master seed."""
    ws = W.batch_windows(256, seed=1)
    assert ws == W.batch_windows(256, seed=1) and ws != W.batch_windows(256, seed=2)
    kinds = {w.model for w, _ in ws}
    assert kinds == {"advdiff", "l96"}
    for i, (w, seed) in enumerate(ws):
        assert seed == 1000 + i
        assert w.s % 4 == 0 and 128 <= w.s <= 2048 and 8 <= w.N <= 96 and w.p in (w.s // 2, w.s // 4)
        if w.model == "l96":
            assert w.dt == 1e-4 and w.outer_loops == 1
    n_l96 = sum(w.model == "l96" for w, _ in ws)
    assert 80 < n_l96 < 176            # a fair coin over 256 windows


def test_small_keeps_length_units():
    """small(): domain-fraction lengths stay for the linear workloads, grid-point
    lengths scale with s for Lorenz-96."""
    a = W.small(W.SCALE, s=256, N=4)
    assert a.soar_b == W.SCALE.soar_b and a.p == 256 * W.SCALE.p // W.SCALE.s
    b = W.small(W.L96, s=100, N=4)
    assert b.soar_b[1] * 100 == pytest.approx(W.L96.soar_b[1] * W.L96.s)


def test_heat_bands_match_the_oracle_model():
    """The heat model bands the benchmark passes to the library are the
    oracle's Sec. 7.2 model (Dirichlet rows and columns empty)."""
    from oracle import model as mdl
    w = W.small(W.HEAT, s=50, N=3, p=10)
    assert np.array_equal(w.heat_bands(), mdl.heat_model(w.s, w.N, w.heat_r).bands)
