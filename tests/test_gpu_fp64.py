"""Parity of the FP64 form (CUDA, through the C ABI) with the oracle."""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu

# The FP64 form must reproduce the oracle's per-step estimates to 1e-10
# relative.  Both sides sum O(mC2) terms of both signs in different orders,
# so the bound is taken relative to max(|I'_n|, 1e-3 <|f|>) where <|f|> is the
# oracle's mean absolute pair-of-pairs term (the scale of the cancellation).
REL = 1e-10


def _check_steps(got, want, absmean):
    scale = np.maximum(np.abs(want), 1e-3 * absmean)
    err = np.abs(got - want) / scale
    assert np.all(err <= REL), (err.max(), got, want)


@pytest.fixture(scope="module")
def medium():
    return synthetic.make_system("medium")


@pytest.fixture(scope="module")
def medium_oracle(medium):
    return oracle.Oracle(medium)


@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (9, 2), (33, 1)])
def test_replay_matches_oracle_tiny(tiny, tiny_oracle, m, n_tau):
    n = 3
    r = synthetic.walker_positions(tiny.centres, n, m, seed=100 + m)
    tau = synthetic.imaginary_times(tiny_oracle.lam(), n, n_tau, seed=7 + m)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_FP64)
    got = ctx.eval_fixed(r, tau)
    want, absmean = tiny_oracle.eval_steps(r, tau, with_abs=True)
    _check_steps(got, want, absmean)


def test_replay_edge_times(tiny, tiny_oracle):
    """tau = 0 (no damping at all) and a long time where most terms underflow."""
    m = 8
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=3)
    tau = np.array([[0.0], [40.0]])
    ctx = pkg.Context(tiny, m, 1, pkg.MCMP2_FP64)
    got = ctx.eval_fixed(r, tau)
    want, absmean = tiny_oracle.eval_steps(r, tau, with_abs=True)
    _check_steps(got, want, absmean)


def test_replay_matches_oracle_medium_system(medium, medium_oracle):
    m, n_tau = 40, 2
    r = synthetic.walker_positions(medium.centres, 1, m, seed=21)
    tau = synthetic.imaginary_times(medium_oracle.lam(), 1, n_tau, seed=22)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_FP64)
    got = ctx.eval_fixed(r, tau)
    want, absmean = medium_oracle.eval_steps(r, tau, with_abs=True)
    _check_steps(got, want, absmean)


def _tile_pairs(bp, bq, tp, m):
    ps, qs = [], []
    for i in range(tp):
        for j in range(tp):
            p, q = bp * tp + i, bq * tp + j
            if p < m and q < m and (bp < bq or i < j):
                ps.append(p)
                qs.append(q)
    return np.array(ps), np.array(qs)


def _tile_index(bp, bq, nb):
    return sum(nb - b for b in range(bp)) + (bq - bp)


def test_full_size_sampled_tiles_match_oracle(medium, medium_oracle):
    """The bench configuration (m = 1024, 4 times): sampled tiles against the oracle."""
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium.centres, 1, m, seed=31)
    tau = synthetic.imaginary_times(medium_oracle.lam(), 1, n_tau, seed=32)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_FP64)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    nb = (m + tp - 1) // tp
    npairs = m * (m - 1) / 2
    assert step == pytest.approx(partials.sum() / npairs / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (0, 1), (5, 77), (nb - 1, nb - 1), (63, nb - 1), (100, 101)]:
        ps, qs = _tile_pairs(bp, bq, tp, m)
        vals = medium_oracle.eval_pairs(r[0], tau[0], ps, qs)  # [n_sel, n_tau]
        want = vals.sum(axis=0)
        got = partials[:, _tile_index(bp, bq, nb)]
        scale = np.maximum(np.abs(want), 1e-3 * np.abs(vals).sum(axis=0))
        assert np.all(np.abs(got - want) <= REL * scale), (bp, bq, got, want)


def test_walk_times_and_estimates_follow_the_oracle(tiny, tiny_oracle):
    """Device Metropolis (with burn-in adaptation), inverse-CDF times and
    estimates reproduce the oracle's walk from the same Philox counters."""
    m, n_tau, seed, burn = 16, 2, 4242, 100
    r0 = synthetic.walker_positions(tiny.centres, 1, m, seed=5)[0]
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_FP64)
    ctx.set_walkers(r0, seed, burn)
    r_o, d_o = tiny_oracle.burn_in(r0, seed, burn)
    r_g, d_g = ctx.get_walkers()
    assert d_g == d_o
    np.testing.assert_allclose(r_g, r_o, rtol=0, atol=1e-12)
    lam = tiny_oracle.lam()
    for st in range(25):
        res = ctx.run_steps(1, seed)
        r_o, _ = tiny_oracle.metropolis(r_o, seed, burn + st, 1, d_o)
        tau = oracle.tau_draws(seed, burn + st, n_tau, lam)
        want, absmean = tiny_oracle.eval_steps(r_o[None], tau[None], with_abs=True)
        r_g, _ = ctx.get_walkers()
        np.testing.assert_allclose(r_g, r_o, rtol=0, atol=1e-12)
        _check_steps(np.array([res["last_step"]]), want, absmean)


def test_blocking_statistics_match_oracle(tiny_soft, soft_oracle):
    m, n_tau, seed, burn, n = 16, 1, 77, 60, 320
    r0 = synthetic.walker_positions(tiny_soft.centres, 1, m, seed=9)[0]
    ctx = pkg.Context(tiny_soft, m, n_tau, pkg.MCMP2_FP64)
    ctx.set_walkers(r0, seed, burn)
    res = ctx.run_steps(n, seed)
    ref = soft_oracle.run(r0, seed, burn, n, n_tau)
    I, s2, sb, nb = oracle.blocking(ref["per_step"])
    assert res["steps"] == n and res["n_blocks"] == nb == 3
    assert res["energy"] == pytest.approx(I, rel=1e-9, abs=1e-12)
    assert res["variance"] == pytest.approx(s2, rel=1e-8)
    assert res["error"] == pytest.approx(sb, rel=1e-8)
    assert res["mean_all"] == pytest.approx(ref["per_step"].mean(), rel=1e-9, abs=1e-12)
    assert res["accept_rate"] == pytest.approx(ref["accepted"] / (m * n), rel=1e-12)


def test_checkpoint_restore_is_bit_identical(tiny_soft):
    m, seed = 12, 5
    r0 = synthetic.walker_positions(tiny_soft.centres, 1, m, seed=1)[0]
    ctx = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_FP64)
    ctx.set_walkers(r0, seed, 40)
    ctx.run_steps(130, seed)
    blob = ctx.checkpoint()
    a = ctx.run_steps(150, seed)
    wa, _ = ctx.get_walkers()
    other = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_FP64)
    other.restore(blob)
    b = other.run_steps(150, seed)
    wb, _ = other.get_walkers()
    assert a == b
    assert np.array_equal(wa, wb)
    with pytest.raises(pkg.McMp2Error):
        other.restore(blob[:-8])


def test_invalid_inputs_are_reported(tiny):
    ctx = pkg.Context(tiny, 4, 1, pkg.MCMP2_FP64)
    r = synthetic.walker_positions(tiny.centres, 1, 4, seed=1)
    r[0, 1, 0, 2] = np.nan
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.eval_fixed(r, np.ones((1, 1)))
    assert e.value.code == -4
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.eval_fixed(synthetic.walker_positions(tiny.centres, 1, 4, seed=1), -np.ones((1, 1)))
    assert e.value.code == -1
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.run_steps(1, 0)  # walkers never set
    assert e.value.code == -2


def test_initial_draw_follows_the_weight_function(tiny):
    """set_walkers(None): positions drawn from the mixture g; per-electron mean and
    mean squared distance from the origin match the mixture's closed forms."""
    import math
    m = 20000
    ctx = pkg.Context(tiny, m, 1, pkg.MCMP2_FP64)
    ctx.set_walkers(None, 99, 0)
    r, _ = ctx.get_walkers()
    pts = r.reshape(-1, 3)
    masses, means, second = [], [], []
    for R, (c1, z1, c2, z2) in zip(tiny.centres, tiny.weight):
        for c, z in ((c1, z1), (c2, z2)):
            masses.append(c * (2 * z / math.pi) ** 0.75 * (math.pi / z) ** 1.5)
            means.append(R)
            second.append(R @ R + 3 * 0.5 / z)
    w = np.array(masses) / np.sum(masses)
    mean = (w[:, None] * np.array(means)).sum(axis=0)
    msq = float(w @ np.array(second))
    n = len(pts)
    sd = np.sqrt(np.maximum(msq - mean @ mean, 1e-12) / n)
    assert np.all(np.abs(pts.mean(axis=0) - mean) < 6 * sd + 1e-12)
    d2 = (pts ** 2).sum(axis=1)
    assert abs(d2.mean() - msq) < 6 * d2.std() / np.sqrt(n)
