"""The mixed-precision (split-BF16 x3 tensor-core) form against the oracle and the FP64 form."""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import bounds

pytestmark = pytest.mark.gpu

# Tolerances from the error model of each form (oracle/bounds.py): a sum of
# summands (a step estimate, a tile's partial sum) may be off by KAPPA times the
# sum of the summands' model standard deviations plus their FP32 trace terms.
# The per-summand comparison itself is in test_gpu_elements.py.
FORMS = {pkg.MCMP2_MIXED: bounds.BF16X3, pkg.MCMP2_TF32: bounds.TF32, pkg.MCMP2_FP64: bounds.FP64}
REL_MIXED = 2e-3  # per-step difference of split BF16 from the FP64 form along a walk, relative


def _steps_ok(orc, r, tau, got, want, prec=pkg.MCMP2_MIXED, interaction=0):
    """Each replayed step estimate within the model tolerance of its form."""
    tol = bounds.steps_tolerance(orc, r, tau, FORMS[prec], interaction)
    return np.abs(got - want) <= tol


def _tile_ok(orc, r_step, tau_step, ps, qs, got, want, prec=pkg.MCMP2_MIXED, interaction=0):
    """A tile's partial sums (per time) within the model tolerance of its summands."""
    tol = bounds.tile_tolerance(orc, r_step, tau_step, list(zip(ps.tolist(), qs.tolist())), FORMS[prec],
                                interaction)
    return np.abs(got - want) <= tol


@pytest.fixture(scope="module")
def medium():
    return synthetic.make_system("medium")


@pytest.fixture(scope="module")
def medium_oracle(medium):
    return oracle.Oracle(medium)


@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (33, 2)])
def test_mixed_replay_matches_oracle_tiny(tiny, tiny_oracle, m, n_tau):
    n = 3
    r = synthetic.walker_positions(tiny.centres, n, m, seed=400 + m)
    tau = synthetic.imaginary_times(tiny_oracle.lam(), n, n_tau, seed=9 + m)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_MIXED)
    got = ctx.eval_fixed(r, tau)
    want = tiny_oracle.eval_steps(r, tau)
    assert np.all(_steps_ok(tiny_oracle, r, tau, got, want)), (got, want)


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_spinor_units_with_an_odd_position_block_count(medium, medium_oracle, prec):
    """m = 136: 272 positions are three 128-position blocks (the last one ragged), so
    the spinor formation's second CTA pair owns the third block and a phantom fourth
    whose rows are zero-filled and never stored."""
    m, n_tau = 136, 1
    r = synthetic.walker_positions(medium.centres, 1, m, seed=137)
    tau = synthetic.imaginary_times(medium_oracle.lam(), 1, n_tau, seed=138)
    ctx = pkg.Context(medium, m, n_tau, prec)
    got = ctx.eval_fixed(r, tau)
    want = medium_oracle.eval_steps(r, tau)
    assert np.all(_steps_ok(medium_oracle, r, tau, got, want, prec)), (got, want)


def test_mixed_replay_matches_oracle_medium_system(medium, medium_oracle):
    m, n_tau = 40, 2
    r = synthetic.walker_positions(medium.centres, 1, m, seed=41)
    tau = synthetic.imaginary_times(medium_oracle.lam(), 1, n_tau, seed=42)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_MIXED)
    got = ctx.eval_fixed(r, tau)
    want = medium_oracle.eval_steps(r, tau)
    assert np.all(_steps_ok(medium_oracle, r, tau, got, want)), (got, want)


def _tile_pairs(bp, bq, tp, m):
    ps, qs = [], []
    for i in range(tp):
        for j in range(tp):
            p, q = bp * tp + i, bq * tp + j
            if p < m and q < m and (bp < bq or i < j):
                ps.append(p)
                qs.append(q)
    return np.array(ps), np.array(qs)


def test_mixed_full_size_sampled_tiles_match_oracle(medium, medium_oracle):
    """The bench configuration: m = 1024, 4 times; sampled 16 x 16 tiles vs the oracle."""
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium.centres, 1, m, seed=51)
    tau = synthetic.imaginary_times(medium_oracle.lam(), 1, n_tau, seed=52)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_MIXED)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    assert tp == 16
    nb = (m + tp - 1) // tp
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (0, 1), (7, 40), (nb - 1, nb - 1), (31, nb - 1)]:
        ps, qs = _tile_pairs(bp, bq, tp, m)
        vals = medium_oracle.eval_pairs(r[0], tau[0], ps, qs)
        want = vals.sum(axis=0)
        k = sum(nb - b for b in range(bp)) + (bq - bp)
        got = partials[:, k]
        assert np.all(_tile_ok(medium_oracle, r[0], tau[0], ps, qs, got, want)), (bp, bq, got, want)


def test_tensor_forms_agree_with_fp64_form_within_a_fifth_of_sigma(medium):
    """The spec bar at the workload (medium system, m = 1024, 4 times per step):
    on one 2000-step walk (20 blocks of N_b = 100; the Metropolis walk is the same FP64
    arithmetic in every form), the mean difference between the split-BF16 / TF32 step
    estimates and the FP64 form's is below a fifth of the walk's sigma-bar (Eq.
    uncertainty).  The FP64 form (0.4 s per step here) evaluates every 20th step; the
    mean difference over the walk is bounded by the sampled mean plus three of its
    standard errors."""
    m, n_tau, seed, burn, n, every = 1024, 4, 909, 500, 2000, 20
    walk = pkg.Context(medium, m, n_tau, pkg.MCMP2_MIXED)
    walk.set_walkers(None, seed, burn)
    per, steps, pos = [], [], []
    for k in range(n):
        per.append(walk.run_steps(1, seed)["last_step"])
        if k % every == 0:
            steps.append(burn + k)
            pos.append(walk.get_walkers()[0])
    walk.close()
    I, s2, sb, nb = oracle.blocking(np.array(per))
    assert nb == 20
    lam = 2.0 * (medium.eps[medium.n_occ:].min() - medium.eps[:medium.n_occ].max())
    r = np.array(pos)
    tau = np.array([oracle.tau_draws(seed, st, n_tau, lam) for st in steps])
    f64 = pkg.Context(medium, m, n_tau, pkg.MCMP2_FP64).eval_fixed(r, tau)
    mixed_replay = pkg.Context(medium, m, n_tau, pkg.MCMP2_MIXED).eval_fixed(r, tau)
    # the walk's own estimates at the sampled steps are the replayed ones
    np.testing.assert_allclose(mixed_replay, np.array(per)[::every], rtol=1e-12, atol=0)
    for prec in (pkg.MCMP2_MIXED, pkg.MCMP2_TF32):
        got = mixed_replay if prec == pkg.MCMP2_MIXED else pkg.Context(medium, m, n_tau, prec).eval_fixed(r, tau)
        d = got - f64
        bound = abs(d.mean()) + 3.0 * d.std(ddof=1) / np.sqrt(len(d))
        print(f"form {prec}: I_N = {I:.5f} +- {sb:.5f} over {nb} blocks; mean difference from FP64 "
              f"{d.mean():.3e} +- {d.std(ddof=1) / np.sqrt(len(d)):.1e} ({bound / sb:.2e} sigma-bar)")
        assert bound < 0.2 * sb


def test_mixed_walk_statistics_and_checkpoint(tiny_soft):
    m, seed = 16, 21
    r0 = synthetic.walker_positions(tiny_soft.centres, 1, m, seed=2)[0]
    ctx = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_MIXED)
    ctx.set_walkers(r0, seed, 50)
    ctx.run_steps(120, seed)
    blob = ctx.checkpoint()
    a = ctx.run_steps(90, seed)
    other = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_MIXED)
    other.restore(blob)
    b = other.run_steps(90, seed)
    assert a == b
    assert a["steps"] == 210 and a["n_blocks"] == 2 and np.isfinite(a["energy"])


@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED])
def test_profile_counters_time_the_contraction_in_graph_replays(tiny_soft, prec):
    m = 32
    ctx = pkg.Context(tiny_soft, m, 2, prec)
    ctx.set_walkers(None, 3, 20)
    ctx.run_steps(2, 3)  # builds the step graph without timing
    ctx.profile(1)
    for _ in range(5):
        ctx.run_steps_async(1, 3)
    ctx.run_steps(3, 3)
    prof = ctx.profile(0)
    assert prof["pair_launches"] == 8
    assert prof["launches"] >= 8 * 5
    assert prof["pair_ms"] > 0.0
    ctx.profile(2)
    ctx.run_steps(2, 3)
    assert ctx.profile(0)["pair_ms"] == 0.0


def test_timing_mode_outside_graphs(tiny):
    """Replay calls issue kernels directly; timing them must work as well."""
    m = 16
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=8)
    tau = synthetic.imaginary_times(2.0, 2, 1, seed=9)
    for prec in (pkg.MCMP2_FP64, pkg.MCMP2_MIXED):
        ctx = pkg.Context(tiny, m, 1, prec)
        ctx.profile(1)
        ctx.eval_fixed(r, tau)
        prof = ctx.profile(0)
        assert prof["pair_launches"] == 2 and prof["pair_ms"] > 0.0


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_size_series_launch_sampled_tiles(prec):
    """The size-series launch (m = 4096 walker pairs, 8 times; a two-unit cluster,
    80 / 360 spinors): sampled 16 x 16 tiles against the oracle's pair values, in
    the bound of each form (split BF16: the tolerance above; TF32: 8 u times the
    tile's absolute expansion)."""
    system = synthetic.make_system("size", n_units=2)
    orc = oracle.Oracle(system)
    m, n_tau = 4096, 8
    r = synthetic.walker_positions(system.centres, 1, m, seed=61)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=62)
    ctx = pkg.Context(system, m, n_tau, prec)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    nb = (m + tp - 1) // tp
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (3, 200), (nb - 1, nb - 1), (128, nb - 1)]:
        ps, qs = _tile_pairs(bp, bq, tp, m)
        vals = orc.eval_pairs(r[0], tau[0], ps, qs)
        want = vals.sum(axis=0)
        got = partials[:, sum(nb - b for b in range(bp)) + (bq - bp)]
        assert np.all(_tile_ok(orc, r[0], tau[0], ps, qs, got, want, prec)), (bp, bq, got, want)


@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED])
def test_odd_basis_count(tiny, prec):
    """A basis with an odd number of functions (the tiny system without its last s
    shell, n_L = 19): the basis kernels' paired stores fall back to single values."""
    import dataclasses
    n_l = tiny.n_l
    keep = np.ones(len(tiny.shell_l), dtype=bool)
    keep[-1] = False
    assert tiny.shell_l[-1] == 0
    rows = np.concatenate([np.arange(k * n_l, (k + 1) * n_l - 1) for k in range(4)])
    odd = dataclasses.replace(tiny, shell_centre=tiny.shell_centre[keep], shell_l=tiny.shell_l[keep],
                              shell_alpha=tiny.shell_alpha[keep], shell_coef=tiny.shell_coef[keep],
                              C=np.ascontiguousarray(tiny.C[rows]))
    assert odd.n_l == 19
    orc = oracle.Oracle(odd)
    m, n_tau = 16, 2
    r = synthetic.walker_positions(odd.centres, 2, m, seed=91)
    tau = synthetic.imaginary_times(orc.lam(), 2, n_tau, seed=92)
    got = pkg.Context(odd, m, n_tau, prec).eval_fixed(r, tau)
    want, absmean = orc.eval_steps(r, tau, with_abs=True)
    if prec == pkg.MCMP2_FP64:
        assert np.all(np.abs(got - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3 * absmean)), (got, want)
    else:
        assert np.all(_steps_ok(orc, r, tau, got, want)), (got, want)
