"""The TF32 tensor-core form against the oracle and the FP64 form.

Tolerance from the error model of the form (oracle/bounds.py): the spinor
values come from the split BF16 x3 products, are scaled and rounded to the
nearest TF32 value (relative error <= 2^-11 per operand) and every propagator
entry is accumulated in FP32; a sum of summands may be off by KAPPA times the
sum of the summands' model standard deviations plus their FP32 trace terms.
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import bounds

pytestmark = pytest.mark.gpu


def _bound(orc, system, r_step, tau_step):
    """Tolerance of one TF32 step estimate (system: unused, kept for the callers' signature)."""
    return bounds.step_tolerance(orc, r_step, tau_step, bounds.TF32)


@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (33, 2)])
def test_tf32_replay_matches_oracle_tiny(tiny, tiny_oracle, m, n_tau):
    n = 2
    r = synthetic.walker_positions(tiny.centres, n, m, seed=400 + m)
    tau = synthetic.imaginary_times(tiny_oracle.lam(), n, n_tau, seed=9 + m)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_TF32)
    got = ctx.eval_fixed(r, tau)
    want = tiny_oracle.eval_steps(r, tau)
    for k in range(n):
        bound = _bound(tiny_oracle, tiny, r[k], tau[k])
        assert abs(got[k] - want[k]) <= bound, (k, got[k], want[k], bound)


def test_tf32_replay_matches_oracle_medium_system():
    medium = synthetic.make_system("medium")
    orc = oracle.Oracle(medium)
    m, n_tau = 24, 2
    r = synthetic.walker_positions(medium.centres, 1, m, seed=41)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=42)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_TF32)
    got = ctx.eval_fixed(r, tau)[0]
    want = orc.eval_steps(r, tau)[0]
    bound = _bound(orc, medium, r[0], tau[0])
    assert abs(got - want) <= bound, (got, want, bound)


def test_tf32_and_bf16x3_forms_share_everything_but_the_contraction(tiny):
    """Same replay in both tensor-core forms: the difference is the TF32 rounding, within its bound,
    and the two forms run the same launches."""
    m, n_tau = 32, 2
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=77)
    tau = synthetic.imaginary_times(2.0, 2, n_tau, seed=78)
    orc = oracle.Oracle(tiny)
    out = {}
    for prec in (pkg.MCMP2_MIXED, pkg.MCMP2_TF32):
        ctx = pkg.Context(tiny, m, n_tau, prec)
        ctx.profile(1)
        out[prec] = ctx.eval_fixed(r, tau)
        prof = ctx.profile(0)
        assert prof["pair_launches"] == 2
    for k in range(2):
        assert abs(out[pkg.MCMP2_TF32][k] - out[pkg.MCMP2_MIXED][k]) <= _bound(orc, tiny, r[k], tau[k])


def test_tf32_walk_checkpoint_round_trip(tiny_soft):
    m, seed = 16, 21
    r0 = synthetic.walker_positions(tiny_soft.centres, 1, m, seed=2)[0]
    ctx = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_TF32)
    ctx.set_walkers(r0, seed, 50)
    ctx.run_steps(120, seed)
    blob = ctx.checkpoint()
    a = ctx.run_steps(90, seed)
    other = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_TF32)
    other.restore(blob)
    b = other.run_steps(90, seed)
    assert a == b
    assert a["steps"] == 210 and a["n_blocks"] == 2 and np.isfinite(a["energy"])


def _tile_pairs(bp, bq, tp, m):
    out = []
    for i in range(tp):
        for j in range(tp):
            p, q = bp * tp + i, bq * tp + j
            if p < m and q < m and (bp < bq or i < j):
                out.append((p, q))
    return out


def test_tf32_full_size_sampled_tiles_match_oracle():
    """The bench configuration (m = 1024, 4 times): sampled 16 x 16 tiles against the oracle's
    per-pair values, each tile's partial sum within the model tolerance of its summands."""
    medium = synthetic.make_system("medium")
    orc = oracle.Oracle(medium)
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium.centres, 1, m, seed=51)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=52)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_TF32)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    assert tp == 16
    nb = (m + tp - 1) // tp
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (7, 40), (nb - 1, nb - 1)]:
        pairs = _tile_pairs(bp, bq, tp, m)
        ps = np.array([p for p, _ in pairs])
        qs = np.array([q for _, q in pairs])
        want = orc.eval_pairs(r[0], tau[0], ps, qs).sum(axis=0)
        bound = bounds.tile_tolerance(orc, r[0], tau[0], pairs, bounds.TF32)
        k = sum(nb - b for b in range(bp)) + (bq - bp)
        got = partials[:, k]
        assert np.all(np.abs(got - want) <= bound), (bp, bq, got, want, bound)
