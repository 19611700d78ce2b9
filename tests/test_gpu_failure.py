"""Failure reporting without a device fault: a bounded wait that runs out.

The tensor-core contraction limits every wait in time.  The test hook makes
the next launch withhold its first operand copy (a barrier nothing
completes); the kernel must give up within the limit, drain, free tensor
memory and return, the call must report MCMP2_ETIMEOUT, the statistics must
be untouched, and the same context must then compute correct results.
"""
import numpy as np
import pytest

import paper_2203_05632_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu


def test_contraction_wait_times_out_and_context_recovers(tiny, tiny_oracle):
    m, n_tau = 16, 1
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=71)
    tau = synthetic.imaginary_times(tiny_oracle.lam(), 2, n_tau, seed=72)
    want, absmean = tiny_oracle.eval_steps(r, tau, with_abs=True)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_MIXED)
    ctx.test_stall_next(0.25)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.eval_fixed(r[:1], tau[:1])
    assert e.value.code == -5  # MCMP2_ETIMEOUT
    got = ctx.eval_fixed(r, tau)  # the context is still usable
    assert np.all(np.abs(got - want) <= 2e-3 * np.abs(want) + 1e-4 * absmean)


def test_timed_out_step_leaves_statistics_untouched(tiny_soft):
    m = 16
    ctx = pkg.Context(tiny_soft, m, 1, pkg.MCMP2_MIXED)
    ctx.set_walkers(None, 5, 20)
    before = ctx.run_steps(3, 5)
    ctx.test_stall_next(0.25)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.run_steps(1, 5)
    assert e.value.code == -5
    after = ctx.run_steps(0, 5)
    assert after["steps"] == before["steps"] and after["mean_all"] == before["mean_all"]
    res = ctx.run_steps(4, 5)
    assert res["steps"] == 7 and np.isfinite(res["mean_all"])


@pytest.mark.parametrize("prec,rel,ab", [(pkg.MCMP2_MIXED, 2e-3, 1e-4), (pkg.MCMP2_TF32, 6.4e-2, 3.2e-3)])
def test_operator_terms_contraction_times_out_and_recovers(tiny, prec, rel, ab):
    """The contraction instances with the Breit terms share the bounded waits: the same
    withheld copy ends the launch with MCMP2_ETIMEOUT, and the context then computes the
    Breit estimate within its tolerance (that of tests/test_gpu_breit.py: the form's
    Coulomb tolerance, absolute part x 9 = sum_AB |c_A c_B|)."""
    import oracle
    orc = oracle.Oracle(tiny, interaction=pkg.MCMP2_BREIT)
    m, n_tau = 33, 2
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=73)
    tau = synthetic.imaginary_times(orc.lam(), 2, n_tau, seed=74)
    want, abs_sum = orc.eval_steps(r, tau, with_abs=True)
    ctx = pkg.Context(tiny, m, n_tau, prec)
    ctx.set_interaction(pkg.MCMP2_BREIT)
    ctx.test_stall_next(0.25)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.eval_fixed(r[:1], tau[:1])
    assert e.value.code == -5  # MCMP2_ETIMEOUT
    got = ctx.eval_fixed(r, tau)
    assert np.all(np.abs(got - want) <= rel * np.abs(want) + 9.0 * ab * abs_sum), (got, want)
