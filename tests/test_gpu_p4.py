"""P4 on the GPU: long walks of every form against the deterministic MP2 energy.

The Monte Carlo energy of Sec. III (Eq. MCMP2 sampled with the weights of
Eq. basisSet and Eq. tauWeight) must agree within 3 sigma-bar with the
sum-over-states E2 of Eq. FinalMP2, computed by the oracle from its own
Coulomb integrals.  On the soft tiny system the walk covers the orbitals well
and sigma-bar is a small fraction of |E2|; on the literal tiny system (core
exponents far outside the weight function) the estimator is heavy-tailed and
the check is a long run of the FP64 form with its own wide sigma-bar.
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import mp2

pytestmark = pytest.mark.gpu


def _walk(system, prec, m, n_tau, burn, steps, seed):
    ctx = pkg.Context(system, m, n_tau, prec)
    r0 = synthetic.walker_positions(system.centres, 1, m, seed=11)[0]
    ctx.set_walkers(r0, seed, burn)
    res = ctx.run_steps(steps, seed)
    ctx.close()
    return res


@pytest.fixture(scope="module")
def soft_e2(tiny_soft, soft_oracle):
    return mp2.mp2_energy(tiny_soft, mp2.spinor_eri(soft_oracle))


@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_long_walk_matches_deterministic_energy_soft(tiny_soft, soft_e2, prec):
    res = _walk(tiny_soft, prec, 64, 2, 500, 20000, 4242)
    assert res["n_blocks"] == 200
    z = (res["energy"] - soft_e2) / res["error"]
    print(f"soft tiny, precision {prec}: E = {res['energy']:.6f} +- {res['error']:.6f}, E2 = {soft_e2:.6f}, z = {z:.2f}")
    assert abs(z) < 3.0, (res["energy"], res["error"], soft_e2)
    assert res["error"] < 0.05 * abs(soft_e2)
    assert 0.3 < res["accept_rate"] < 0.7


def test_long_walk_matches_deterministic_energy_literal_tiny(tiny, tiny_oracle):
    e2 = mp2.mp2_energy(tiny, mp2.spinor_eri(tiny_oracle))
    res = _walk(tiny, pkg.MCMP2_FP64, 64, 1, 1000, 50000, 77)
    z = (res["energy"] - e2) / res["error"]
    print(f"literal tiny, FP64: E = {res['energy']:.6f} +- {res['error']:.6f}, E2 = {e2:.6f}, z = {z:.2f}")
    assert abs(z) < 3.0, (res["energy"], res["error"], e2)
