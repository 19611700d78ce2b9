"""Pins of the two-component variant (Sec. II: the Monte Carlo algorithm holds
for two-component Hamiltonians), CPU only.

A two-component system has spinors (alpha, beta) over the large basis only; the
oracle evaluates it as the four-component estimator whose small-component rows
are zero, i.e. with 2 x 2 propagator blocks embedded in the 4 x 4 ones.  These
tests pin that evaluation against the explicit sum over states (P2) and the
deterministic MP2 energy (P4) on two-component systems, and check the generator.
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import mp2

from test_oracle_pins import _explicit_sum, _four_points


@pytest.fixture(scope="module")
def tiny2c():
    return synthetic.make_system("tiny", two_component=True)


@pytest.fixture(scope="module")
def soft2c():
    return synthetic.make_system("tiny", soft=True, two_component=True)


def test_generator_gives_orthonormal_kramers_paired_two_spinors(tiny2c):
    n_l = tiny2c.n_l
    assert tiny2c.n_comp == 2
    assert np.all(tiny2c.C[2 * n_l:] == 0)
    s_ll, _ = synthetic.overlap_matrices(tiny2c)
    ca, cb = tiny2c.C[:n_l], tiny2c.C[n_l:2 * n_l]
    M = ca.conj().T @ s_ll @ ca + cb.conj().T @ s_ll @ cb
    np.testing.assert_allclose(M, np.eye(tiny2c.n_orb), atol=1e-10)
    # Kramers partners: phi_{2k+1} = K phi_{2k}, K (a, b) = (-conj b, conj a).
    np.testing.assert_allclose(tiny2c.C[:n_l, 1::2], -np.conj(cb[:, 0::2]), atol=1e-10)
    np.testing.assert_allclose(tiny2c.C[n_l:2 * n_l, 1::2], np.conj(ca[:, 0::2]), atol=1e-10)
    np.testing.assert_array_equal(tiny2c.eps[0::2], tiny2c.eps[1::2])


@pytest.mark.parametrize("tau", [0.05, 0.7])
def test_two_component_trace_form_equals_explicit_sum_over_states(tiny2c, tau):
    """P2 for two-spinors: the trace form equals the orbital sum of Eq. FinalMP2
    with rho_kl = phi_k^dag phi_l over the two components."""
    orc = oracle.Oracle(tiny2c)
    pts = _four_points()
    got = orc.pair_value(*pts, tau)
    want = _explicit_sum(orc, tiny2c, pts, tau)
    assert abs(got - want) <= 1e-11 * abs(want)
    # The spinor values really have two components.
    assert np.all(orc.spinors_at(pts[0])[:, 2:] == 0)


def test_two_component_mc_estimate_matches_deterministic_mp2(soft2c):
    """P4 for the two-component variant: the oracle's walk agrees with the
    sum-over-states E2 within 3 sigma."""
    orc = oracle.Oracle(soft2c)
    E2 = mp2.mp2_energy(soft2c, mp2.spinor_eri(orc))
    r0 = synthetic.walker_positions(soft2c.centres, 1, 16, seed=11)[0]
    means, errs = [], []
    for seed in range(6):
        res = orc.run(r0, 200 + seed, 300, 3000, 1)
        I, _, sb, _ = oracle.blocking(res["per_step"])
        means.append(I)
        errs.append(sb)
    mean = float(np.mean(means))
    err = float(np.sqrt(np.sum(np.square(errs)))) / len(errs)
    assert abs(mean - E2) < 3.0 * err, (mean, err, E2)
    assert err < 0.25 * abs(E2)
