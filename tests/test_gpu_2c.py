"""The two-component variant (mcmp2_load_system_2c) against the oracle, in all three forms.

Two-spinors (alpha, beta) over the large basis: G- and G+ are 2 x 2 blocks in the
trace form of Eq. MCMP2 (Sec. II names two-component Hamiltonians as covered by
the same algorithm).  Parity bar as for the four-component FP64 form: 1e-10
relative per step estimate, relative to max(|I'_n|, 1e-3 <|f|>); the tensor-core
forms (32 x 32-pair tiles) are held to the bounds of their four-component tests.
The oracle evaluates the same estimator with the small-component rows of C zero.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import mp2

from test_gpu_fp64 import _check_steps, _tile_index, _tile_pairs
from test_gpu_mixed import _steps_ok, _tile_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny2c():
    return synthetic.make_system("tiny", two_component=True)


@pytest.fixture(scope="module")
def tiny2c_oracle(tiny2c):
    return oracle.Oracle(tiny2c)


@pytest.fixture(scope="module")
def medium2c():
    return synthetic.make_system("medium", two_component=True)


@pytest.fixture(scope="module")
def medium2c_oracle(medium2c):
    return oracle.Oracle(medium2c)


@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (33, 2)])
def test_two_component_replay_matches_oracle_tiny(tiny2c, tiny2c_oracle, m, n_tau):
    n = 3
    r = synthetic.walker_positions(tiny2c.centres, n, m, seed=400 + m)
    tau = synthetic.imaginary_times(tiny2c_oracle.lam(), n, n_tau, seed=9 + m)
    ctx = pkg.Context(tiny2c, m, n_tau, pkg.MCMP2_FP64)
    got = ctx.eval_fixed(r, tau)
    want, absmean = tiny2c_oracle.eval_steps(r, tau, with_abs=True)
    _check_steps(got, want, absmean)


def test_two_component_replay_matches_oracle_medium(medium2c, medium2c_oracle):
    m, n_tau = 40, 2
    r = synthetic.walker_positions(medium2c.centres, 1, m, seed=41)
    tau = synthetic.imaginary_times(medium2c_oracle.lam(), 1, n_tau, seed=42)
    ctx = pkg.Context(medium2c, m, n_tau, pkg.MCMP2_FP64)
    got = ctx.eval_fixed(r, tau)
    want, absmean = medium2c_oracle.eval_steps(r, tau, with_abs=True)
    _check_steps(got, want, absmean)


def test_two_component_full_size_sampled_tiles(medium2c, medium2c_oracle):
    """m = 1024 walker pairs, 4 times: sampled tiles against the oracle's pair values."""
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium2c.centres, 1, m, seed=51)
    tau = synthetic.imaginary_times(medium2c_oracle.lam(), 1, n_tau, seed=52)
    ctx = pkg.Context(medium2c, m, n_tau, pkg.MCMP2_FP64)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    nb = (m + tp - 1) // tp
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (3, 90), (nb - 1, nb - 1), (64, nb - 1)]:
        ps, qs = _tile_pairs(bp, bq, tp, m)
        vals = medium2c_oracle.eval_pairs(r[0], tau[0], ps, qs)
        want = vals.sum(axis=0)
        got = partials[:, _tile_index(bp, bq, nb)]
        scale = np.maximum(np.abs(want), 1e-3 * np.abs(vals).sum(axis=0))
        assert np.all(np.abs(got - want) <= 1e-10 * scale), (bp, bq, got, want)


def test_two_component_equals_four_component_with_zero_small_rows(tiny2c):
    """The 2 x 2 kernels and the 4 x 4 kernels fed the same coefficients (small rows
    zero) give the same step estimates."""
    m, n_tau = 24, 2
    r = synthetic.walker_positions(tiny2c.centres, 2, m, seed=61)
    tau = synthetic.imaginary_times(oracle.Oracle(tiny2c).lam(), 2, n_tau, seed=62)
    two = pkg.Context(tiny2c, m, n_tau, pkg.MCMP2_FP64).eval_fixed(r, tau)
    four = pkg.Context(dataclasses.replace(tiny2c, n_comp=4), m, n_tau, pkg.MCMP2_FP64).eval_fixed(r, tau)
    np.testing.assert_allclose(two, four, rtol=1e-12, atol=0)


def test_two_component_walk_follows_the_oracle(tiny2c, tiny2c_oracle):
    m, n_tau, seed, burn = 16, 1, 515, 60
    r0 = synthetic.walker_positions(tiny2c.centres, 1, m, seed=6)[0]
    ctx = pkg.Context(tiny2c, m, n_tau, pkg.MCMP2_FP64)
    ctx.set_walkers(r0, seed, burn)
    r_o, d_o = tiny2c_oracle.burn_in(r0, seed, burn)
    lam = tiny2c_oracle.lam()
    for st in range(10):
        res = ctx.run_steps(1, seed)
        r_o, _ = tiny2c_oracle.metropolis(r_o, seed, burn + st, 1, d_o)
        tau = oracle.tau_draws(seed, burn + st, n_tau, lam)
        want, absmean = tiny2c_oracle.eval_steps(r_o[None], tau[None], with_abs=True)
        _check_steps(np.array([res["last_step"]]), want, absmean)


def test_two_component_long_walk_matches_deterministic_energy():
    """P4 for the two-component variant on the GPU (soft tiny system)."""
    soft2c = synthetic.make_system("tiny", soft=True, two_component=True)
    e2 = mp2.mp2_energy(soft2c, mp2.spinor_eri(oracle.Oracle(soft2c)))
    ctx = pkg.Context(soft2c, 64, 2, pkg.MCMP2_FP64)
    ctx.set_walkers(synthetic.walker_positions(soft2c.centres, 1, 64, seed=11)[0], 4242, 500)
    res = ctx.run_steps(20000, 4242)
    z = (res["energy"] - e2) / res["error"]
    print(f"soft tiny 2c, FP64: E = {res['energy']:.6f} +- {res['error']:.6f}, E2 = {e2:.6f}, z = {z:.2f}")
    assert abs(z) < 3.0, (res["energy"], res["error"], e2)
    assert res["error"] < 0.05 * abs(e2)


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (33, 2), (70, 1)])
def test_two_component_tensor_forms_match_oracle_tiny(tiny2c, tiny2c_oracle, prec, m, n_tau):
    """32 x 32-pair tiles of 2 x 2 blocks (ragged: m = 33, 70 span two and three
    tile rows) within the error model of each form."""
    n = 2
    r = synthetic.walker_positions(tiny2c.centres, n, m, seed=500 + m)
    tau = synthetic.imaginary_times(tiny2c_oracle.lam(), n, n_tau, seed=19 + m)
    ctx = pkg.Context(tiny2c, m, n_tau, prec)
    got = ctx.eval_fixed(r, tau)
    want = tiny2c_oracle.eval_steps(r, tau)
    assert np.all(_steps_ok(tiny2c_oracle, r, tau, got, want, prec)), (got, want)


def test_two_component_spinor_units_with_an_odd_position_block_count(medium2c, medium2c_oracle):
    """m = 136: three 128-position blocks, so the spinor formation's second CTA pair
    owns a ragged block and a phantom one (two-component units: components 0, 1)."""
    m, n_tau = 136, 1
    r = synthetic.walker_positions(medium2c.centres, 1, m, seed=139)
    tau = synthetic.imaginary_times(medium2c_oracle.lam(), 1, n_tau, seed=140)
    ctx = pkg.Context(medium2c, m, n_tau, pkg.MCMP2_MIXED)
    got = ctx.eval_fixed(r, tau)
    want = medium2c_oracle.eval_steps(r, tau)
    assert np.all(_steps_ok(medium2c_oracle, r, tau, got, want)), (got, want)


def test_two_component_mixed_full_size_sampled_tiles(medium2c, medium2c_oracle):
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium2c.centres, 1, m, seed=71)
    tau = synthetic.imaginary_times(medium2c_oracle.lam(), 1, n_tau, seed=72)
    ctx = pkg.Context(medium2c, m, n_tau, pkg.MCMP2_MIXED)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    assert tp == 32
    nb = (m + tp - 1) // tp
    assert partials.shape[1] == nb * (nb + 1) // 2
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (0, 1), (5, 20), (nb - 1, nb - 1), (15, nb - 1)]:
        ps, qs = _tile_pairs(bp, bq, tp, m)
        vals = medium2c_oracle.eval_pairs(r[0], tau[0], ps, qs)
        want = vals.sum(axis=0)
        got = partials[:, _tile_index(bp, bq, nb)]
        assert np.all(_tile_ok(medium2c_oracle, r[0], tau[0], ps, qs, got, want)), (bp, bq, got, want)


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_two_component_tensor_forms_agree_with_fp64_within_a_fifth_of_sigma(medium2c, prec):
    m, n_tau, seed, n = 96, 2, 909, 400
    r0 = synthetic.walker_positions(medium2c.centres, 1, m, seed=4)[0]
    per = {}
    for pr in (pkg.MCMP2_FP64, prec):
        ctx = pkg.Context(medium2c, m, n_tau, pr)
        ctx.set_walkers(r0, seed, 100)
        per[pr] = np.array([ctx.run_steps(1, seed)["last_step"] for _ in range(n)])
        ctx.close()
    d = per[prec] - per[pkg.MCMP2_FP64]
    _, _, sb, nb = oracle.blocking(per[pkg.MCMP2_FP64])
    assert nb == 4
    assert abs(d.mean()) < 0.2 * sb, (d.mean(), sb)


def test_two_component_mixed_long_walk_matches_deterministic_energy():
    soft2c = synthetic.make_system("tiny", soft=True, two_component=True)
    e2 = mp2.mp2_energy(soft2c, mp2.spinor_eri(oracle.Oracle(soft2c)))
    ctx = pkg.Context(soft2c, 64, 2, pkg.MCMP2_MIXED)
    ctx.set_walkers(synthetic.walker_positions(soft2c.centres, 1, 64, seed=11)[0], 4242, 500)
    res = ctx.run_steps(20000, 4242)
    z = (res["energy"] - e2) / res["error"]
    print(f"soft tiny 2c, split BF16: E = {res['energy']:.6f} +- {res['error']:.6f}, E2 = {e2:.6f}, z = {z:.2f}")
    assert abs(z) < 3.0, (res["energy"], res["error"], e2)


def test_two_component_guards(tiny2c):
    mixed = pkg.Context(tiny2c, 8, 1, pkg.MCMP2_MIXED)
    with pytest.raises(pkg.McMp2Error) as e:
        mixed.set_interaction(pkg.MCMP2_GAUNT)
    assert e.value.code == pkg.MCMP2_EUNSUPPORTED
    ctx = pkg.Context(tiny2c, 8, 1, pkg.MCMP2_FP64)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.set_interaction(pkg.MCMP2_GAUNT)
    assert e.value.code == pkg.MCMP2_EUNSUPPORTED
    r = synthetic.walker_positions(tiny2c.centres, 1, 8, seed=1)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.backward(r, np.ones((1, 1)))
    assert e.value.code == pkg.MCMP2_EUNSUPPORTED
    # A checkpoint records that the system is two-component.
    ctx.set_walkers(r[0], 3, 10)
    blob = ctx.checkpoint()
    four = pkg.Context(dataclasses.replace(tiny2c, n_comp=4), 8, 1, pkg.MCMP2_FP64)
    with pytest.raises(pkg.McMp2Error):
        four.restore(blob)
