"""The Gaunt and Breit interaction (Sec. II operator) against the oracle.

FP64 form: the parity bar of the Coulomb FP64 form, 1e-10 relative per step estimate
(relative to max(|I'_n|, 1e-3 <|f|>)).  Tensor-core forms (split BF16 x3 and TF32, the
operators applied to G- in the trace epilogue): the error model of each form
(oracle/bounds.py) with the operator traces, summed over the summands of a step or of a
tile (the per-summand comparison is in test_gpu_elements.py).  Plus a walk on a system
with order-one small components against the deterministic Coulomb + Gaunt MP2 energy (P4
with the Gaunt term), split BF16 against the FP64 form on one walk (within a fifth of
sigma-bar), and the guards: the adjoint keeps the Coulomb operator, two-component systems
have no small components for it, and checkpoints record the interaction.
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import bounds, mp2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def strong():
    return synthetic.make_system("tiny", soft=True, small_scale=1.0)


def _ok(got, want, absmean):
    return np.abs(got - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3 * absmean)


FORMS = {pkg.MCMP2_MIXED: bounds.BF16X3, pkg.MCMP2_TF32: bounds.TF32}


def _steps_tol(orc, r, tau, prec, interaction):
    """Tolerance of each replayed step estimate: the error model of the form with the operators."""
    return bounds.steps_tolerance(orc, r, tau, FORMS[prec], interaction)


@pytest.mark.parametrize("interaction", [pkg.MCMP2_GAUNT, pkg.MCMP2_BREIT])
@pytest.mark.parametrize("m,n_tau", [(16, 1), (13, 3), (2, 1), (33, 2)])
@pytest.mark.parametrize("which", ["tiny", "strong"])
def test_interaction_replay_matches_oracle(tiny, strong, interaction, m, n_tau, which):
    system = tiny if which == "tiny" else strong
    orc = oracle.Oracle(system, interaction=interaction)
    n = 2
    r = synthetic.walker_positions(system.centres, n, m, seed=300 + m)
    tau = synthetic.imaginary_times(orc.lam(), n, n_tau, seed=7 + m)
    ctx = pkg.Context(system, m, n_tau, pkg.MCMP2_FP64)
    ctx.set_interaction(interaction)
    got = ctx.eval_fixed(r, tau)
    want, absmean = orc.eval_steps(r, tau, with_abs=True)
    assert np.all(_ok(got, want, absmean)), (got, want)
    # and the interaction changes the estimate (by far on the strong system)
    ctx.set_interaction(pkg.MCMP2_COULOMB)
    coul = ctx.eval_fixed(r, tau)
    assert np.all(np.abs(coul - got) > (1e-3 if which == "strong" else 1e-12) * np.abs(got))


def test_breit_replay_medium_system():
    medium = synthetic.make_system("medium")
    orc = oracle.Oracle(medium, interaction=pkg.MCMP2_BREIT)
    m, n_tau = 24, 2
    r = synthetic.walker_positions(medium.centres, 1, m, seed=61)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=62)
    ctx = pkg.Context(medium, m, n_tau, pkg.MCMP2_FP64)
    ctx.set_interaction(pkg.MCMP2_BREIT)
    got = ctx.eval_fixed(r, tau)
    want, absmean = orc.eval_steps(r, tau, with_abs=True)
    assert np.all(_ok(got, want, absmean)), (got, want)


def test_gaunt_walk_matches_deterministic_gaunt_energy(strong):
    orc = oracle.Oracle(strong, interaction=pkg.MCMP2_GAUNT)
    e_gaunt = mp2.mp2_energy(strong, mp2.spinor_eri_gaunt(orc))
    e_coul = mp2.mp2_energy(strong, mp2.spinor_eri(orc))
    ctx = pkg.Context(strong, 64, 2, pkg.MCMP2_FP64)
    ctx.set_interaction(pkg.MCMP2_GAUNT)
    ctx.set_walkers(synthetic.walker_positions(strong.centres, 1, 64, seed=11)[0], 4243, 500)
    res = ctx.run_steps(20000, 4243)
    z = (res["energy"] - e_gaunt) / res["error"]
    print(f"strong small components, Gaunt: E = {res['energy']:.6f} +- {res['error']:.6f}, "
          f"E2(Gaunt) = {e_gaunt:.6f}, E2(Coulomb) = {e_coul:.6f}, z = {z:.2f}")
    assert abs(z) < 3.0
    assert abs(res["energy"] - e_coul) > 5.0 * res["error"]


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
@pytest.mark.parametrize("interaction", [pkg.MCMP2_GAUNT, pkg.MCMP2_BREIT])
@pytest.mark.parametrize("m,n_tau", [(16, 1), (33, 2), (2, 1)])
@pytest.mark.parametrize("which", ["tiny", "strong"])
def test_interaction_tensor_forms_match_oracle(tiny, strong, prec, interaction, m, n_tau, which):
    """Operator terms in the tensor-core trace epilogue: 1, 3 and 1 (ragged) 16-pair blocks."""
    system = tiny if which == "tiny" else strong
    orc = oracle.Oracle(system, interaction=interaction)
    n = 2
    r = synthetic.walker_positions(system.centres, n, m, seed=500 + m)
    tau = synthetic.imaginary_times(orc.lam(), n, n_tau, seed=17 + m)
    ctx = pkg.Context(system, m, n_tau, prec)
    ctx.set_interaction(interaction)
    got = ctx.eval_fixed(r, tau)
    want = orc.eval_steps(r, tau)
    tol = _steps_tol(orc, r, tau, prec, interaction)
    assert np.all(np.abs(got - want) <= tol), (got, want, tol)
    if which == "strong" and m > 2 and prec == pkg.MCMP2_MIXED:
        # the operator terms move the estimate by far more than the split BF16 tolerance
        ctx.set_interaction(pkg.MCMP2_COULOMB)
        coul = ctx.eval_fixed(r, tau)
        assert np.all(np.abs(coul - got) > 10.0 * tol), (coul, got, tol)


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_breit_tensor_forms_medium_system(prec):
    medium = synthetic.make_system("medium")
    orc = oracle.Oracle(medium, interaction=pkg.MCMP2_BREIT)
    m, n_tau = 40, 2
    r = synthetic.walker_positions(medium.centres, 1, m, seed=71)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=72)
    ctx = pkg.Context(medium, m, n_tau, prec)
    ctx.set_interaction(pkg.MCMP2_BREIT)
    got = ctx.eval_fixed(r, tau)
    want = orc.eval_steps(r, tau)
    assert np.all(np.abs(got - want) <= _steps_tol(orc, r, tau, prec, pkg.MCMP2_BREIT)), (got, want)


@pytest.mark.parametrize("prec,interaction", [(pkg.MCMP2_MIXED, pkg.MCMP2_BREIT), (pkg.MCMP2_MIXED, pkg.MCMP2_GAUNT),
                                              (pkg.MCMP2_TF32, pkg.MCMP2_BREIT)])
def test_interaction_full_size_sampled_tiles(prec, interaction):
    """The bench launch (m = 1024 walker pairs, 4 times) with the operator terms: sampled
    16 x 16 tiles of the tensor-core forms against the oracle."""
    medium = synthetic.make_system("medium")
    orc = oracle.Oracle(medium, interaction=interaction)
    m, n_tau = 1024, 4
    r = synthetic.walker_positions(medium.centres, 1, m, seed=81)
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=82)
    ctx = pkg.Context(medium, m, n_tau, prec)
    ctx.set_interaction(interaction)
    step = ctx.eval_fixed(r, tau)[0]
    partials, tp = ctx.debug_partials()
    assert tp == 16
    nb = (m + tp - 1) // tp
    assert step == pytest.approx(partials.sum() / (m * (m - 1) / 2) / n_tau, rel=1e-12)
    for bp, bq in [(0, 0), (9, 50), (nb - 1, nb - 1), (31, nb - 1)]:
        pairs = [(bp * tp + i, bq * tp + j) for i in range(tp) for j in range(tp)
                 if bp * tp + i < m and bq * tp + j < m and (bp < bq or i < j)]
        ps, qs = np.array([p for p, _ in pairs]), np.array([q for _, q in pairs])
        vals = orc.eval_pairs(r[0], tau[0], ps, qs)
        want = vals.sum(axis=0)
        k = sum(nb - b for b in range(bp)) + (bq - bp)
        tol = bounds.tile_tolerance(orc, r[0], tau[0], pairs, FORMS[prec], interaction)
        assert np.all(np.abs(partials[:, k] - want) <= tol), (bp, bq, partials[:, k], want, tol)


def test_breit_split_bf16_agrees_with_fp64_form_within_a_fifth_of_sigma(strong):
    """Same walk (FP64 sampling in both forms) with the Breit terms on the system with
    order-one small components: the mean difference of the split BF16 and FP64 step
    estimates is far below 0.2 sigma-bar of the FP64 run."""
    m, n_tau, seed, n = 64, 2, 909, 400
    r0 = synthetic.walker_positions(strong.centres, 1, m, seed=5)[0]
    per = {}
    for prec in (pkg.MCMP2_FP64, pkg.MCMP2_MIXED):
        ctx = pkg.Context(strong, m, n_tau, prec)
        ctx.set_interaction(pkg.MCMP2_BREIT)
        ctx.set_walkers(r0, seed, 100)
        per[prec] = np.array([ctx.run_steps(1, seed)["last_step"] for _ in range(n)])
        ctx.close()
    d = per[pkg.MCMP2_MIXED] - per[pkg.MCMP2_FP64]
    I, s2, sb, nb = oracle.blocking(per[pkg.MCMP2_FP64])
    assert nb == 4
    assert abs(d.mean()) < 0.2 * sb, (d.mean(), sb)


def test_guards_and_checkpoints(tiny):
    for prec in (pkg.MCMP2_MIXED, pkg.MCMP2_TF32):  # the tensor-core forms take every interaction
        ctx = pkg.Context(tiny, 16, 1, prec)
        ctx.set_interaction(pkg.MCMP2_GAUNT)
        ctx.set_interaction(pkg.MCMP2_BREIT)
        ctx.set_interaction(pkg.MCMP2_COULOMB)
    ctx = pkg.Context(tiny, 16, 1, pkg.MCMP2_FP64)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.set_interaction(3)
    assert e.value.code == -1
    ctx.set_interaction(pkg.MCMP2_BREIT)
    r = synthetic.walker_positions(tiny.centres, 1, 16, seed=3)
    tau = synthetic.imaginary_times(2.0, 1, 1, seed=4)
    with pytest.raises(pkg.McMp2Error) as e:
        ctx.backward(r, tau)
    assert e.value.code == -7
    ctx.set_walkers(r[0], 5, 20)
    ctx.run_steps(30, 5)
    blob = ctx.checkpoint()
    a = ctx.run_steps(40, 5)
    other = pkg.Context(tiny, 16, 1, pkg.MCMP2_FP64)
    with pytest.raises(pkg.McMp2Error):
        other.restore(blob)  # Coulomb context: another integrand
    other.set_interaction(pkg.MCMP2_BREIT)
    other.restore(blob)
    assert other.run_steps(40, 5) == a
