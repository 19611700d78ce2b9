"""The Gaunt and Breit interaction (Sec. II operator) in the FP64 form against the oracle.

Parity bar as for the Coulomb FP64 form: 1e-10 relative per step estimate (relative to
max(|I'_n|, 1e-3 <|f|>)).  Plus a walk on a system with order-one small components
against the deterministic Coulomb + Gaunt MP2 energy (P4 with the Gaunt term), and the
guards: the tensor-core forms and the adjoint keep the Coulomb operator, and checkpoints
record the interaction.
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import mp2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def strong():
    return synthetic.make_system("tiny", soft=True, small_scale=1.0)


def _ok(got, want, absmean):
    return np.abs(got - want) <= 1e-10 * np.maximum(np.abs(want), 1e-3 * absmean)


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


def test_guards_and_checkpoints(tiny):
    for prec in (pkg.MCMP2_MIXED, pkg.MCMP2_TF32):
        ctx = pkg.Context(tiny, 16, 1, prec)
        with pytest.raises(pkg.McMp2Error) as e:
            ctx.set_interaction(pkg.MCMP2_GAUNT)
        assert e.value.code == -7
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
