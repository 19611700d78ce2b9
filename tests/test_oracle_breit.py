"""Pins of the oracle's Gaunt and Breit integrands (CPU).

The interaction operator of Sec. II,
    g_ij = 1/r_ij - alpha(i).alpha(j) / (2 r_ij) - (alpha(i).r_ij)(alpha(j).r_ij) / (2 r_ij^3),
enters Eq. FinalMP2 through its two-electron integrals; the paper keeps only
the Coulomb term.  The oracle's trace form places each pair's operator at the
points where the propagators meet.  Pinned here against
  * the explicit sum over states at fixed points, with the transition
    densities rho^O_kl = phi_k^dag O phi_l written out (numpy, independent of
    the C code), for both the Gaunt and the full Breit operator;
  * the limit of zero small components, where alpha (which couples large
    and small components) drops out;
  * the symmetries of the integrand (pair swap -> complex conjugate; swapping
    the electrons of both pairs leaves it unchanged);
  * the deterministic Coulomb + Gaunt MP2 energy (Gaunt integrals from the
    Coulomb integrals of large x small function products), which a Monte
    Carlo walk must reproduce within 3 sigma on a system whose small
    components are of order one.
The gauge term has no deterministic integral here; its contraction pattern
is pinned pointwise only.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import mp2

PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def _alpha(v):
    """alpha . v in the component order (L-alpha, L-beta, S-alpha, S-beta)."""
    s = np.tensordot(np.asarray(v, dtype=np.complex128), PAULI, axes=1)
    out = np.zeros((4, 4), dtype=np.complex128)
    out[:2, 2:] = s
    out[2:, :2] = s
    return out


def _terms(ra, rb, interaction):
    """[(c, O)] with g(a,b) = (1/r_ab) sum c O(a) O(b)."""
    terms = [(1.0, np.eye(4, dtype=np.complex128))]
    if interaction >= 1:
        terms += [(-0.5, _alpha(e)) for e in np.eye(3)]
    if interaction >= 2:
        n = (np.asarray(ra) - np.asarray(rb)) / np.linalg.norm(np.asarray(ra) - np.asarray(rb))
        terms.append((-0.5, _alpha(n)))
    return terms


def _explicit_sum(orc, system, pts, tau, interaction):
    """-1/2 sum_AB c_A c_B sum_ijab e^{(ei+ej-ea-eb) tau} rho^A_ia(1) rho^A_jb(2)
    [rho^B_ai(3) rho^B_bj(4) - rho^B_bi(3) rho^B_aj(4)] times N_g^2/(g1 g2 g3 g4) e^{lambda tau}/lambda."""
    o = system.n_occ
    phis = [orc.spinors_at(p) for p in pts]
    e = system.eps
    occ, vir = slice(0, o), slice(o, None)
    D = e[occ][:, None, None, None] + e[occ][None, None, :, None] - e[vir][None, :, None, None] \
        - e[vir][None, None, None, :]
    W = np.exp(D * tau)
    F = 0.0
    for cA, OA in _terms(pts[0], pts[1], interaction):
        rA = [np.einsum("kc,cd,ld->kl", phis[x].conj(), OA, phis[x]) for x in (0, 1)]
        for cB, OB in _terms(pts[2], pts[3], interaction):
            rB = [np.einsum("kc,cd,ld->kl", phis[x].conj(), OB, phis[x]) for x in (2, 3)]
            ia1, jb2 = rA[0][occ, vir], rA[1][occ, vir]
            ai3, bj4 = rB[0][vir, occ], rB[1][vir, occ]
            N = np.einsum("ia,jb->iajb", ia1, jb2) * (np.einsum("ai,bj->iajb", ai3, bj4)
                                                       - np.einsum("bi,aj->iajb", ai3, bj4))
            F = F + cA * cB * (-0.5) * np.sum(W * N)
    g = [orc.g(p) for p in pts]
    lam = orc.lam()
    return F * orc.Ng() ** 2 / (g[0] * g[1] * g[2] * g[3]) * math.exp(lam * tau) / lam


def _four_points():
    return np.array([[0.1, 0.3, -0.2], [0.5, -0.4, 1.2], [-0.3, 0.2, 0.4], [0.2, 0.6, 1.7]])


@pytest.fixture(scope="module")
def strong():
    return synthetic.make_system("tiny", soft=True, small_scale=1.0)


@pytest.mark.parametrize("interaction", [1, 2])
@pytest.mark.parametrize("tau", [0.05, 0.7])
@pytest.mark.parametrize("which", ["tiny", "strong"])
def test_trace_form_equals_explicit_sum_with_interaction_terms(tiny, strong, interaction, tau, which):
    system = tiny if which == "tiny" else strong
    orc = oracle.Oracle(system, interaction=interaction)
    pts = _four_points()
    got = orc.pair_value(*pts, tau)
    want = _explicit_sum(orc, system, pts, tau, interaction)
    assert abs(got - want) <= 1e-11 * abs(want)
    # the interaction terms matter at this point (on the strong system by far)
    coulomb = oracle.Oracle(system).pair_value(*pts, tau)
    assert abs(got - coulomb) > (1e-3 if which == "strong" else 1e-9) * abs(coulomb)


def test_interaction_terms_vanish_without_small_components(tiny):
    nr = synthetic.nonrelativistic_variant(tiny)
    pts = _four_points()
    ref = oracle.Oracle(nr).pair_value(*pts, 0.3)
    for interaction in (1, 2):
        assert oracle.Oracle(nr, interaction=interaction).pair_value(*pts, 0.3) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("interaction", [1, 2])
def test_breit_integrand_symmetries(strong, interaction):
    orc = oracle.Oracle(strong, interaction=interaction)
    r1, r2, r3, r4 = _four_points()
    v = orc.pair_value(r1, r2, r3, r4, 0.4)
    assert orc.pair_value(r3, r4, r1, r2, 0.4) == pytest.approx(np.conj(v), rel=1e-12)
    assert orc.pair_value(r2, r1, r4, r3, 0.4) == pytest.approx(v, rel=1e-12)


def test_gaunt_integrals_are_hermitian_and_symmetric(strong):
    V = mp2.spinor_eri_gaunt(oracle.Oracle(strong))
    assert np.abs(V - V.transpose(1, 0, 3, 2).conj()).max() <= 1e-14 * np.abs(V).max()
    assert np.abs(V - V.transpose(2, 3, 0, 1)).max() <= 1e-12 * np.abs(V).max()


def test_gaunt_walk_matches_deterministic_gaunt_energy(strong):
    """P4 with the Coulomb + Gaunt interaction: the oracle's walk reproduces the
    sum-over-states energy within 3 sigma, and is far from the Coulomb-only one."""
    orc = oracle.Oracle(strong, interaction=1)
    e_gaunt = mp2.mp2_energy(strong, mp2.spinor_eri_gaunt(orc))
    e_coul = mp2.mp2_energy(strong, mp2.spinor_eri(orc))
    r0 = synthetic.walker_positions(strong.centres, 1, 16, seed=11)[0]
    means, errs = [], []
    for seed in range(4):
        res = orc.run(r0, 100 + seed, 300, 2000, 1)
        I, _, sb, _ = oracle.blocking(res["per_step"])
        means.append(I)
        errs.append(sb)
    mean = float(np.mean(means))
    err = float(np.sqrt(np.sum(np.square(errs)))) / len(errs)
    assert abs(mean - e_gaunt) < 3.0 * err, (mean, err, e_gaunt)
    assert abs(mean - e_coul) > 5.0 * err, (mean, err, e_coul)
