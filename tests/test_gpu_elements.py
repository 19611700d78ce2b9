"""Every summand of sampled tiles of the full-size launch against the oracle, one by one.

The summand of Eq. redundant -- Re f/(w w w) for one pair of walker pairs (p, q)
and one imaginary time, f the trace form of Eq. MCMP2 (reading R1) with the
interaction of Sec. II -- is recorded by mcmp2_debug_elements for whole tiles of
the launch the benchmark times (medium system, m = 1024 walker pairs, 4 times per
step) and compared with oracle.eval_pairs element by element.  Tolerances
(oracle/bounds.py, first-order probabilistic error model of each form, sigma per
element from exact derivatives of the summand):
  FP64 form:      |got - want| <= 1e-10 |want| + KAPPA sigma_FP64 + epi
  split BF16 x3:  |got - want| <= KAPPA sigma_BF16x3 + epi
  TF32:           |got - want| <= KAPPA sigma_TF32 + epi
(KAPPA = 8; epi: the FP32 trace arithmetic).  The observed max |got - want| / sigma
is printed.  Plus the separations that make the operator terms visible at that
tolerance: on a system with order-one small components the Gaunt summands differ
from the Coulomb ones, and the full Breit summands from the Gaunt ones, by more
than ten times the tolerance summed over the tile, in both tensor-core forms.
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import bounds

pytestmark = pytest.mark.gpu

FORMS = {pkg.MCMP2_FP64: bounds.FP64, pkg.MCMP2_MIXED: bounds.BF16X3, pkg.MCMP2_TF32: bounds.TF32}
NAMES = {pkg.MCMP2_FP64: "fp64", pkg.MCMP2_MIXED: "bf16x3", pkg.MCMP2_TF32: "tf32"}
INTER = {pkg.MCMP2_COULOMB: "coulomb", pkg.MCMP2_GAUNT: "gaunt", pkg.MCMP2_BREIT: "breit"}


@pytest.fixture(scope="module")
def medium():
    return synthetic.make_system("medium")


@pytest.fixture(scope="module")
def medium_2c():
    return synthetic.make_system("medium", two_component=True)


def _check_tiles(system, prec, interaction, m, n_tau, tiles_of, seed):
    orc = oracle.Oracle(system, interaction=interaction)
    r = synthetic.walker_positions(system.centres, 1, m, seed=seed)[0]
    tau = synthetic.imaginary_times(orc.lam(), 1, n_tau, seed=seed + 1)[0]
    ctx = pkg.Context(system, m, n_tau, prec)
    if interaction != pkg.MCMP2_COULOMB:
        ctx.set_interaction(interaction)
    tp = ctx.tile_pairs()
    nb = (m + tp - 1) // tp
    worst = 0.0
    for bp, bq in tiles_of(nb):
        got, step, tp_ = ctx.debug_elements(r, tau, bp, bq)
        assert tp_ == tp and np.isfinite(step)
        pairs = bounds.tile_pairs(bp, bq, tp, m)
        ii = np.array([p - bp * tp for p, _ in pairs])
        jj = np.array([q - bq * tp for _, q in pairs])
        g = got[:, ii, jj].T  # [pairs][n_tau]
        want = orc.eval_pairs(r, tau, np.array([p for p, _ in pairs]), np.array([q for _, q in pairs]))
        _, sig, epi = bounds.element_model(orc, r, tau, pairs, FORMS[prec], interaction)
        tol = bounds.KAPPA * sig + epi + (1e-10 * np.abs(want) if prec == pkg.MCMP2_FP64 else 0.0)
        d = np.abs(g - want)
        bad = d > tol
        assert not bad.any(), (bp, bq, np.argwhere(bad)[:5], g[bad][:5], want[bad][:5], tol[bad][:5])
        # every entry outside p < q < m is exactly zero
        mask = np.ones((tp, tp), dtype=bool)
        mask[ii, jj] = False
        assert np.all(got[:, mask] == 0.0)
        worst = max(worst, float(np.max(d / (sig + 1e-300))))
    print(f"{system.name} {NAMES[prec]} {INTER[interaction]} m={m}: max |got - want| / sigma = {worst:.3g}")
    return worst


@pytest.mark.parametrize("interaction", [pkg.MCMP2_COULOMB, pkg.MCMP2_GAUNT, pkg.MCMP2_BREIT])
@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_every_summand_of_sampled_full_size_tiles(medium, prec, interaction):
    """m = 1024, 4 times (the benchmark's launch): a diagonal tile, an interior one, the last."""
    _check_tiles(medium, prec, interaction, 1024, 4, lambda nb: [(0, 0), (7, nb // 2 + 3), (nb - 1, nb - 1)], 51)


@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_every_summand_two_component(medium_2c, prec):
    """Two-component spinors (2 x 2 blocks; 32-pair tiles in the tensor-core forms)."""
    _check_tiles(medium_2c, prec, pkg.MCMP2_COULOMB, 1024, 4, lambda nb: [(0, 0), (3, nb // 2 + 4), (nb - 1, nb - 1)],
                 53)


@pytest.mark.parametrize("prec", [pkg.MCMP2_FP64, pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_every_summand_ragged_launch(medium, prec):
    """m = 1000 walker pairs: the last tile row and column are ragged (zeros past m)."""
    _check_tiles(medium, prec, pkg.MCMP2_COULOMB, 1000, 3, lambda nb: [(0, nb - 1), (nb - 1, nb - 1)], 57)


@pytest.mark.parametrize("prec", [pkg.MCMP2_MIXED, pkg.MCMP2_TF32])
def test_operator_terms_exceed_the_tolerance(prec):
    """Order-one small components: Gaunt - Coulomb and Breit - Gaunt, summed over two
    16 x 16 tiles, each exceed ten times the summed element tolerance."""
    strong = synthetic.make_system("tiny", soft=True, small_scale=1.0)
    m, n_tau = 64, 2
    r = synthetic.walker_positions(strong.centres, 1, m, seed=31)[0]
    tau = synthetic.imaginary_times(oracle.Oracle(strong).lam(), 1, n_tau, seed=32)[0]
    ctx = pkg.Context(strong, m, n_tau, prec)
    tiles = [(0, 1), (1, 1)]
    got, tol = {}, {}
    for inter in (pkg.MCMP2_COULOMB, pkg.MCMP2_GAUNT, pkg.MCMP2_BREIT):
        ctx.set_interaction(inter)
        orc = oracle.Oracle(strong, interaction=inter)
        vals, tols = [], []
        for bp, bq in tiles:
            el, _, tp = ctx.debug_elements(r, tau, bp, bq)
            pairs = bounds.tile_pairs(bp, bq, tp, m)
            ii = np.array([p - bp * tp for p, _ in pairs])
            jj = np.array([q - bq * tp for _, q in pairs])
            vals.append(el[:, ii, jj].T)
            want, sig, epi = bounds.element_model(orc, r, tau, pairs, FORMS[prec], inter)
            tols.append(bounds.KAPPA * sig + epi)
            assert np.all(np.abs(el[:, ii, jj].T - orc.eval_pairs(r, tau, np.array([p for p, _ in pairs]),
                                                                  np.array([q for _, q in pairs])))
                          <= tols[-1])
        got[inter], tol[inter] = np.concatenate(vals), np.concatenate(tols)
    for a, b in ((pkg.MCMP2_GAUNT, pkg.MCMP2_COULOMB), (pkg.MCMP2_BREIT, pkg.MCMP2_GAUNT)):
        sep = np.abs(got[a] - got[b]).sum() / tol[a].sum()
        print(f"{NAMES[prec]} {INTER[a]} - {INTER[b]}: summed |difference| = {sep:.1f} x summed tolerance")
        assert sep > 10.0
