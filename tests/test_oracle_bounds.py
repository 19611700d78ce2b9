"""Pins of the error model (oracle/bounds.py) that the element-by-element GPU tests use.

1. The model's summands are the oracle's: oracle.eval_pairs (the C restatement of
   Eq. redundant's quotient, trace form of Eq. MCMP2, Sec. II operators) equals the
   PyTorch evaluation from scaled operands, Coulomb, Gaunt and Breit.
2. The model's standard deviation is the one a perturbation experiment measures:
   perturbing every operand X(x)_ck by independent normal errors of standard
   deviation s |X(x)_ck| in its real and imaginary parts moves each summand by a
   random amount whose empirical standard deviation over many draws matches the
   linearised sigma (a wrong derivative, a dropped operand or a mis-assembled
   variance fails this).
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import bounds


@pytest.fixture(scope="module")
def strong():
    return synthetic.make_system("tiny", soft=True, small_scale=1.0)


@pytest.mark.parametrize("interaction", [0, 1, 2])
def test_model_summands_are_the_oracle_pair_values(strong, interaction):
    orc = oracle.Oracle(strong, interaction=interaction)
    m = 24
    r = synthetic.walker_positions(strong.centres, 1, m, seed=71)[0]
    tau = synthetic.imaginary_times(orc.lam(), 1, 2, seed=72)[0]
    pairs = bounds.tile_pairs(0, 1, 16, m) + bounds.tile_pairs(0, 0, 16, m)[:20]
    want = orc.eval_pairs(r, tau, np.array([p for p, _ in pairs]), np.array([q for _, q in pairs]))
    vals, sig, epi = bounds.element_model(orc, r, tau, pairs, bounds.FP64, interaction)
    assert np.all(np.abs(vals - want) <= 1e-10 * np.abs(want) + bounds.KAPPA * sig + epi)
    assert np.median(np.abs(vals - want) / np.abs(want)) < 1e-13


def test_tile_pairs_enumerates_the_upper_triangle():
    assert bounds.tile_pairs(0, 0, 3, 10) == [(0, 1), (0, 2), (1, 2)]
    assert bounds.tile_pairs(1, 2, 2, 5) == [(2, 4), (3, 4)]
    assert len(bounds.tile_pairs(0, 1, 16, 20)) == 16 * 4


@pytest.mark.parametrize("interaction", [0, 2])
def test_model_sigma_matches_a_perturbation_experiment(strong, interaction):
    import torch

    orc = oracle.Oracle(strong, interaction=interaction)
    m = 12
    r = synthetic.walker_positions(strong.centres, 1, m, seed=81)[0]
    tau = synthetic.imaginary_times(orc.lam(), 1, 1, seed=82)[0]
    pairs = bounds.tile_pairs(0, 0, m, m)[:24]
    s = 1e-7
    form = bounds.Form(u_gemm=0.0, u_rep=s, u_acc=0.0, u_pack=0.0, u_epi=0.0)
    vals, sig, _ = bounds.element_model(orc, r, tau, pairs, form, interaction)
    ts = bounds.TileSetup(orc, r, pairs, interaction)
    X = ts.PH * ts.scales(tau[0])[None, None, :, None]
    rng = np.random.default_rng(5)
    draws = []
    with torch.no_grad():
        for _ in range(400):
            dX = s * np.abs(X) * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape))
            e, _, _ = bounds.summands(ts, torch.tensor(X + dX))
            draws.append(e.numpy() - vals[:, 0])
    emp = np.std(np.array(draws), axis=0)
    ratio = emp / sig[:, 0]
    # 400 draws: the empirical standard deviation is within ~4 % (one sigma) of the true one
    assert np.all((ratio > 0.8) & (ratio < 1.2)), ratio


def test_model_terms_add_for_the_forms(strong):
    """The TF32 operand rounding dominates split BF16, which dominates FP64."""
    orc = oracle.Oracle(strong)
    m = 10
    r = synthetic.walker_positions(strong.centres, 1, m, seed=91)[0]
    tau = synthetic.imaginary_times(orc.lam(), 1, 1, seed=92)[0]
    pairs = bounds.tile_pairs(0, 0, m, m)
    s = {f: bounds.element_model(orc, r, tau, pairs, form)[1] for f, form in
         (("fp64", bounds.FP64), ("bf16", bounds.BF16X3), ("tf32", bounds.TF32))}
    assert np.all(s["fp64"] < 1e-6 * s["bf16"]) and np.all(s["bf16"] < s["tf32"])


def test_sum_model_sigma_matches_a_perturbation_experiment(strong):
    """The standard deviation of a SUM of summands that share walker pairs: perturbing each
    position's operands once (shared by all its summands) moves the sum as sum_model says;
    adding the per-summand sigmas in quadrature would miss the correlation."""
    import torch

    orc = oracle.Oracle(strong, interaction=2)
    m = 10
    r = synthetic.walker_positions(strong.centres, 1, m, seed=83)[0]
    tau = synthetic.imaginary_times(orc.lam(), 1, 1, seed=84)[0]
    pairs = [(p, q) for p in range(m) for q in range(p + 1, m)]
    s = 1e-7
    form = bounds.Form(u_gemm=0.0, u_rep=s, u_acc=0.0, u_pack=0.0, u_epi=0.0)
    sig, _ = bounds.sum_model(orc, r, tau, pairs, form, 2)
    ts = bounds.TileSetup(orc, r, pairs, 2)
    XU = ts.PHU * ts.scales(tau[0])[None, None, :, None]
    rng = np.random.default_rng(6)
    with torch.no_grad():
        base = float(bounds.summands(ts, torch.tensor(np.stack([XU[ts.ip, 0], XU[ts.ip, 1], XU[ts.iq, 0],
                                                                XU[ts.iq, 1]])))[0].sum())
        draws = []
        for _ in range(400):
            Y = XU + s * np.abs(XU) * (rng.standard_normal(XU.shape) + 1j * rng.standard_normal(XU.shape))
            X = np.stack([Y[ts.ip, 0], Y[ts.ip, 1], Y[ts.iq, 0], Y[ts.iq, 1]])
            draws.append(float(bounds.summands(ts, torch.tensor(X))[0].sum()) - base)
    ratio = np.std(draws) / sig[0]
    assert 0.85 < ratio < 1.15, ratio
