"""The TF32 tensor-core form against the oracle and the FP64 form.

Tolerance derived from the arithmetic of the form: the spinor values come
from the split BF16 x3 products (~2^-16), are scaled and rounded to the
nearest TF32 value (relative error <= 2^-11 per operand), and every
propagator entry G(x, y)_cd = sum_k X(x)_ck conj(X(y)_dk) is accumulated in
FP32 from products of two such operands, so
    |delta G_cd| <= 2 u |G|_cd,  u = 2^-11 + 2^-16,
with |G|_cd = sum_k |X(x)_ck| |X(y)_dk| the absolute expansion.  A pair-of-
pairs term -1/2 T(1p,1q) T(2p,2q) + 1/2 tr[G- G+ G- G+] is a sum of products
of four propagator entries, so its error is at most 8 u times the same
expression built from absolute expansions (|f|_pq below), times a_p a_q / lambda.
The step estimate is compared with that bound summed over its terms
(plus the FP32 accumulation, far smaller).
"""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu

U_TF32 = 2.0 ** -11 + 2.0 ** -16


def _abs_expansion_sum(orc, system, r_step, tau_step, pairs=None):
    """Sum over the step's pair-of-pairs terms (or the given (p, q) list) and times of
    |f|_pq a_p a_q / lambda, with every propagator entry replaced by its absolute expansion."""
    m = r_step.shape[0]
    n_occ = system.n_occ
    eps = np.asarray(system.eps)
    e_h, e_l = eps[:n_occ].max(), eps[n_occ:].min()
    lam = 2.0 * (e_l - e_h)
    ng = orc.Ng()
    if pairs is None:
        pairs = [(p, q) for p in range(m) for q in range(p + 1, m)]
    phi = np.zeros((m, 2, orc.n_orb, 4), dtype=np.complex128)
    a = np.zeros(m)
    for p in sorted({i for pq in pairs for i in pq}):
        for e in range(2):
            phi[p, e] = orc.spinors_at(r_step[p, e])
        a[p] = ng / (orc.g(r_step[p, 0]) * orc.g(r_step[p, 1]))
    total = np.zeros(len(tau_step))
    for t, tau in enumerate(tau_step):
        s_occ = np.exp((eps[:n_occ] - e_h) * tau / 2.0)
        s_vir = np.exp(-(eps[n_occ:] - e_l) * tau / 2.0)
        xo = np.abs(phi[:, :, :n_occ, :]) * s_occ[None, None, :, None]  # |X-| [m][e][i][c]
        xv = np.abs(phi[:, :, n_occ:, :]) * s_vir[None, None, :, None]  # |X+| [m][e][a][c]
        for p, q in pairs:
            gm = {(e, f): xo[p, e].T @ xo[q, f] for e in range(2) for f in range(2)}  # [c][d]
            gp = {(e, f): xv[p, e].T @ xv[q, f] for e in range(2) for f in range(2)}
            t1 = np.sum(gm[0, 0] * gp[0, 0])
            t2 = np.sum(gm[1, 1] * gp[1, 1])
            # tr[G-(1q,1p) G+(1p,2q) G-(2q,2p) G+(2p,1q)] with absolute entries
            x = np.trace(gm[0, 0].T @ gp[0, 1] @ gm[1, 1].T @ gp[1, 0])
            total[t] += (0.5 * t1 * t2 + 0.5 * x) * a[p] * a[q] / lam
    return total


def _bound(orc, system, r_step, tau_step):
    m = r_step.shape[0]
    n_pairs = m * (m - 1) // 2
    return 8.0 * U_TF32 * _abs_expansion_sum(orc, system, r_step, tau_step).sum() / (n_pairs * len(tau_step))


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
    per-pair values, each tile's partial sum within 8u times the tile's absolute expansion."""
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
        bound = 8.0 * U_TF32 * _abs_expansion_sum(orc, medium, r[0][: max(ps.max(), qs.max()) + 1], tau[0], pairs)
        k = sum(nb - b for b in range(bp)) + (bq - bp)
        got = partials[:, k]
        assert np.all(np.abs(got - want) <= bound), (bp, bq, got, want, bound)
