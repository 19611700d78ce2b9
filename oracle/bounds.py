"""Error model of the GPU forms for element-by-element checks -- TEST INFRASTRUCTURE ONLY.

The summand of Eq. redundant for one pair of walker pairs (p, q) and one
imaginary time is, in the trace form of Eq. MCMP2 with the exponential shifts
of the propagators (so that exp(lambda tau) / lambda becomes 1 / lambda),

    e = Re{ -1/2 sum_AB c_A c_B ( tr[G-31 O_A G+13 O_B] tr[G-42 O_A G+24 O_B]
                                  - tr[G-31 O_A G+14 O_B G-42 O_A G+23 O_B] ) } a_p a_q / lambda,

with G-(x,y)_cd = sum_i X(x)_ci conj(X(y)_di) over the occupied spinors scaled by
exp((eps_i - eps_HOMO) tau / 2), G+ likewise over the virtual ones scaled by
exp(-(eps_a - eps_LUMO) tau / 2), points 1, 2 of pair p and 3, 4 of pair q, and
the operators O of the interaction of Sec. II (O_0 = 1, c_0 = 1 only, for the
Coulomb operator).

A worst-case bound (every rounding error aligned) is useless here: the orbital
sums of each propagator entry cancel, so the absolute expansion of a summand
(every number replaced by its modulus) is typically 10^4 - 10^5 times the
summand.  The model used instead is first-order probabilistic error analysis
(independent rounding errors add in quadrature):

 * each scaled operand X(x)_ck carries an error of standard deviation
       s(x)_ck = sqrt( (u_gemm n(x)_ck)^2 + (u_rep |X(x)_ck|)^2 ),
   n(x)_ck = s_k(tau) sqrt(sum_P |U_cPk|^2 f_P(x)^2) the 2-norm of the terms of
   the spinor formation phi^c_k = sum_P U_cPk f_P (f = g_mu and its
   gradients, U = C folded with the Pauli matrices), u_gemm the relative
   error of one of those terms and u_rep the relative error with which the
   contraction's operands represent X;
 * every propagator entry adds u_acc times the 2-norm of its terms (FP32
   accumulation), and the G- entries parked as 24-bit floats add u_pack |G-|;
 * the summand's error then has standard deviation
       sigma^2 = sum |de/dX|^2 s^2 + sum_entries |de/dG|^2 (u_acc ||terms||_2)^2
                 + sum_{G- entries} |de/dG-|^2 (u_pack |G-|)^2,
   the derivatives taken exactly (PyTorch CPU autograd in complex128);
 * the FP32 trace arithmetic of the epilogue adds at most
   u_epi sum_AB |c_A c_B| (|direct| + |exchange|) a_p a_q / lambda.

A test then accepts |got - want| <= KAPPA sigma + epilogue term.  For a sum of
summands (a step estimate, a tile's partial sum) the operand errors of a walker
pair's positions are shared by every summand using the pair, so the sum is
linearised as a whole (sum_model).  Only the test suite and the smoke check use
this module.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import mp2

KAPPA = 8.0  # accepted multiple of the model's standard deviation


@dataclasses.dataclass(frozen=True)
class Form:
    """Relative error parameters of one arithmetic form (see the module docstring)."""
    u_gemm: float
    u_rep: float
    u_acc: float
    u_pack: float
    u_epi: float


# FP64 form: DFMA everywhere (a few units of 2^-53 per term, basis values from
# the device's exp), no packing, FP64 traces.
FP64 = Form(u_gemm=2.0 ** -50, u_rep=2.0 ** -50, u_acc=2.0 ** -50, u_pack=0.0, u_epi=2.0 ** -48)
# Split BF16 x3: FP32 basis values and coefficients split hi + lo (each ~2^-18), the
# dropped lo*lo product (~2^-18), FP32 accumulation; the same split for the
# contraction's operands; G- parked with 15 stored significand bits.
BF16X3 = Form(u_gemm=2.0 ** -17, u_rep=2.0 ** -17, u_acc=2.0 ** -24, u_pack=2.0 ** -16, u_epi=2.0 ** -20)
# TF32: the split-BF16 spinor formation, then operands rounded to nearest TF32 (2^-11).
TF32 = Form(u_gemm=2.0 ** -17, u_rep=2.0 ** -11, u_acc=2.0 ** -24, u_pack=2.0 ** -16, u_epi=2.0 ** -20)

_SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def _operators(n_vec, interaction):
    """O_A (4 x 4) and c_A of the interaction at a pair with unit vector n (Sec. II)."""
    ops = [np.eye(4, dtype=np.complex128)]
    cs = [1.0]
    if interaction >= 1:
        blocks = [_SIGMA[k] for k in range(3)]
        if interaction >= 2:
            blocks.append(np.tensordot(n_vec, _SIGMA, axes=1))
        for b in blocks:
            o = np.zeros((4, 4), dtype=np.complex128)
            o[:2, 2:] = b
            o[2:, :2] = b
            ops.append(o)
            cs.append(-0.5)
    return np.array(ops), np.array(cs)


def tile_pairs(bp: int, bq: int, tp: int, m: int):
    """(p, q) with p < q < m of the tile (bp, bq) of tp x tp walker pairs, row-major over (i, j)."""
    out = []
    for i in range(tp):
        for j in range(tp):
            p, q = bp * tp + i, bq * tp + j
            if p < m and q < m and p < q:
                out.append((p, q))
    return out


def _point_data(orc, U, r):
    """Spinor values phi [n_orb][4] and the 2-norms n [n_orb][4] of their formation terms at r."""
    phi = orc.spinors_at(r)
    v, g = orc.basis_at(r)
    f = np.zeros(4 * len(v))
    f[0::4] = v
    f[1::4] = g[:, 0]
    f[2::4] = g[:, 1]
    f[3::4] = g[:, 2]
    nrm = np.sqrt(np.einsum("cpk,p->kc", np.abs(U) ** 2, f ** 2))
    return phi, nrm


class TileSetup:
    """Spinor values, formation norms, weights and operators of the listed summands."""

    def __init__(self, orc, r_step, pairs, interaction: int = 0):
        system = orc.system
        self.n_occ = system.n_occ
        self.eps = np.asarray(system.eps)
        self.e_h, self.e_l = self.eps[:self.n_occ].max(), self.eps[self.n_occ:].min()
        lam = 2.0 * (self.e_l - self.e_h)
        ng = orc.Ng()
        U = mp2.real_function_coefficients(system)
        idx = sorted({i for pq in pairs for i in pq})
        phi, nrm, a, unit = {}, {}, {}, {}
        for p in idx:
            d0 = _point_data(orc, U, r_step[p, 0])
            d1 = _point_data(orc, U, r_step[p, 1])
            phi[p] = (d0[0], d1[0])
            nrm[p] = (d0[1], d1[1])
            a[p] = ng / (orc.g(r_step[p, 0]) * orc.g(r_step[p, 1]))
            d = np.asarray(r_step[p, 0]) - np.asarray(r_step[p, 1])
            unit[p] = d / np.linalg.norm(d)
        P = np.array([p for p, _ in pairs])
        Q = np.array([q for _, q in pairs])
        # Points 1, 2 (pair p) and 3, 4 (pair q): [4][B][n_orb][4]
        self.PH = np.stack([np.stack([phi[p][0] for p in P]), np.stack([phi[p][1] for p in P]),
                            np.stack([phi[q][0] for q in Q]), np.stack([phi[q][1] for q in Q])])
        self.NR = np.stack([np.stack([nrm[p][0] for p in P]), np.stack([nrm[p][1] for p in P]),
                            np.stack([nrm[q][0] for q in Q]), np.stack([nrm[q][1] for q in Q])])
        # The same per walker pair (positions shared by several summands): [U][2][n_orb][4]
        # and each summand's (p, q) as indices into it.
        where = {p: i for i, p in enumerate(idx)}
        self.PHU = np.stack([np.stack(phi[p]) for p in idx])
        self.NRU = np.stack([np.stack(nrm[p]) for p in idx])
        self.ip = np.array([where[p] for p in P])
        self.iq = np.array([where[q] for q in Q])
        self.w = np.array([a[p] * a[q] / lam for p, q in pairs])
        self.OA = np.stack([_operators(unit[p], interaction)[0] for p in P])  # [B][nA][4][4]
        self.OB = np.stack([_operators(unit[q], interaction)[0] for q in Q])
        cA = _operators(unit[P[0]], interaction)[1]
        self.CC = np.outer(cA, cA)

    def scales(self, tau):
        n = self.n_occ
        return np.concatenate([np.exp((self.eps[:n] - self.e_h) * tau / 2.0),
                               np.exp(-(self.eps[n:] - self.e_l) * tau / 2.0)])


def summands(ts: TileSetup, X, keep_graph: bool = False):
    """The summands e (torch, [B]) from scaled operands X [4][B][n_orb][4] (a complex128
    tensor), plus the propagator blocks and the direct / exchange traces."""
    import torch

    o = slice(0, ts.n_occ)
    v = slice(ts.n_occ, None)
    OAt, OBt = torch.tensor(ts.OA), torch.tensor(ts.OB)
    CC = torch.tensor(ts.CC)

    def green(x, y, ks):  # G(x, y)_cd = sum_k X(x)_kc conj(X(y)_kd), batched
        return torch.einsum("bkc,bkd->bcd", X[x][:, ks], X[y][:, ks].conj())

    G = {"m31": green(2, 0, o), "m42": green(3, 1, o), "p13": green(0, 2, v), "p24": green(1, 3, v),
         "p14": green(0, 3, v), "p23": green(1, 2, v)}
    if keep_graph:
        for g in G.values():
            g.retain_grad()

    def tr2(g1, g2):  # tr[G O_A G' O_B] for every (A, B): [B][nA][nB]
        return torch.einsum("bcd,bade,bef,bgfc->bag", g1, OAt, g2, OBt)

    d1 = tr2(G["m31"], G["p13"])
    d2 = tr2(G["m42"], G["p24"])
    x = torch.einsum("bcd,bade,bef,bgfh,bhi,baij,bjk,bgkc->bag", G["m31"], OAt, G["p14"], OBt, G["m42"], OAt,
                     G["p23"], OBt)
    direct = (CC[None] * d1 * d2).sum(dim=(1, 2))
    exch = (CC[None] * x).sum(dim=(1, 2))
    e = (-0.5 * (direct - exch)).real * torch.tensor(ts.w)
    mag = ((CC.abs()[None] * (d1 * d2).abs()).sum(dim=(1, 2)) + (CC.abs()[None] * x.abs()).sum(dim=(1, 2)))
    return e, G, mag * torch.tensor(ts.w)


def element_model(orc, r_step, tau_step, pairs, form: Form, interaction: int = 0):
    """(values, sigma, epi) of the listed summands, arrays [len(pairs)][n_tau]:
    the summands in FP64 (the same quantity oracle.eval_pairs returns), the model's
    standard deviation of a form's error in them, and the epilogue term."""
    import torch

    ts = TileSetup(orc, r_step, pairs, interaction)
    n_occ = ts.n_occ
    vals = np.zeros((len(pairs), len(tau_step)))
    sig = np.zeros_like(vals)
    epi = np.zeros_like(vals)
    for t, tau in enumerate(tau_step):
        s = ts.scales(tau)[None, None, :, None]
        X = ts.PH * s
        SX = np.sqrt((form.u_gemm * ts.NR * s) ** 2 + (form.u_rep * np.abs(X)) ** 2)
        Xt = torch.tensor(X, requires_grad=True)
        e, G, mag = summands(ts, Xt, keep_graph=True)
        e.sum().backward()
        var = ((Xt.grad.abs().numpy() * SX) ** 2).sum(axis=(0, 2, 3))
        for key, g in G.items():
            ks = slice(0, n_occ) if key[0] == "m" else slice(n_occ, None)
            x, y = {"m31": (2, 0), "m42": (3, 1), "p13": (0, 2), "p24": (1, 3), "p14": (0, 3), "p23": (1, 2)}[key]
            norm2 = np.sqrt(np.einsum("bkc,bkd->bcd", np.abs(X[x][:, ks]) ** 2, np.abs(X[y][:, ks]) ** 2))
            gg = g.grad.abs().numpy()
            var += ((gg * form.u_acc * norm2) ** 2).sum(axis=(1, 2))
            if key[0] == "m":
                var += ((gg * form.u_pack * np.abs(g.detach().numpy())) ** 2).sum(axis=(1, 2))
        vals[:, t] = e.detach().numpy()
        sig[:, t] = np.sqrt(var)
        epi[:, t] = form.u_epi * mag.detach().numpy()
    return vals, sig, epi


def sum_model(orc, r_step, tau_step, pairs, form: Form, interaction: int = 0):
    """(sigma, epi) per time of the SUM of the listed summands.  The operand errors of a
    walker pair's two positions are shared by every summand that uses the pair, so the
    sum is linearised as a whole (derivatives with respect to the per-position operands);
    the propagator-entry terms (FP32 accumulation, parking) belong to one summand each and
    add in quadrature; the epilogue terms add linearly."""
    import torch

    ts = TileSetup(orc, r_step, pairs, interaction)
    n_occ = ts.n_occ
    sig = np.zeros(len(tau_step))
    epi = np.zeros(len(tau_step))
    for t, tau in enumerate(tau_step):
        s = ts.scales(tau)[None, None, :, None]
        XU = ts.PHU * s  # [U][2][n_orb][4]
        SXU = np.sqrt((form.u_gemm * ts.NRU * s) ** 2 + (form.u_rep * np.abs(XU)) ** 2)
        XUt = torch.tensor(XU, requires_grad=True)
        X = torch.stack([XUt[ts.ip, 0], XUt[ts.ip, 1], XUt[ts.iq, 0], XUt[ts.iq, 1]])
        e, G, mag = summands(ts, X, keep_graph=True)
        e.sum().backward()
        var = float(((XUt.grad.abs().numpy() * SXU) ** 2).sum())
        Xn = X.detach().numpy()
        for key, g in G.items():
            ks = slice(0, n_occ) if key[0] == "m" else slice(n_occ, None)
            x, y = {"m31": (2, 0), "m42": (3, 1), "p13": (0, 2), "p24": (1, 3), "p14": (0, 3), "p23": (1, 2)}[key]
            norm2 = np.sqrt(np.einsum("bkc,bkd->bcd", np.abs(Xn[x][:, ks]) ** 2, np.abs(Xn[y][:, ks]) ** 2))
            gg = g.grad.abs().numpy()
            var += float(((gg * form.u_acc * norm2) ** 2).sum())
            if key[0] == "m":
                var += float(((gg * form.u_pack * np.abs(g.detach().numpy())) ** 2).sum())
        sig[t] = np.sqrt(var)
        epi[t] = form.u_epi * float(mag.detach().numpy().sum())
    return sig, epi


def step_tolerance(orc, r_step, tau_step, form: Form, interaction: int = 0) -> float:
    """Tolerance of one step estimate I'_n = (1/n_tau) sum_t (1/mC2) sum_{p<q} e:
    KAPPA times the model standard deviation of that mean (the sum linearised as a
    whole, sum_model; the times are added linearly, since they share the spinor
    values' errors) plus its epilogue terms."""
    m = r_step.shape[0]
    pairs = [(p, q) for p in range(m) for q in range(p + 1, m)]
    sig, epi = sum_model(orc, r_step, tau_step, pairs, form, interaction)
    n = len(pairs) * len(tau_step)
    return (KAPPA * sig.sum() + epi.sum()) / n


def tile_tolerance(orc, r_step, tau_step, pairs, form: Form, interaction: int = 0):
    """Tolerance of a sum of the listed summands, per time: KAPPA times the model standard
    deviation of the sum (sum_model) plus its epilogue terms."""
    sig, epi = sum_model(orc, r_step, tau_step, pairs, form, interaction)
    return KAPPA * sig + epi


def steps_tolerance(orc, r, tau, form: Form, interaction: int = 0):
    """step_tolerance for each step of a replay (r [n][m][2][3], tau [n][n_tau])."""
    return np.array([step_tolerance(orc, r[k], tau[k], form, interaction) for k in range(len(r))])
