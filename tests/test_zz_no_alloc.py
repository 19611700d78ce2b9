"""The allocation-free entry point against the regular replay entry point and the oracle.

Callers that cannot allocate device memory use mcmp2_pair_sum_f64_noalloc,
whose intermediate sums live in a fixed array inside the library; it must
give the same step estimate as mcmp2_eval_fixed (FP64 form) for the same
samples, call after call, and both must be the oracle's I'_n of Eq. redundant
(oracle.eval_steps) to the FP64 parity tolerance.
"""
import numpy as np
import pytest

import paper_2203_05632_gb300 as pkg
import synthetic
from paper_2203_05632_gb300 import _binding as B

pytestmark = pytest.mark.gpu

REL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _inputs(system, orc, r, tau):
    """Spinor rows, propagator scales and pair weights of one step (device tensors)."""
    import torch
    m = r.shape[0]
    n_orb = system.n_orb
    phi = np.stack([orc.spinors_at(r[p, e]) for p in range(m) for e in range(2)])  # [2m][n_orb][4]
    rows = np.ascontiguousarray(phi.transpose(0, 2, 1).reshape(8 * m, n_orb))  # row 4x + c
    o = system.n_occ
    homo, lumo = system.eps[:o].max(), system.eps[o:].min()
    arg = np.concatenate([system.eps[:o] - homo, -(system.eps[o:] - lumo)])
    scale = np.exp(0.5 * arg[None, :] * tau[:, None])
    a = np.array([orc.Ng() / (orc.g(r[p, 0]) * orc.g(r[p, 1])) for p in range(m)])
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(rows.view(np.float64).copy()).to(dev), torch.from_numpy(scale).to(dev),
            torch.from_numpy(a).to(dev))


@pytest.mark.parametrize("m,n_tau", [(16, 2), (37, 1)])
def test_noalloc_matches_replay_on_two_calls(tiny, tiny_oracle, m, n_tau):
    import torch
    r = synthetic.walker_positions(tiny.centres, 2, m, seed=600 + m)
    tau = synthetic.imaginary_times(tiny_oracle.lam(), 2, n_tau, seed=601 + m)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_FP64)
    replay = ctx.eval_fixed(r, tau)
    want, absmean = tiny_oracle.eval_steps(r, tau, with_abs=True)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(2):  # two calls in a row, different samples
        phi, scale, a = _inputs(tiny, tiny_oracle, r[k], tau[k])
        B.pair_sum_f64_noalloc(m, tiny.n_occ, tiny.n_vir, n_tau, phi, scale, a, tiny_oracle.lam(), out)
        torch.cuda.synchronize()
        got = float(out.item())
        scale_k = max(abs(want[k]), 1e-3 * absmean[k])
        assert abs(got - want[k]) <= REL * scale_k, (k, got, want[k])      # the oracle
        assert abs(got - replay[k]) <= REL * scale_k, (k, got, replay[k])  # the regular entry point


def test_noalloc_rejects_sizes_beyond_its_scratch(tiny, tiny_oracle):
    import torch
    m = 8
    r = synthetic.walker_positions(tiny.centres, 1, m, seed=5)[0]
    phi, scale, a = _inputs(tiny, tiny_oracle, r, np.array([0.5]))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big_m = 8 * 400  # 400 pair blocks -> 80,200 tiles > 65,536 partial sums
    with pytest.raises(pkg.McMp2Error) as e:
        B.pair_sum_f64_noalloc(big_m, tiny.n_occ, tiny.n_vir, 1, phi, scale, a, tiny_oracle.lam(), out)
    assert e.value.code == -6
    with pytest.raises(pkg.McMp2Error) as e:
        B.pair_sum_f64_noalloc(m, tiny.n_occ, tiny.n_vir, 1, phi, scale, a, -1.0, out)
    assert e.value.code == -1
