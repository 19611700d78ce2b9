"""The adjoint (mcmp2_backward) against finite differences under common random
numbers, against the oracle, and against the analytic orbital-energy gradient
of the deterministic MP2 energy."""
import numpy as np
import pytest

import oracle
import paper_2203_05632_gb300 as pkg
import synthetic
from oracle import mp2

pytestmark = pytest.mark.gpu

H = 1e-5       # central-difference step
REL_FD = 1e-6  # adjoint vs central differences


@pytest.fixture(scope="module")
def adj_system():
    return synthetic.make_system("adjoint")


def _samples(system, lam, n, m, n_tau, seed):
    r = synthetic.walker_positions(system.centres, n, m, seed=seed)
    tau = synthetic.imaginary_times(lam, n, n_tau, seed=seed + 1)
    return r, tau


def _lam(system):
    o = system.n_occ
    return 2.0 * (system.eps[o:].min() - system.eps[:o].max())


def _non_frontier(system):
    """Orbitals whose energy can move by +-H without changing eps_HOMO or eps_LUMO."""
    o = system.n_occ
    homo, lumo = system.eps[:o].max(), system.eps[o:].min()
    return [k for k in range(system.n_orb) if system.eps[k] not in (homo, lumo)]


def test_backward_energy_equals_replay(adj_system):
    r, tau = _samples(adj_system, _lam(adj_system), 2, 24, 2, 5)
    ctx = pkg.Context(adj_system, 24, 2, pkg.MCMP2_FP64)
    e, _, _ = ctx.backward(r, tau)
    assert e == pytest.approx(ctx.eval_fixed(r, tau).mean(), rel=1e-11, abs=1e-14)


def test_eps_gradient_matches_central_differences(adj_system):
    m, n_tau = 24, 2
    r, tau = _samples(adj_system, _lam(adj_system), 3, m, n_tau, 7)
    ctx = pkg.Context(adj_system, m, n_tau, pkg.MCMP2_FP64)
    _, d_eps, _ = ctx.backward(r, tau)
    eps0 = adj_system.eps.copy()
    ks = _non_frontier(adj_system)
    pick = [ks[0], ks[len(ks) // 3], ks[len(ks) // 2], ks[-5], ks[-1]] + [adj_system.n_occ - 3]
    scale = np.abs(d_eps).max()
    for k in pick:
        e = []
        for sgn in (1, -1):
            eps = eps0.copy()
            eps[k] += sgn * H
            ctx.load(eps=eps)
            e.append(ctx.eval_fixed(r, tau).mean())
        fd = (e[0] - e[1]) / (2 * H)
        assert abs(fd - d_eps[k]) <= REL_FD * max(abs(d_eps[k]), 1e-3 * scale), (k, fd, d_eps[k])
    ctx.load(eps=eps0)


@pytest.mark.parametrize("block", ["all", "large", "small"])
def test_C_gradient_matches_central_differences(adj_system, block):
    m, n_tau = 24, 2
    r, tau = _samples(adj_system, _lam(adj_system), 3, m, n_tau, 9)
    ctx = pkg.Context(adj_system, m, n_tau, pkg.MCMP2_FP64)
    _, _, d_C = ctx.backward(r, tau)
    C0 = adj_system.C.copy()
    n_l = adj_system.n_l
    rng = np.random.default_rng(11)
    D = rng.standard_normal(C0.shape) + 1j * rng.standard_normal(C0.shape)
    if block == "large":
        D[2 * n_l:] = 0
    elif block == "small":
        D[:2 * n_l] = 0
        D *= 1.0 / 274.0  # the small-component coefficients are O(1/2c)
    D *= np.abs(C0).max() / np.abs(D).max()
    e = []
    for sgn in (1, -1):
        ctx.load(C=C0 + sgn * H * D)
        e.append(ctx.eval_fixed(r, tau).mean())
    fd = (e[0] - e[1]) / (2 * H)
    ad = float(np.real(np.sum(np.conj(d_C) * D)))
    assert abs(fd - ad) <= REL_FD * max(abs(ad), 1e-12), (fd, ad)
    ctx.load(C=C0)


def test_gradient_matches_oracle_finite_differences(tiny, tiny_oracle):
    """An independent forward (the oracle) differentiated numerically."""
    import dataclasses
    m, n_tau = 12, 1
    r, tau = _samples(tiny, tiny_oracle.lam(), 2, m, n_tau, 13)
    ctx = pkg.Context(tiny, m, n_tau, pkg.MCMP2_FP64)
    _, d_eps, d_C = ctx.backward(r, tau)
    k = _non_frontier(tiny)[0]
    vals = []
    for sgn in (1, -1):
        eps = tiny.eps.copy()
        eps[k] += sgn * H
        vals.append(oracle.Oracle(dataclasses.replace(tiny, eps=eps)).eval_steps(r, tau).mean())
    fd = (vals[0] - vals[1]) / (2 * H)
    assert abs(fd - d_eps[k]) <= 1e-5 * max(abs(d_eps[k]), 1e-3 * np.abs(d_eps).max()), (fd, d_eps[k])
    rng = np.random.default_rng(3)
    D = (rng.standard_normal(tiny.C.shape) + 1j * rng.standard_normal(tiny.C.shape)) * 0.1
    vals = []
    for sgn in (1, -1):
        vals.append(oracle.Oracle(dataclasses.replace(tiny, C=tiny.C + sgn * H * D)).eval_steps(r, tau).mean())
    fd = (vals[0] - vals[1]) / (2 * H)
    ad = float(np.real(np.sum(np.conj(d_C) * D)))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_autograd_function_returns_the_adjoint(adj_system):
    import torch
    from paper_2203_05632_gb300.autograd import mcmp2_energy
    m, n_tau = 16, 1
    r, tau = _samples(adj_system, _lam(adj_system), 2, m, n_tau, 15)
    ctx = pkg.Context(adj_system, m, n_tau, pkg.MCMP2_FP64)
    eps = torch.tensor(adj_system.eps, dtype=torch.float64, requires_grad=True)
    C = torch.tensor(adj_system.C, dtype=torch.complex128, requires_grad=True)
    E = mcmp2_energy(eps, C, ctx, r, tau)
    (2.0 * E).backward()
    e_ref, d_eps, d_C = ctx.backward(r, tau)
    assert float(E) == pytest.approx(e_ref, rel=1e-12)
    np.testing.assert_allclose(eps.grad.numpy(), 2.0 * d_eps, rtol=1e-12, atol=0)
    np.testing.assert_allclose(C.grad.numpy(), 2.0 * d_C, rtol=1e-12, atol=0)


def test_mc_eps_gradient_matches_deterministic_mp2(tiny_soft, soft_oracle):
    """P7: the Monte Carlo gradient over many walk samples agrees with the analytic
    dE2/d eps_k of Eq. FinalMP2 within its statistical error."""
    m, n_tau, seed = 16, 1, 31
    lam = soft_oracle.lam()
    r = synthetic.walker_positions(tiny_soft.centres, 1, m, seed=4)[0]
    r, delta = soft_oracle.burn_in(r, seed, 300)
    n_blocks, per_block = 12, 250
    pos = np.zeros((n_blocks * per_block, m, 2, 3))
    taus = np.zeros((n_blocks * per_block, n_tau))
    for st in range(n_blocks * per_block):
        r, _ = soft_oracle.metropolis(r, seed, 300 + st, 1, delta)
        pos[st] = r
        taus[st] = oracle.tau_draws(seed, 300 + st, n_tau, lam)
    ctx = pkg.Context(tiny_soft, m, n_tau, pkg.MCMP2_FP64)
    grads = np.array([ctx.backward(pos[b * per_block:(b + 1) * per_block],
                                   taus[b * per_block:(b + 1) * per_block])[1] for b in range(n_blocks)])
    mc = grads.mean(axis=0)
    err = grads.std(axis=0, ddof=1) / np.sqrt(n_blocks)
    exact = mp2.mp2_energy_eps_gradient(tiny_soft, mp2.spinor_eri(soft_oracle))
    z = (mc - exact) / np.maximum(err, 1e-12)
    assert np.max(np.abs(z)) < 5.0, (mc, exact, err)
    assert np.mean(z ** 2) < 4.0, z


def _walk_samples(system, m, n_tau, n, seed):
    """n steps of the device walk (FP64 Metropolis, identical in every form) and n x n_tau
    times from the inverse CDF: the fixed-seed samples of a replay."""
    walker = pkg.Context(system, m, n_tau, pkg.MCMP2_MIXED)
    walker.set_walkers(None, seed, 500)
    r = np.empty((n, m, 2, 3))
    for k in range(n):
        walker.run_steps_async(1, seed)
        r[k] = walker.get_walkers()[0]
    walker.close()
    return r, synthetic.imaginary_times(_lam(system), n, n_tau, seed=seed + 1)


def test_adjoint_at_the_adjoint_configuration(adj_system):
    """The adjoint workload as configured: m = 512 walker pairs, one time per step, 2000
    fixed-seed steps of the walk.  dE/d eps (an occupied and a virtual orbital) and dE/dC
    along a direction through every coefficient against plain central differences with
    h = 1e-5 under the same samples, to 1e-6 relative.  The coefficient direction is
    relative (each C entry moved by h times itself times a unit complex normal), so the
    O(h^2) truncation stays ~1e-10 although the estimate is of degree 8 in C."""
    import time
    m, n_tau, n = 512, 1, 2000
    r, tau = _walk_samples(adj_system, m, n_tau, n, 4242)
    ctx = pkg.Context(adj_system, m, n_tau, pkg.MCMP2_FP64)
    t0 = time.perf_counter()
    e_fwd = ctx.eval_fixed(r, tau).mean()
    t1 = time.perf_counter()
    e0, d_eps, d_C = ctx.backward(r, tau)
    t2 = time.perf_counter()
    print(f"adjoint workload, {n} steps: forward {1e3 * (t1 - t0) / n:.2f} ms/step, "
          f"backward {1e3 * (t2 - t1) / n:.2f} ms/step")
    assert e0 == pytest.approx(e_fwd, rel=1e-11)
    eps0, C0 = adj_system.eps.copy(), adj_system.C.copy()
    ks = _non_frontier(adj_system)
    occ = [k for k in ks if k < adj_system.n_occ]
    vir = [k for k in ks if k >= adj_system.n_occ]
    scale = np.abs(d_eps).max()
    for k in (occ[len(occ) // 2], vir[len(vir) // 3]):
        e = []
        for sgn in (1, -1):
            eps = eps0.copy()
            eps[k] += sgn * H
            ctx.load(eps=eps)
            e.append(ctx.eval_fixed(r, tau).mean())
        fd = (e[0] - e[1]) / (2 * H)
        print(f"dE/d eps[{k}]: adjoint {d_eps[k]:.10e}, central difference {fd:.10e}")
        assert abs(fd - d_eps[k]) <= REL_FD * max(abs(d_eps[k]), 1e-3 * scale), (k, fd, d_eps[k])
    ctx.load(eps=eps0)
    rng = np.random.default_rng(23)
    D = C0 * (rng.standard_normal(C0.shape) + 1j * rng.standard_normal(C0.shape)) / np.sqrt(2.0)
    e = []
    for sgn in (1, -1):
        ctx.load(C=C0 + sgn * H * D)
        e.append(ctx.eval_fixed(r, tau).mean())
    ctx.load(C=C0)
    fd = (e[0] - e[1]) / (2 * H)
    ad = float(np.real(np.sum(np.conj(d_C) * D)))
    print(f"dE/dC along a relative direction: adjoint {ad:.10e}, central difference {fd:.10e}")
    assert abs(fd - ad) <= REL_FD * max(abs(ad), 1e-12), (fd, ad)
