"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: published
known-answer values, closed forms, finite differences, symmetries of the
definitions, an explicit sum over states, the nonrelativistic scalar formula
printed in the paper, or the deterministic MP2 energy.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
import synthetic
from oracle import mp2

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------

def _kat_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answer():
    for ctr, key, out in _kat_rows():
        assert list(oracle.philox4x32_10(ctr, key)) == out


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc for curand's host Philox")
def test_philox_matches_curand_host_routine():
    rng = np.random.default_rng(5)
    cases = rng.integers(0, 2 ** 32, size=(64, 6), dtype=np.uint64).astype(np.uint32)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "chk")
        subprocess.run(["nvcc", "-O2", "-o", exe, os.path.join(HERE, "philox_curand_check.cu")],
                       check=True, capture_output=True)
        inp = "\n".join(" ".join(f"{int(x):08x}" for x in row) for row in cases) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for row, line in zip(cases, out):
        want = [int(x, 16) for x in line.split()]
        assert list(oracle.philox4x32_10(row[:4], row[4:])) == want


def test_tau_inverse_cdf_distribution():
    """tau = -ln(u)/lambda follows w(tau) = lambda exp(-lambda tau) (Eq. tauWeight)."""
    lam = 1.7
    taus = np.concatenate([oracle.tau_draws(99, st, 500, lam) for st in range(40)])
    assert taus.min() >= 0.0
    res = stats.kstest(taus, lambda t: 1.0 - np.exp(-lam * t))
    assert res.pvalue > 1e-3


def test_laplace_transform_of_denominator():
    """P1: <exp(-Delta tau)/w(tau)> = Int exp(-Delta tau) dtau = 1/Delta (the Laplace
    transform of 1/D), and at Delta = lambda every sample is exactly 1/lambda."""
    lam = 0.8
    taus = np.concatenate([oracle.tau_draws(7, st, 1000, lam) for st in range(200)])
    w = lam * np.exp(-lam * taus)
    for delta in (0.6 * lam, 1.3 * lam, 2.0 * lam, 5.0 * lam):
        x = np.exp(-delta * taus) / w
        err = x.std() / math.sqrt(len(x))
        assert abs(x.mean() - 1.0 / delta) < 5 * err, delta
    x = np.exp(-lam * taus) / w
    assert np.max(np.abs(x * lam - 1.0)) < 1e-12


# --------------------------------------------------------------------------
# Basis, spinors, weight function
# --------------------------------------------------------------------------

def test_basis_gradient_matches_finite_differences(tiny_oracle):
    rng = np.random.default_rng(0)
    for r in rng.normal(0.0, 0.8, size=(6, 3)):
        v, g = tiny_oracle.basis_at(r)
        h = 1e-5
        fd = np.stack([(tiny_oracle.basis_at(r + h * e)[0] - tiny_oracle.basis_at(r - h * e)[0]) / (2 * h)
                       for e in np.eye(3)], axis=1)
        assert np.allclose(fd, g, rtol=1e-6, atol=1e-7 * np.abs(g).max())


def test_cartesian_functions_follow_their_definition(tiny, tiny_oracle):
    """g_mu(r) = coef (x-Ax)^a (y-Ay)^b (z-Az)^c exp(-alpha |r-A|^2), in the documented order."""
    r = np.array([0.31, -0.47, 0.88])
    v, _ = tiny_oracle.basis_at(r)
    mu = 0
    for c, l, a, k in zip(tiny.shell_centre, tiny.shell_l, tiny.shell_alpha, tiny.shell_coef):
        d = r - tiny.centres[c]
        for pw in synthetic.CARTESIAN[int(l)]:
            want = k * np.prod(d ** np.array(pw)) * math.exp(-a * d @ d)
            assert v[mu] == pytest.approx(want, rel=1e-14, abs=1e-300)
            mu += 1


def test_small_components_are_sigma_dot_grad_of_the_small_coefficients(tiny, tiny_oracle):
    """Kinetic balance (after Eq. C): phi^S = i(sigma.p) chi = (sigma.grad) chi with chi = sum_mu C^S_mu g_mu e_s,
    checked by finite differences of chi built from basis values only."""
    n_l = tiny.n_l
    sig = mp2.PAULI

    def chi(r):
        v, _ = tiny_oracle.basis_at(r)
        return np.stack([v @ tiny.C[2 * n_l:3 * n_l], v @ tiny.C[3 * n_l:]], axis=1)  # [n_orb, 2]

    r = np.array([0.2, 0.4, 0.7])
    h = 1e-5
    dchi = [(chi(r + h * e) - chi(r - h * e)) / (2 * h) for e in np.eye(3)]
    want = sum(np.einsum("cs,ks->kc", sig[j], dchi[j]) for j in range(3))
    got = tiny_oracle.spinors_at(r)
    assert np.allclose(got[:, 2:], want, rtol=1e-6, atol=1e-8 * np.abs(want).max())
    v, _ = tiny_oracle.basis_at(r)
    assert np.allclose(got[:, 0], v @ tiny.C[:n_l], rtol=1e-13, atol=1e-15)
    assert np.allclose(got[:, 1], v @ tiny.C[n_l:2 * n_l], rtol=1e-13, atol=1e-15)


def test_kramers_partners_pointwise(tiny, tiny_oracle):
    """Columns 2j+1 hold the time-reversed partner: phi' = K phi with K = -i sigma_y C
    on each 2-spinor, i.e. (a, b) -> (-conj b, conj a), at every point."""
    for r in np.random.default_rng(3).normal(0.0, 0.7, size=(4, 3)):
        phi = tiny_oracle.spinors_at(r)
        a, b = phi[0::2], phi[1::2]
        want = np.stack([-a[:, 1].conj(), a[:, 0].conj(), -a[:, 3].conj(), a[:, 2].conj()], axis=1)
        assert np.allclose(b, want, rtol=1e-11, atol=1e-11 * np.abs(a).max())


def test_weight_function_definition(tiny, tiny_oracle):
    """Eq. basisSet with N_zeta = (2 zeta / pi)^{3/4}."""
    r = np.array([0.4, -0.1, 1.1])
    want = 0.0
    for R, (c1, z1, c2, z2) in zip(tiny.centres, tiny.weight):
        d2 = float((r - R) @ (r - R))
        want += c1 * (2 * z1 / math.pi) ** 0.75 * math.exp(-z1 * d2)
        want += c2 * (2 * z2 / math.pi) ** 0.75 * math.exp(-z2 * d2)
    assert tiny_oracle.g(r) == pytest.approx(want, rel=1e-14)


def test_table1_parameters_match_the_paper():
    for line in open(os.path.join(GOLDEN, "table1_weight_parameters.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        assert tuple(float(x) for x in vals) == synthetic.TABLE1[name]


def test_Ng_closed_form_matches_reciprocal_space_quadrature(tiny, tiny_oracle):
    """N_g = Int Int g g / r12 by a 1-D k-space integral for each pair of Gaussians:
    (2/pi) Int_0^inf exp(-k^2 (a+b)/(4ab)) sin(kR)/(kR) dk for unit charges."""
    total = 0.0
    for I, (RA, wa) in enumerate(zip(tiny.centres, tiny.weight)):
        for J, (RB, wb) in enumerate(zip(tiny.centres, tiny.weight)):
            R = float(np.linalg.norm(RA - RB))
            for ca, a in ((wa[0], wa[1]), (wa[2], wa[3])):
                for cb, b in ((wb[0], wb[1]), (wb[2], wb[3])):
                    f = (lambda k, a=a, b=b, R=R: math.exp(-k * k * (a + b) / (4 * a * b))
                         * (math.sin(k * R) / (k * R) if R > 0 and k > 0 else 1.0))
                    val, _ = integrate.quad(f, 0.0, np.inf, limit=400, epsabs=0, epsrel=1e-12)
                    charge = ca * (2 * a / math.pi) ** 0.75 * (math.pi / a) ** 1.5 \
                        * cb * (2 * b / math.pi) ** 0.75 * (math.pi / b) ** 1.5
                    total += charge * 2.0 / math.pi * val
    assert tiny_oracle.Ng() == pytest.approx(total, rel=1e-9)


def test_lambda_definition(tiny, tiny_oracle):
    homo = tiny.eps[:tiny.n_occ].max()
    lumo = tiny.eps[tiny.n_occ:].min()
    assert tiny_oracle.lam() == 2.0 * (lumo - homo)


def test_metropolis_samples_the_pair_weight(soft_oracle, tiny_soft):
    """The walk is stationary in w(r1,r2) = g g /(N_g r12), so <r12>_w = (Int g)^2 / N_g."""
    s = tiny_soft
    int_g = sum(c * (2 * z / math.pi) ** 0.75 * (math.pi / z) ** 1.5
                for row in s.weight for c, z in ((row[0], row[1]), (row[2], row[3])))
    want = int_g ** 2 / soft_oracle.Ng()
    m = 64
    r = synthetic.walker_positions(s.centres, 1, m, seed=1)[0]
    r, delta = soft_oracle.burn_in(r, 12, 1000)
    per_step = []
    step = 1000
    for _ in range(4000):
        r, _ = soft_oracle.metropolis(r, 12, step, 1, delta)
        step += 1
        per_step.append(np.linalg.norm(r[:, 0] - r[:, 1], axis=1).mean())
    mean, _, err, _ = oracle.blocking(np.array(per_step), 100)
    assert abs(mean - want) < 4 * err, (mean, want, err)


# --------------------------------------------------------------------------
# Green's functions and the integrand
# --------------------------------------------------------------------------

def _four_points():
    return np.array([[0.1, 0.3, -0.2], [0.5, -0.4, 1.2], [-0.3, 0.2, 0.4], [0.2, 0.6, 1.7]])


def test_green_functions_are_hermitian_in_their_points(tiny_oracle):
    """P6: G(y, x) = G(x, y)^dagger for both propagators."""
    x, y = _four_points()[:2]
    px, py = tiny_oracle.spinors_at(x), tiny_oracle.spinors_at(y)
    for kind in (-1, 1):
        gxy = tiny_oracle.green(px, py, 0.37, kind)
        gyx = tiny_oracle.green(py, px, 0.37, kind)
        assert np.allclose(gyx, gxy.conj().T, rtol=1e-13, atol=1e-15 * np.abs(gxy).max())


def test_pair_swap_gives_complex_conjugate(tiny_oracle):
    """P6: f(r3,r4,r1,r2) = conj f(r1,r2,r3,r4), so sum_{p<q} Re f = 1/2 sum_{p!=q} f."""
    r1, r2, r3, r4 = _four_points()
    a = tiny_oracle.pair_value(r1, r2, r3, r4, 0.21)
    b = tiny_oracle.pair_value(r3, r4, r1, r2, 0.21)
    assert b == pytest.approx(a.conjugate(), rel=1e-12)
    c = tiny_oracle.pair_value(r2, r1, r4, r3, 0.21)
    assert c == pytest.approx(a, rel=1e-12)


def _explicit_sum(orc, system, pts, tau):
    """-1/2 sum_{ijab} e^{(ei+ej-ea-eb) tau} rho_ia(1) rho_jb(2) [rho_ai(3) rho_bj(4) - rho_bi(3) rho_aj(4)]
    times N_g^2/(g1 g2 g3 g4) e^{lambda tau}/lambda, rho_kl = phi_k^dag phi_l (Eq. FinalMP2
    after the Laplace transform, summed over states at fixed points)."""
    o = system.n_occ
    phis = [orc.spinors_at(p) for p in pts]
    rho = [np.einsum("kc,lc->kl", ph.conj(), ph) for ph in phis]
    e = system.eps
    occ, vir = slice(0, o), slice(o, None)
    D = e[occ][:, None, None, None] + e[occ][None, None, :, None] - e[vir][None, :, None, None] \
        - e[vir][None, None, None, :]
    ia1 = rho[0][occ, vir]
    jb2 = rho[1][occ, vir]
    ai3 = rho[2][vir, occ]
    bj4 = rho[3][vir, occ]
    N = np.einsum("ia,jb->iajb", ia1, jb2) * (np.einsum("ai,bj->iajb", ai3, bj4)
                                               - np.einsum("bi,aj->iajb", ai3, bj4))
    F = -0.5 * np.sum(np.exp(D * tau) * N)
    g = [orc.g(p) for p in pts]
    lam = orc.lam()
    return F * orc.Ng() ** 2 / (g[0] * g[1] * g[2] * g[3]) * math.exp(lam * tau) / lam


@pytest.mark.parametrize("tau", [0.05, 0.4, 2.5])
def test_trace_form_equals_explicit_sum_over_states(tiny, tiny_oracle, tau):
    """P2: the 4x4 trace form of Eq. MCMP2 equals the explicit orbital sum of
    Eq. FinalMP2 at fixed points, as a complex number."""
    pts = _four_points()
    got = tiny_oracle.pair_value(*pts, tau)
    want = _explicit_sum(tiny_oracle, tiny, pts, tau)
    assert abs(got - want) <= 1e-11 * abs(want)


def test_nonrelativistic_limit_is_the_printed_scalar_formula(tiny):
    """P3: with zero small components and spinors (psi e_a, psi e_b) from real psi,
    the integrand equals the printed -2/+1 form of Eq. MCMP2 with scalar
    spatial-orbital Green's functions o(x,y), v(x,y)."""
    nr = synthetic.nonrelativistic_variant(tiny)
    orc = oracle.Oracle(nr)
    n_l = nr.n_l
    c = nr.C[:n_l, 0::2].real  # spatial orbitals
    e = nr.eps[0::2]
    o = nr.n_occ // 2
    for tau in (0.1, 0.9):
        pts = _four_points()
        psi = [orc.basis_at(p)[0] @ c for p in pts]

        def og(x, y):
            return float(np.sum(psi[x][:o] * psi[y][:o] * np.exp(e[:o] * tau)))

        def vg(x, y):
            return float(np.sum(psi[x][o:] * psi[y][o:] * np.exp(-e[o:] * tau)))

        F = -2.0 * og(0, 2) * vg(2, 0) * og(1, 3) * vg(3, 1) + og(0, 2) * vg(3, 0) * og(1, 3) * vg(2, 1)
        g = [orc.g(p) for p in pts]
        lam = orc.lam()
        want = F * orc.Ng() ** 2 / np.prod(g) * math.exp(lam * tau) / lam
        got = orc.pair_value(*pts, tau)
        assert got.real == pytest.approx(want, rel=1e-12)
        assert abs(got.imag) <= 1e-12 * abs(want)


def test_replay_estimator_averages_pairs_and_times(tiny, tiny_oracle):
    """Eq. redundant: I'_n = (1/n_tau) sum_t (1/mC2) sum_{p<q} Re f/(w w w)."""
    m = 5
    r = synthetic.walker_positions(tiny.centres, 1, m, seed=4)
    tau = np.array([[0.3, 1.1]])
    got = tiny_oracle.eval_steps(r, tau)[0]
    vals = [tiny_oracle.pair_value(r[0, p, 0], r[0, p, 1], r[0, q, 0], r[0, q, 1], t).real
            for t in tau[0] for p in range(m) for q in range(p + 1, m)]
    assert got == pytest.approx(np.mean(vals), rel=1e-12)


# --------------------------------------------------------------------------
# Statistics
# --------------------------------------------------------------------------

def test_blocking_formula():
    """Eq. uncertainty with N_b = 4: block means known by construction."""
    x = np.array([1, 3, 1, 3, 2, 2, 2, 2, 0, 4, 4, 0, 9.0])  # trailing partial block dropped
    I, s2, sb, nb = oracle.blocking(x, 4)
    means = np.array([2.0, 2.0, 2.0])
    assert nb == 3
    assert I == pytest.approx(2.0)
    assert s2 == pytest.approx(np.mean((means - 2.0) ** 2))
    y = np.concatenate([np.full(4, 1.0), np.full(4, 3.0)])
    I, s2, sb, nb = oracle.blocking(y, 4)
    assert (I, s2, nb) == (2.0, 1.0, 2)
    assert sb == pytest.approx(1.0 / math.sqrt(2.0))


# --------------------------------------------------------------------------
# Deterministic MP2 (Eq. FinalMP2) and its integrals
# --------------------------------------------------------------------------

def _ss_closed(A, a, B, b, C, c, D, d):
    p, q = a + b, c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    Kab = math.exp(-a * b / p * float((A - B) @ (A - B)))
    Kcd = math.exp(-c * d / q * float((C - D) @ (C - D)))
    R = float(np.linalg.norm(P - Q))
    rho = p * q / (p + q)
    coul = math.erf(math.sqrt(rho) * R) / R if R > 0 else 2 * math.sqrt(rho / math.pi)
    return Kab * Kcd * (math.pi / p) ** 1.5 * (math.pi / q) ** 1.5 * coul


_CEN = [np.array([0.0, 0.1, -0.2]), np.array([0.7, -0.3, 0.4]), np.array([-0.5, 0.8, 0.3]),
        np.array([0.2, -0.6, 1.1])]
_EXP = [0.9, 0.35, 1.7, 0.6]
_S = (0, 0, 0)


def test_eri_s_functions_closed_form():
    A, B, C, D = _CEN
    a, b, c, d = _EXP
    got = mp2.prim_eri(A, a, _S, B, b, _S, C, c, _S, D, d, _S)
    assert got == pytest.approx(_ss_closed(A, a, B, b, C, c, D, d), rel=1e-12)
    got = mp2.prim_eri(A, a, _S, A, b, _S, A, c, _S, A, d, _S)  # all on one centre (R = 0)
    assert got == pytest.approx(_ss_closed(A, a, A, b, A, c, A, d), rel=1e-12)


@pytest.mark.parametrize("slot", [0, 1, 2, 3])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_eri_p_functions_are_centre_derivatives(slot, axis):
    """(x-A_x) exp(-a|r-A|^2) = (1/2a) d/dA_x exp(-a|r-A|^2): a p-type integral is a
    centre derivative of the closed-form s-type one."""
    h = 1e-4
    pw = [_S] * 4
    pw[slot] = tuple(1 if k == axis else 0 for k in range(3))
    args = []
    for k in range(4):
        args += [_CEN[k], _EXP[k], pw[k]]
    got = mp2.prim_eri(*args)

    def closed(shift):
        cen = [c.copy() for c in _CEN]
        cen[slot][axis] += shift
        return _ss_closed(cen[0], _EXP[0], cen[1], _EXP[1], cen[2], _EXP[2], cen[3], _EXP[3])

    want = (closed(h) - closed(-h)) / (2 * h) / (2 * _EXP[slot])
    assert got == pytest.approx(want, rel=2e-7, abs=1e-9)


@pytest.mark.parametrize("pw", [(2, 0, 0), (1, 1, 0), (0, 1, 1)])
def test_eri_d_functions_are_second_centre_derivatives(pw):
    """x^2 e = (d^2/dA^2 e + 2a e)/(4a^2) and xy e = (d/dAx d/dAy e)/(4a^2) on slot 2."""
    h = 2e-3
    slot = 2
    a = _EXP[slot]
    args = []
    for k in range(4):
        args += [_CEN[k], _EXP[k], pw if k == slot else _S]
    got = mp2.prim_eri(*args)

    def closed(dx, dy, dz):
        cen = [c.copy() for c in _CEN]
        cen[slot] = cen[slot] + np.array([dx, dy, dz])
        return _ss_closed(cen[0], _EXP[0], cen[1], _EXP[1], cen[2], _EXP[2], cen[3], _EXP[3])

    axes = [k for k in range(3) for _ in range(pw[k])]
    e = [np.eye(3)[k] * h for k in axes]
    if axes[0] == axes[1]:
        d2 = (closed(*e[0]) - 2 * closed(0, 0, 0) + closed(*(-e[0]))) / h ** 2
        want = (d2 + 2 * a * closed(0, 0, 0)) / (4 * a * a)
    else:
        d2 = (closed(*(e[0] + e[1])) - closed(*(e[0] - e[1])) - closed(*(e[1] - e[0]))
              + closed(*(-e[0] - e[1]))) / (4 * h * h)
        want = d2 / (4 * a * a)
    assert got == pytest.approx(want, rel=1e-5, abs=1e-8)


@pytest.fixture(scope="module")
def tiny_eri(tiny_oracle):
    return mp2.spinor_eri(tiny_oracle)


def test_spinor_integrals_symmetries_and_positivity(tiny, tiny_eri):
    V = tiny_eri
    assert np.allclose(V, V.transpose(2, 3, 0, 1), atol=1e-12 * np.abs(V).max())
    assert np.allclose(V, V.transpose(1, 0, 3, 2).conj(), atol=1e-12 * np.abs(V).max())
    n = tiny.n_orb
    A = V.transpose(1, 0, 2, 3).reshape(n * n, n * n)  # int rho_kl^* rho_mn / r12
    assert np.allclose(A, A.conj().T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > -1e-10 * np.abs(A).max()


def test_spinor_integrals_match_real_space_quadrature_of_one_density(tiny, tiny_oracle, tiny_eri):
    """(kk|ll) for diffuse-dominated spinors against an independent route: the
    self-consistent check (kk|kk) >= 0 and a Monte Carlo estimate of
    Int Int rho_k(1) rho_l(2)/r12 with importance sampling from the pair weight."""
    V = tiny_eri
    o = tiny.n_occ
    k, l = o - 1, o  # HOMO-like and LUMO-like spinors
    rng = np.random.default_rng(2)
    n = 40000
    # sample r1, r2 independently from a broad Gaussian centred between the atoms
    mid = tiny.centres.mean(axis=0)
    sig = 1.6
    r1 = mid + sig * rng.standard_normal((n, 3))
    r2 = mid + sig * rng.standard_normal((n, 3))
    dens = lambda r: np.exp(-np.sum((r - mid) ** 2, axis=1) / (2 * sig * sig)) / (2 * math.pi * sig * sig) ** 1.5  # noqa
    rho_k = np.array([np.sum(np.abs(tiny_oracle.spinors_at(x)[k]) ** 2) for x in r1])
    rho_l = np.array([np.sum(np.abs(tiny_oracle.spinors_at(x)[l]) ** 2) for x in r2])
    w = rho_k * rho_l / np.linalg.norm(r1 - r2, axis=1) / (dens(r1) * dens(r2))
    est, err = w.mean(), w.std() / math.sqrt(n)
    assert abs(V[k, k, l, l].real - est) < 5 * err + 1e-3 * abs(est)


def test_mc_estimate_matches_deterministic_mp2_soft(tiny_soft, soft_oracle):
    """P4 (CPU form): the Monte Carlo run of Sec. III agrees with the sum-over-states
    E2 of Eq. FinalMP2 within 3 sigma on a system the walk covers well."""
    E2 = mp2.mp2_energy(tiny_soft, mp2.spinor_eri(soft_oracle))
    r0 = synthetic.walker_positions(tiny_soft.centres, 1, 16, seed=11)[0]
    means, errs = [], []
    for seed in range(6):
        res = soft_oracle.run(r0, 100 + seed, 300, 3000, 1)
        I, _, sb, _ = oracle.blocking(res["per_step"])
        means.append(I)
        errs.append(sb)
    mean = float(np.mean(means))
    err = float(np.sqrt(np.sum(np.square(errs)))) / len(errs)
    assert abs(mean - E2) < 3.0 * err, (mean, err, E2)
    assert err < 0.25 * abs(E2)


def test_deterministic_energy_is_invariant_to_spinor_phases(tiny, tiny_oracle, tiny_eri):
    """E2 is a sum over states: multiplying each spinor by a phase leaves it unchanged."""
    import dataclasses
    ph = np.exp(1j * np.random.default_rng(8).uniform(0, 2 * np.pi, tiny.n_orb))
    s2 = dataclasses.replace(tiny, C=tiny.C * ph[None, :])
    e1 = mp2.mp2_energy(tiny, tiny_eri)
    e2 = mp2.mp2_energy(s2, mp2.spinor_eri(oracle.Oracle(s2)))
    assert e2 == pytest.approx(e1, rel=1e-11)
