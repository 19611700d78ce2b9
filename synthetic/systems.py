"""Seeded synthetic molecular systems standing in for Dirac-Hartree-Fock output.

The paper's MC-MP2 step consumes spinor expansion coefficients and orbital
energies produced by a preceding DHF calculation (Sec. IV), plus the
weight-function parameters of Table 1.  The molecules' basis sets and DHF
spinors are not available here, so this module draws seeded stand-ins with
the same shapes:

* atom-centred even-tempered Cartesian Gaussian shells (s/p/d);
* 4-component spinor coefficients C (rows: L-alpha, L-beta, S-alpha, S-beta
  coefficient blocks of n_L rows each), drawn complex-normal with the small
  block scaled by 1/(2c), completed into Kramers pairs by time reversal and
  Loewdin-orthonormalised in the 4-component overlap metric;
* orbital energies log-uniform in [-Z^2/2, -0.3] (occupied) and [0.1, 50]
  (virtual), equal within a Kramers pair;
* weight-function parameters (c1, zeta1, c2, zeta2) per centre from Table 1,
  or, for the nuclear charges Table 1 lacks (50 and 17), from the
  weight-function scan (SCANNED_WEIGHTS).

This module is an input generator only.  It evaluates no basis function or
spinor at a point and contains none of the Monte Carlo MP2 arithmetic; the
overlap integrals it computes exist only to orthonormalise the stand-in
spinors.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

SPEED_OF_LIGHT = 137.035999  # atomic units, used only to scale the small-component block
ENVELOPE_LN = 1.0  # width (in ln alpha) of the exponent window of a spinor draw

# Cartesian component order of a shell of angular momentum l.
CARTESIAN = {
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)],
}

# Table 1 weight-function parameters (c1, zeta1, c2, zeta2) by element.
TABLE1 = {
    "H": (0.25, 0.06, 0.15, 0.6),
    "O": (0.8, 0.2, 1.0, 0.4),
    "Cu": (0.8, 0.35, 2.0, 0.6),
    "Ag": (0.1, 0.1, 0.8, 0.6),
    "Au": (0.05, 0.6, 4.0, 0.8),
}
# Nuclear charges used by the synthetic clusters, mapped onto the nearest
# Table 1 row (Z=30 takes the Cu row, Z=80 Au, Z=1 H).
TABLE1_ROW_FOR_Z = {1: "H", 17: "O", 30: "Cu", 50: "Ag", 80: "Au"}
# Z = 50 and Z = 17 have no Table 1 row.  Their (c1, zeta1, c2, zeta2) were chosen
# by the weight-function scan (paper_2203_05632_gb300/wscan.py) on the medium
# system: the most diffuse exponent stays at 0.1, below twice the sum of the
# smallest occupied and virtual exponents (0.05 each), so f^2/w decays at large
# distance, and a second Gaussian of exponent 5 (Sn) or 3 (Cl) puts ~10 % of the
# weight near the nuclei, where the occupied density is up to 10^5 times g of the
# nearest Table 1 rows (Ag, O).  With them sigma-bar_N sqrt(N) stays within
# 20 % from 10^4 to 4 x 10^4 steps; with the Ag and O rows it does not settle.
SCANNED_WEIGHTS = {50: (0.5, 0.1, 1.0, 5.0), 17: (0.5, 0.1, 0.5, 3.0)}


def weight_row(z: int):
    """(c1, zeta1, c2, zeta2) of Eq. basisSet for nuclear charge z."""
    if z in SCANNED_WEIGHTS:
        return SCANNED_WEIGHTS[z]
    return TABLE1[TABLE1_ROW_FOR_Z[z]]


@dataclasses.dataclass
class System:
    """A synthetic system in the layout the library and the oracle take."""

    name: str
    centres: np.ndarray  # [n_c, 3] float64, bohr
    charges: np.ndarray  # [n_c] int32
    shell_centre: np.ndarray  # [n_sh] int32
    shell_l: np.ndarray  # [n_sh] int32 (0, 1 or 2)
    shell_alpha: np.ndarray  # [n_sh] float64
    shell_coef: np.ndarray  # [n_sh] float64
    n_occ: int
    n_vir: int
    C: np.ndarray  # [4 n_L, n_orb] complex128, occupied columns first
    eps: np.ndarray  # [n_orb] float64
    weight: np.ndarray  # [n_c, 4] float64: c1, zeta1, c2, zeta2
    n_comp: int = 4  # 2: two-component spinors (alpha, beta rows only; the small rows of C are zero)

    @property
    def n_l(self) -> int:
        return int(sum(len(CARTESIAN[int(l)]) for l in self.shell_l))

    @property
    def n_orb(self) -> int:
        return self.n_occ + self.n_vir

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.centres, self.shell_centre, self.shell_l, self.shell_alpha,
                  self.shell_coef, self.C, self.eps, self.weight):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(f"{self.n_occ},{self.n_vir},{self.n_comp}".encode())
        return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# Cartesian Gaussian overlaps (input preparation only)
# --------------------------------------------------------------------------

_GH_T, _GH_W = np.polynomial.hermite.hermgauss(8)  # exact for degree <= 15


def _expand(shell_centre, shell_l, shell_alpha, shell_coef, centres):
    rows = []
    for c, l, a, k in zip(shell_centre, shell_l, shell_alpha, shell_coef):
        for pw in CARTESIAN[int(l)]:
            rows.append((int(c), pw[0], pw[1], pw[2], float(a), float(k)))
    cen = np.array([centres[r[0]] for r in rows], dtype=np.float64).reshape(-1, 3)
    pw = np.array([[r[1], r[2], r[3]] for r in rows], dtype=np.int64).reshape(-1, 3)
    al = np.array([r[4] for r in rows], dtype=np.float64)
    co = np.array([r[5] for r in rows], dtype=np.float64)
    return cen, pw, al, co


def _ov1d(a, b, A, B, al, be):
    """1-D integral of (x-A)^a (x-B)^b exp(-al(x-A)^2 - be(x-B)^2), broadcast.

    Gauss-Hermite quadrature with 8 nodes integrates the polynomial part
    exactly for a + b <= 15.  Negative powers denote an absent term (0)."""
    p = al + be
    P = (al * A + be * B) / p
    pre = np.exp(-al * be / p * (A - B) ** 2) / np.sqrt(p)
    x = P[..., None] + _GH_T / np.sqrt(p)[..., None]
    aa = np.maximum(a, 0)[..., None]
    bb = np.maximum(b, 0)[..., None]
    val = pre * np.sum(_GH_W * (x - A[..., None]) ** aa * (x - B[..., None]) ** bb, axis=-1)
    return np.where((a < 0) | (b < 0), 0.0, val)


def overlap_matrices(sys_or_shells, centres=None):
    """Return (S_LL, S_SS): <g_mu|g_nu> and <grad g_mu . grad g_nu>.

    S_SS is the overlap of the kinetically balanced small-component basis
    (sigma.grad)(g e_s): the Pauli cross terms cancel for real g, leaving the
    gradient dot product, diagonal in spin."""
    if isinstance(sys_or_shells, System):
        s = sys_or_shells
        cen, pw, al, co = _expand(s.shell_centre, s.shell_l, s.shell_alpha, s.shell_coef, s.centres)
    else:
        cen, pw, al, co = _expand(*sys_or_shells, centres)
    n = len(al)
    A = cen[:, None, :].repeat(n, 1)
    B = cen[None, :, :].repeat(n, 0)
    ai = pw[:, None, :].repeat(n, 1)
    bi = pw[None, :, :].repeat(n, 0)
    aa = al[:, None].repeat(n, 1)
    bb = al[None, :].repeat(n, 0)
    O = [[[None] * 3 for _ in range(3)] for _ in range(3)]
    for da in (-1, 0, 1):
        for db in (-1, 0, 1):
            O[da + 1][db + 1] = [
                _ovl for _ovl in (
                    _ov1d(ai[..., d] + da, bi[..., d] + db, A[..., d], B[..., d], aa, bb)
                    for d in range(3))
            ]
    base = [O[1][1][d] for d in range(3)]
    s_ll = base[0] * base[1] * base[2]
    s_ss = np.zeros_like(s_ll)
    for d in range(3):
        a = ai[..., d].astype(np.float64)
        b = bi[..., d].astype(np.float64)
        dd = (a * b * O[0][0][d]
              - 2.0 * bb * a * O[0][2][d]
              - 2.0 * aa * b * O[2][0][d]
              + 4.0 * aa * bb * O[2][2][d])
        others = [base[e] for e in range(3) if e != d]
        s_ss += dd * others[0] * others[1]
    cc = np.outer(co, co)
    return s_ll * cc, s_ss * cc


# --------------------------------------------------------------------------
# Basis shells and geometry
# --------------------------------------------------------------------------

def _primitive_norm(alpha: float, l: int) -> float:
    """Normalisation of x^l exp(-alpha r^2) (the axis-aligned component)."""
    dfact = 1.0
    for k in range(2 * l - 1, 0, -2):
        dfact *= k
    return (2.0 * alpha / math.pi) ** 0.75 * (4.0 * alpha) ** (l / 2.0) / math.sqrt(dfact)


def _even_tempered(alpha0: float, beta: float, n: int):
    return [alpha0 * beta ** k for k in range(n)]


def _shells_for(centre_index: int, spec):
    """spec: list of (l, alpha0, beta, n) tuples."""
    out = []
    for l, a0, beta, n in spec:
        for a in _even_tempered(a0, beta, n):
            out.append((centre_index, l, a, _primitive_norm(a, l)))
    return out


# Basis recipes per element and config (even-tempered, Cartesian).
_TINY_ZN = [(0, 0.05, 2.5, 11), (1, 0.05, 2.5, 2)]                 # 11 + 6 = 17
_TINY_H = [(0, 0.05, 2.5, 3)]                                       # 3
_MED_SN = [(0, 0.05, 2.5, 14), (1, 0.08, 2.5, 8), (2, 0.2, 2.5, 3)]  # 14+24+18 = 56
_MED_CL = [(0, 0.05, 2.5, 8), (1, 0.08, 2.5, 6), (2, 0.2, 2.5, 2)]   # 8+18+12 = 38
_ADJ_SN = [(0, 0.05, 2.5, 12), (1, 0.08, 2.5, 6), (2, 0.2, 2.5, 3)]  # 12+18+18 = 48
_ADJ_CL = [(0, 0.05, 2.5, 9), (1, 0.08, 2.5, 5), (2, 0.2, 2.5, 2)]   # 9+15+12 = 36
_SIZE_HG = [(0, 0.1, 2.5, 16), (1, 0.1, 2.5, 8), (2, 0.2, 2.5, 4)]   # 16+24+24 = 64
_SIZE_CL = [(0, 0.1, 2.5, 8), (1, 0.1, 2.5, 5)]                      # 8+15 = 23


def _geometry(config: str, n_units: int = 1):
    if config == "tiny":
        return [30, 1], np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.5]])
    if config == "medium":
        a = 4.5 / (2.0 * math.sqrt(2.0))  # Sn4 tetrahedron with 4.5 bohr edges
        sn = np.array([[a, a, a], [a, -a, -a], [-a, a, -a], [-a, -a, a]])
        cl = np.array([sn[0] + 4.0 * sn[0] / np.linalg.norm(sn[0]),
                       sn[1] + 4.0 * sn[1] / np.linalg.norm(sn[1])])
        return [50, 50, 50, 50, 17, 17], np.vstack([sn, cl])
    if config == "adjoint":
        return [50, 17, 17], np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 4.2], [4.0, 0.0, -1.3]])
    if config == "size":
        charges, pos = [], []
        for u in range(n_units):
            i, j, k = (u >> 0) & 1, (u >> 1) & 1, (u >> 2) & 1
            hg = np.array([5.0 * i, 5.0 * j, 5.0 * k])
            out = np.array([2 * i - 1, 2 * j - 1, 2 * k - 1], dtype=np.float64)
            out /= np.linalg.norm(out)
            perp = np.cross(out, [0.0, 0.0, 1.0] if abs(out[2]) < 0.9 else [1.0, 0.0, 0.0])
            perp /= np.linalg.norm(perp)
            charges += [80, 17, 17]
            pos += [hg, hg + 4.3 * out, hg + 4.3 * perp]
        return charges, np.array(pos)
    raise ValueError(config)


def _recipe(config: str, z: int):
    table = {
        "tiny": {30: _TINY_ZN, 1: _TINY_H},
        "medium": {50: _MED_SN, 17: _MED_CL},
        "adjoint": {50: _ADJ_SN, 17: _ADJ_CL},
        "size": {80: _SIZE_HG, 17: _SIZE_CL},
    }
    return table[config][z]


# --------------------------------------------------------------------------
# Spinors
# --------------------------------------------------------------------------

def time_reversed_coefficients(c: np.ndarray, n_l: int) -> np.ndarray:
    """Coefficients of K phi for the spinor with coefficient column(s) c.

    With K = -i sigma_y (x) complex conjugation acting on each 2-spinor:
    K(g e_a) = g e_b and K(g e_b) = -g e_a for the large basis, while the
    kinetically balanced small basis obeys K chi^S_a = -chi^S_b and
    K chi^S_b = chi^S_a (K anticommutes with the factor i in i(sigma.p))."""
    la, lb, sa, sb = (c[k * n_l:(k + 1) * n_l] for k in range(4))
    return np.concatenate([-np.conj(lb), np.conj(la), np.conj(sb), -np.conj(sa)], axis=0)


def _loewdin(C: np.ndarray, metric: np.ndarray) -> np.ndarray:
    M = C.conj().T @ metric @ C
    w, V = np.linalg.eigh(M)
    return C @ (V * (1.0 / np.sqrt(w))) @ V.conj().T


# Soft variant of the tiny system: the same geometry and counts with exponents
# and orbital energies kept within the extent of the Table 1 weight function,
# so the Monte Carlo estimate converges in seconds (used to pin the estimator).
_SOFT_ZN = [(0, 0.05, 2.5, 5), (1, 0.05, 2.5, 4)]                  # 5 + 12 = 17
_SOFT_H = [(0, 0.08, 2.5, 3)]                                        # 3
# Soft variant of the medium system: the same shell counts (n_L = 300) with
# the even-tempered ratio 1.4 instead of 2.5 (largest exponent 3.9 instead of
# 7,450), so that with the soft energy windows no orbital is much tighter than
# the weight function and the estimator has a finite variance.
_SOFT_SN = [(0, 0.05, 1.4, 14), (1, 0.08, 1.4, 8), (2, 0.2, 1.4, 3)]
_SOFT_CL = [(0, 0.05, 1.4, 8), (1, 0.08, 1.4, 6), (2, 0.2, 1.4, 2)]
# Soft variant of the size-series units (Z=80 + 2 Z=17, 110 functions per unit),
# ratio 1.3 (largest exponent 5.1).
_SOFT_HG = [(0, 0.1, 1.3, 16), (1, 0.1, 1.3, 8), (2, 0.2, 1.3, 4)]
_SOFT_SIZE_CL = [(0, 0.1, 1.3, 8), (1, 0.1, 1.3, 5)]


def make_system(config: str, seed: int = 2203, n_units: int = 1, soft: bool = False,
                small_scale: float | None = None, two_component: bool = False,
                weights: dict | None = None) -> System:
    """Draw one of the synthetic systems.

    config: "tiny" (Z=30 + Z=1, n_L = 20, 4 occ / 16 vir),
            "medium" (4 x Z=50 + 2 x Z=17, n_L = 300, 80 occ / 400 vir),
            "adjoint" (Z=50 + 2 x Z=17, n_L = 120, 24 occ / 120 vir),
            "size" (n_units x (Z=80 + 2 x Z=17), n_L = 110 per unit,
                    40 occ / 180 vir per unit).
    small_scale: factor on the random small-component coefficients before
    orthonormalisation (default 1/(2c), the kinetic-balance size); a test
    system with small_scale = 1 has small components of order one, so terms
    that couple large and small components (the Gaunt/Breit interaction) are
    of the size of the Coulomb ones.
    two_component: two-component spinors (alpha, beta) over the large basis
    only, orthonormal in S_LL; C keeps 4 n_L rows with the small rows zero and
    the system is marked n_comp = 2.
    weights: optional {Z: (c1, zeta1, c2, zeta2)} replacing the weight-function
    parameters of those nuclear charges (the spinors and energies are unchanged)."""
    rng = np.random.default_rng(seed)
    charges, centres = _geometry(config, n_units)
    shells = []
    for ic, z in enumerate(charges):
        recipe = _recipe(config, z)
        if soft:
            assert config in ("tiny", "medium", "size"), "soft variants exist for the tiny, medium and size systems"
            if config == "size":
                recipe = {80: _SOFT_HG, 17: _SOFT_SIZE_CL}[z]
            else:
                recipe = {30: _SOFT_ZN, 1: _SOFT_H, 50: _SOFT_SN, 17: _SOFT_CL}[z]
        shells += _shells_for(ic, recipe)
    shell_centre = np.array([s[0] for s in shells], dtype=np.int32)
    shell_l = np.array([s[1] for s in shells], dtype=np.int32)
    shell_alpha = np.array([s[2] for s in shells], dtype=np.float64)
    shell_coef = np.array([s[3] for s in shells], dtype=np.float64)
    n_l = int(sum(len(CARTESIAN[int(l)]) for l in shell_l))

    n_occ, n_vir = {
        "tiny": (4, 16), "medium": (80, 400), "adjoint": (24, 120),
        "size": (40 * n_units, 180 * n_units),
    }[config]
    n_orb = n_occ + n_vir
    assert n_orb % 2 == 0 and n_occ % 2 == 0

    s_ll, s_ss = overlap_matrices((shell_centre, shell_l, shell_alpha, shell_coef), centres)
    z = np.zeros_like(s_ll)
    metric = np.block([[s_ll, z, z, z], [z, s_ll, z, z], [z, z, s_ss, z], [z, z, z, s_ss]])

    zmax = max(charges)
    n_pair_occ, n_pair_vir = n_occ // 2, n_vir // 2
    occ_lo, vir_hi = (2.0, 3.0) if soft else (zmax * zmax / 2.0, 50.0)
    e_occ = -np.exp(rng.uniform(math.log(0.3), math.log(occ_lo), n_pair_occ))
    e_vir = np.exp(rng.uniform(math.log(0.1), math.log(vir_hi), n_pair_vir))
    e_occ.sort()
    e_vir.sort()
    eps_pairs = np.concatenate([e_occ, e_vir])
    eps = np.repeat(eps_pairs, 2)

    half = rng.standard_normal((4 * n_l, n_orb // 2)) + 1j * rng.standard_normal((4 * n_l, n_orb // 2))
    half[2 * n_l:] *= (1.0 / (2.0 * SPEED_OF_LIGHT)) if small_scale is None else float(small_scale)
    if two_component:
        half[2 * n_l:] = 0.0
    # Per-entry spread: each basis function counts with unit norm, and an
    # orbital of energy eps draws mostly on functions whose exponent matches
    # its spatial extent (alpha ~ 0.57 |eps|, the best single Gaussian for a
    # hydrogenic 1s level), a log-normal window of width ENVELOPE_LN.  DHF
    # spinors have this energy/extent relation; isotropic draws would give
    # every orbital a large amplitude on the tightest functions.
    diag = np.sqrt(np.concatenate([np.diag(s_ll)] * 2 + [np.diag(s_ss)] * 2))
    fn_alpha = np.repeat(shell_alpha, [len(CARTESIAN[int(l)]) for l in shell_l])
    alpha4 = np.tile(fn_alpha, 4)
    target = 0.57 * np.abs(eps_pairs)
    env = np.exp(-np.log(alpha4[:, None] / target[None, :]) ** 2 / (2.0 * ENVELOPE_LN ** 2))
    half *= env / diag[:, None]
    C = np.empty((4 * n_l, n_orb), dtype=np.complex128)
    C[:, 0::2] = half
    C[:, 1::2] = time_reversed_coefficients(half, n_l)
    C = _loewdin(C, metric)

    weight = np.array([(weights or {}).get(z_, weight_row(z_)) for z_ in charges], dtype=np.float64)
    name = config if config != "size" else f"size{n_units}"
    if soft:
        name += "-soft"
    if small_scale is not None:
        name += f"-small{small_scale:g}"
    if two_component:
        name += "-2c"
    return System(name=name, centres=np.ascontiguousarray(centres, dtype=np.float64),
                  charges=np.array(charges, dtype=np.int32), shell_centre=shell_centre,
                  shell_l=shell_l, shell_alpha=shell_alpha, shell_coef=shell_coef,
                  n_occ=n_occ, n_vir=n_vir, C=np.ascontiguousarray(C), eps=eps, weight=weight,
                  n_comp=2 if two_component else 4)


def nonrelativistic_variant(system: System, seed: int = 7) -> System:
    """Closed-shell spin-orbital spinors (psi e_a, psi e_b) with zero small components.

    Real spatial orbitals psi are drawn at random in the large basis and
    Loewdin-orthonormalised with S_LL; each spatial orbital yields a Kramers
    pair (psi alpha, psi beta) sharing one energy."""
    rng = np.random.default_rng(seed)
    n_l = system.n_l
    s_ll, _ = overlap_matrices(system)
    n_sp = system.n_orb // 2
    c = rng.standard_normal((n_l, n_sp)) / np.sqrt(np.diag(s_ll))[:, None]
    M = c.T @ s_ll @ c
    w, V = np.linalg.eigh(M)
    c = c @ (V / np.sqrt(w)) @ V.T
    C = np.zeros((4 * n_l, system.n_orb), dtype=np.complex128)
    C[:n_l, 0::2] = c
    C[n_l:2 * n_l, 1::2] = c
    return dataclasses.replace(system, name=system.name + "-nr", C=C)
