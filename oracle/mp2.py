"""Deterministic relativistic MP2 energy (Eq. FinalMP2) -- TEST INFRASTRUCTURE ONLY.

The spinor two-electron integrals (kl|mn) = Int Int phi_k^dag phi_l (1)
(1/r12) phi_m^dag phi_n (2) are assembled from Coulomb integrals over the real
functions f_{4mu+0} = g_mu, f_{4mu+j} = d_j g_mu (computed in C by
McMurchie-Davidson), and the energy is the plain sum over i, j, a, b of
Eq. FinalMP2.  Written for small systems only (the tiny configuration).
"""
from __future__ import annotations

import numpy as np

from . import _f64, _ptr, lib

# Pauli matrices sigma_x, sigma_y, sigma_z.
PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def real_function_coefficients(system) -> np.ndarray:
    """U[c, P, k] with phi_k^c(r) = sum_P U[c, P, k] f_P(r).

    Large components follow Eq. C directly; the small 2-spinor is
    sum_mu sum_s C^{S s}_{mu k} (sigma.grad)(g_mu e_s) (kinetic balance, after Eq. C), i.e.
    component c' of it takes sigma_j[c', s] C^{S s}_{mu k} on f_{4mu+1+j}."""
    n_l = system.n_l
    n = system.n_orb
    C = system.C
    U = np.zeros((4, 4 * n_l, n), dtype=np.complex128)
    for mu in range(n_l):
        U[0, 4 * mu] = C[mu]
        U[1, 4 * mu] = C[n_l + mu]
        for j in range(3):
            for cp in range(2):
                for s in range(2):
                    U[2 + cp, 4 * mu + 1 + j] += PAULI[j, cp, s] * C[(2 + s) * n_l + mu]
    return U


def function_pairs(n_l: int) -> np.ndarray:
    """Unordered pairs (P <= Q) that occur in spinor densities: both large
    (value functions) or both small (gradient functions)."""
    large = [4 * mu for mu in range(n_l)]
    small = [4 * mu + j for mu in range(n_l) for j in (1, 2, 3)]
    pairs = [(large[a], large[b]) for a in range(len(large)) for b in range(a, len(large))]
    pairs += [(small[a], small[b]) for a in range(len(small)) for b in range(a, len(small))]
    return np.array(pairs, dtype=np.int32)


def pair_coulomb_matrix(oracle, pairs: np.ndarray) -> np.ndarray:
    n = len(pairs)
    out = np.zeros((n, n))
    rc = lib().mp2_pair_eri_matrix(oracle.sp, n, _ptr(np.ascontiguousarray(pairs, dtype=np.int32)),
                                   _ptr(out), oracle.n_threads)
    if rc != 0:
        raise ValueError(f"mp2_pair_eri_matrix failed ({rc})")
    return out


def ao_eri(oracle, P, Q, R, S) -> float:
    pq = np.array([P, Q], dtype=np.int32)
    rs = np.array([R, S], dtype=np.int32)
    return lib().mp2_ao_eri(oracle.sp, _ptr(pq), _ptr(rs))


def prim_eri(A, a, pa, B, b, pb, C, c, pc, D, d, pd) -> float:
    i = lambda v: np.ascontiguousarray(v, dtype=np.int32)  # noqa: E731
    return lib().mp2_prim_eri(_ptr(_f64(A)), a, _ptr(i(pa)), _ptr(_f64(B)), b, _ptr(i(pb)),
                              _ptr(_f64(C)), c, _ptr(i(pc)), _ptr(_f64(D)), d, _ptr(i(pd)))


def spinor_eri(oracle) -> np.ndarray:
    """V[k, l, m, n] = (kl|mn) over all spinors (chemists' notation)."""
    system = oracle.system
    n = system.n_orb
    U = real_function_coefficients(system)
    pairs = function_pairs(system.n_l)
    J = pair_coulomb_matrix(oracle, pairs)
    P, Q = pairs[:, 0], pairs[:, 1]
    # rho_kl = sum_c conj(phi_k^c) phi_l^c = sum_{P,Q} D^{kl}_{PQ} f_P f_Q; fold (P,Q) and (Q,P).
    D = np.einsum("cpk,cpl->klp", U[:, P, :].conj(), U[:, Q, :])
    off = P != Q
    D[:, :, off] += np.einsum("cpk,cpl->klp", U[:, Q[off], :].conj(), U[:, P[off], :])
    D = D.reshape(n * n, -1)
    V = D @ J @ D.T
    return V.reshape(n, n, n, n)


def mixed_function_pairs(n_l: int) -> np.ndarray:
    """Pairs (value function, gradient function) that occur in densities phi_k^dag alpha phi_l:
    alpha couples the large components (values) with the small ones (gradients)."""
    large = [4 * mu for mu in range(n_l)]
    small = [4 * mu + j for mu in range(n_l) for j in (1, 2, 3)]
    return np.array([(p, q) for p in large for q in small], dtype=np.int32)


def alpha_matrices() -> np.ndarray:
    """alpha_x, alpha_y, alpha_z in the component order (L-alpha, L-beta, S-alpha, S-beta):
    sigma_k in the off-diagonal 2 x 2 blocks."""
    A = np.zeros((3, 4, 4), dtype=np.complex128)
    for k in range(3):
        A[k, 0:2, 2:4] = PAULI[k]
        A[k, 2:4, 0:2] = PAULI[k]
    return A


def spinor_eri_gaunt(oracle) -> np.ndarray:
    """V[k, l, m, n] = (kl|mn) - 1/2 sum_j (kl|alpha_j . alpha_j|mn): the spinor integrals of the
    Coulomb + Gaunt interaction 1/r12 - alpha(1).alpha(2)/(2 r12) (Sec. II) in chemists' notation.
    The Gaunt densities rho^j_kl = phi_k^dag alpha_j phi_l are expanded over (value, gradient)
    function pairs and contracted with their Coulomb integrals."""
    system = oracle.system
    n = system.n_orb
    U = real_function_coefficients(system)
    pairs = mixed_function_pairs(system.n_l)
    J = pair_coulomb_matrix(oracle, pairs)
    P, Q = pairs[:, 0], pairs[:, 1]
    V = spinor_eri(oracle)
    for A in alpha_matrices():
        # f_P f_Q = f_Q f_P: the unordered pair collects both orderings.
        D = np.einsum("cpk,cd,dpl->klp", U[:, P, :].conj(), A, U[:, Q, :])
        D += np.einsum("cpk,cd,dpl->klp", U[:, Q, :].conj(), A, U[:, P, :])
        D = D.reshape(n * n, -1)
        V = V - 0.5 * (D @ J @ D.T).reshape(n, n, n, n)
    return V


def mp2_energy(system, V: np.ndarray) -> float:
    """E2 = 1/2 sum_{ij occ} sum_{ab vir} (ia|jb)[(ai|bj) - (bi|aj)] / (e_i + e_j - e_a - e_b)."""
    o, v = system.n_occ, system.n_vir
    e = system.eps
    occ = np.arange(o)
    vir = np.arange(o, o + v)
    ia_jb = V[np.ix_(occ, vir, occ, vir)]            # (ia|jb)[i,a,j,b]
    ai_bj = V[np.ix_(vir, occ, vir, occ)].transpose(1, 0, 3, 2)  # (ai|bj)[i,a,j,b]
    bi_aj = V[np.ix_(vir, occ, vir, occ)].transpose(1, 2, 3, 0)  # (bi|aj)[i,a,j,b]
    D = e[occ][:, None, None, None] + e[occ][None, None, :, None] - e[vir][None, :, None, None] \
        - e[vir][None, None, None, :]
    return float(np.real(0.5 * np.sum(ia_jb * (ai_bj - bi_aj) / D)))


def mp2_energy_eps_gradient(system, V: np.ndarray) -> np.ndarray:
    """dE2/d eps_k at fixed spinors: -1/2 sum N_ijab / D^2 * dD/d eps_k."""
    o, v = system.n_occ, system.n_vir
    e = system.eps
    occ = np.arange(o)
    vir = np.arange(o, o + v)
    N = V[np.ix_(occ, vir, occ, vir)] * (V[np.ix_(vir, occ, vir, occ)].transpose(1, 0, 3, 2)
                                         - V[np.ix_(vir, occ, vir, occ)].transpose(1, 2, 3, 0))
    D = e[occ][:, None, None, None] + e[occ][None, None, :, None] - e[vir][None, :, None, None] \
        - e[vir][None, None, None, :]
    W = np.real(-0.5 * N / D ** 2)
    grad = np.zeros(o + v)
    grad[:o] += W.sum(axis=(1, 2, 3)) + W.sum(axis=(0, 1, 3))
    grad[o:] -= W.sum(axis=(0, 2, 3)) + W.sum(axis=(0, 1, 2))
    return grad
