"""CPU check of the operator algebra the tensor-core trace epilogue relies on for the
Gaunt and Breit terms (Sec. II): a lane-by-lane model of the eight lanes (e, c) of one
pair of pairs, written in the epilogue's order, against the operator traces of the
trace form written out (direct tr[G-31 O_A G+13 O_B] tr[G-42 O_A G+24 O_B], exchange
tr[G-31 O_A G+14 O_B G-42 O_A G+23 O_B], summed with c_A c_B).

What it fixes: M_AB = O_A G- O_B carries both operators (Hermitian alpha), the row maps
c -> c^3 (alpha_x, alpha_y) and c -> c^2 (alpha_z) with their phases, the half-split dot
products that give all four column operators, the halving exchanges over the four lanes
of an electron (slot k = 4A + B, lane c keeping A = 2 (c & 1) + (c >> 1)), the merged
alpha_x / alpha_y exchange product (1 - s_c s_c''), and alpha.n as a linear combination.
Random complex blocks, no GPU.
"""
import numpy as np
import pytest

SIGMA = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]


def alpha(v):
    s = sum(v[k] * SIGMA[k] for k in range(3))
    o = np.zeros((4, 4), complex)
    o[:2, 2:] = s
    o[2:, :2] = s
    return o


def coef(k):
    return 1.0 if k == 0 else -0.5


def traces(breit, G1, G2, P11, P22, P12, P21, n_p, n_q):
    """-1/2 (D - X) written out; G1 = G-(1p,1q), G2 = G-(2p,2q), P11 = G+(1p,1q),
    P22 = G+(2p,2q), P12 = G+(1p,2q), P21 = G+(2p,1q)."""
    def terms(n):
        t = [(np.eye(4), 1.0)] + [(alpha(np.eye(3)[k]), -0.5) for k in range(3)]
        return t + [(alpha(n), -0.5)] if breit else t
    d = x = 0.0
    for OA, cA in terms(n_p):
        for OB, cB in terms(n_q):
            d += cA * cB * np.trace(G1.conj().T @ OA @ P11 @ OB) * np.trace(G2.conj().T @ OA @ P22 @ OB)
            x += cA * cB * np.trace(G1.conj().T @ OA @ P12 @ OB @ G2.conj().T @ OA @ P21 @ OB)
    return (-0.5 * (d - x)).real


def row_dots(R, Y):
    """h_B = sum_d conj((R O_B)_d) Y_d, B = 0, x, y, z, from half-split dot products."""
    r = np.conj(R)
    f = np.sum(r * Y)
    ex, ox = r[3] * Y[0] + r[1] * Y[2], r[2] * Y[1] + r[0] * Y[3]
    ez, oz = r[2] * Y[0] + r[0] * Y[2], r[3] * Y[1] + r[1] * Y[3]
    return np.array([f, ex + ox, 1j * (ox - ex), ez - oz])


def lanes(breit, own, dia, off, n_p, n_q, parity_phase=True):
    """The epilogue's value for one pair of pairs: own[e] = G-(xe, ye), dia[e] = G+(xe, ye),
    off[e] = G+(xe, y(1-e)); lane 4e + c holds row c of each."""
    v = np.zeros((8, 16), complex)
    tn = np.zeros((8, 5), complex)
    for l in range(8):
        e, c = l >> 2, l & 3
        sc = -1.0 if c & 1 else 1.0
        H0, H3, H2 = (row_dots(own[e][c ^ k], dia[e][c]) for k in (0, 3, 2))
        v[l] = np.concatenate([H0, H3, 1j * (sc if parity_phase else 1.0) * H3, sc * H2])
        if breit:
            tn[l, :4] = n_p[0] * v[l, 4:8] + n_p[1] * v[l, 8:12] + n_p[2] * v[l, 12:16]
            tn[l, 4] = n_q @ tn[l, 1:4]
    # halving exchanges over the lanes c of each electron
    half = np.zeros((8, 8), complex)
    for l in range(8):
        keep = v[l, 8:] if l & 1 else v[l, :8]
        p = l ^ 1
        half[l] = keep + (v[p, :8] if p & 1 else v[p, 8:])
    quarter = np.zeros((8, 4), complex)
    for l in range(8):
        keep = half[l, 4:] if l & 2 else half[l, :4]
        p = l ^ 2
        quarter[l] = keep + (half[p, :4] if p & 2 else half[p, 4:])
    tn_sum = np.array([tn[l] + tn[l ^ 1] + tn[l ^ 2] + tn[l ^ 3] for l in range(8)])
    total = 0.0
    for l in range(8):
        e, c = l >> 2, l & 3
        A = 2 * (c & 1) + (c >> 1)
        T, W = quarter[l], quarter[l ^ 4]
        dl = coef(A) * sum(coef(B) * (T[B] * W[B]).real for B in range(4))
        if breit:
            dl += coef(A) * -0.5 * ((n_q @ T[1:]) * (n_q @ W[1:])).real
            dl += 0.25 * -0.5 * sum(coef(B) * (tn_sum[l, B] * tn_sum[l ^ 4, B]).real for B in range(5))
        dl *= 0.5
        xl = 0.0
        sc = -1.0 if c & 1 else 1.0
        for s in range(2):
            cpp = (c + s) & 3 if e == 0 else (c + 2 - s) & 3
            ro = off[1 - e][cpp]
            sp = -1.0 if cpp & 1 else 1.0
            H = {k: row_dots(own[e][c ^ k], ro) for k in (0, 3, 2)}
            G = {k: row_dots(own[1 - e][cpp ^ k], off[e][c]) for k in (0, 3, 2)}

            def prod(g, h):
                out = g[0] * h[0] - 0.5 * np.sum(g[1:] * h[1:])
                if breit:
                    out += -0.5 * (n_q @ g[1:]) * (n_q @ h[1:])
                return out.real
            xl += prod(G[0], H[0]) - 0.5 * (1 - sc * sp) * prod(G[3], H[3]) - 0.5 * sc * sp * prod(G[2], H[2])
            if breit:
                a1 = (n_p[0] + 1j * n_p[1] * sp) * G[3] + n_p[2] * sp * G[2]
                a2 = (n_p[0] + 1j * n_p[1] * sc) * H[3] + n_p[2] * sc * H[2]
                xl += -0.5 * prod(a1, a2)
        total += dl - xl
    return -0.5 * total


@pytest.mark.parametrize("breit", [False, True])
def test_lane_model_equals_operator_traces(breit):
    rng = np.random.default_rng(2203)
    for _ in range(25):
        blocks = [rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for _ in range(6)]
        G1, G2, P11, P22, P12, P21 = blocks
        n_p, n_q = (u / np.linalg.norm(u) for u in rng.normal(size=(2, 3)))
        want = traces(breit, G1, G2, P11, P22, P12, P21, n_p, n_q)
        got = lanes(breit, [G1, G2], [P11, P22], [P12, P21], n_p, n_q)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_lane_model_sees_a_dropped_phase():
    """A plausible slip, alpha_y's row phase taken as i on every row (its sign alternates with
    the row parity), changes the value: the check is sensitive to the phases.  (A sign flip
    of a whole operator is not such a slip: the interaction holds O_A at both points.)"""
    rng = np.random.default_rng(5632)
    G1, G2, P11, P22, P12, P21 = [rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)) for _ in range(6)]
    n = np.array([0.0, 0.0, 1.0])
    want = traces(False, G1, G2, P11, P22, P12, P21, n, n)
    good = lanes(False, [G1, G2], [P11, P22], [P12, P21], n, n)
    bad = lanes(False, [G1, G2], [P11, P22], [P12, P21], n, n, parity_phase=False)
    assert good == pytest.approx(want, rel=1e-12)
    assert abs(bad - want) > 1e-3 * abs(want)
