"""The seeded input generators: sizes, energy windows and exponent ranges of the
systems the tests and the benchmark draw (CPU only)."""
import numpy as np

import synthetic


def test_medium_and_soft_medium_share_the_workload_sizes():
    med = synthetic.make_system("medium")
    soft = synthetic.make_system("medium", soft=True)
    for s in (med, soft):
        assert s.n_l == 300 and s.n_occ == 80 and s.n_vir == 400 and len(s.centres) == 6
    # Soft: largest exponent within the weight function's reach, valence-like energies.
    assert med.shell_alpha.max() > 1000.0
    assert soft.shell_alpha.max() < 4.0
    assert soft.eps[:80].min() >= -2.0 and soft.eps[:80].max() <= -0.3
    assert soft.eps[80:].min() >= 0.1 and soft.eps[80:].max() <= 3.0
    # Orthonormal 4-component spinors in the 4-component metric.
    s_ll, s_ss = synthetic.overlap_matrices(soft)
    n = soft.n_l
    blocks = [soft.C[k * n:(k + 1) * n] for k in range(4)]
    M = sum(b.conj().T @ S @ b for b, S in zip(blocks, (s_ll, s_ll, s_ss, s_ss)))
    np.testing.assert_allclose(M, np.eye(soft.n_orb), atol=1e-9)


def test_generators_are_seeded():
    for kw in ({"config": "tiny"}, {"config": "size", "soft": True}):
        a = synthetic.make_system(**kw)
        assert a.digest() == synthetic.make_system(**kw).digest()
        assert synthetic.make_system(seed=7, **kw).digest() != a.digest()


def test_soft_size_units_keep_the_unit_sizes():
    for n in (1, 2):
        lit = synthetic.make_system("size", n_units=n)
        soft = synthetic.make_system("size", n_units=n, soft=True)
        assert soft.n_l == lit.n_l == 110 * n
        assert (soft.n_occ, soft.n_vir) == (lit.n_occ, lit.n_vir) == (40 * n, 180 * n)
        assert soft.shell_alpha.max() < 6.0 < lit.shell_alpha.max()
        assert soft.eps[:soft.n_occ].min() >= -2.0 and soft.eps[soft.n_occ:].max() <= 3.0
        # the weight function's most diffuse Gaussian lies inside 4x the most diffuse basis exponent
        assert soft.weight[:, [1, 3]].min() < 4.0 * soft.shell_alpha.min()
