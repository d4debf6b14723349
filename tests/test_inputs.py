"""The seeded input generators: the distributions the synthetic workloads claim.

Haar U(3) and SU(3) by orthonormalised Ginibre matrices, the fat and Naik
link scales, complex Z2 and Gaussian sources. Pure numpy, no GPU.
"""
import numpy as np

import hisq_inputs as gen


def test_haar_matrices_are_unitary_with_the_right_determinant():
    rng = np.random.Generator(np.random.PCG64(7))
    u = gen.haar_u3(rng, 2000)
    s = gen.haar_su3(rng, 2000)
    eye = np.eye(3)
    for m in (u, s):
        assert np.allclose(np.einsum("kij,kil->kjl", m.conj(), m), eye, atol=1e-13)
    assert np.allclose(np.abs(np.linalg.det(u)), 1.0, atol=1e-13)
    assert np.allclose(np.linalg.det(s), 1.0, atol=1e-12)


def test_haar_moments():
    """Under Haar measure E|U_ij|^2 = 1/3 and E|U_ij|^4 = 1/6 for U(3); the
    phase of det U is uniform. 20000 samples: 5-sigma bands."""
    rng = np.random.Generator(np.random.PCG64(11))
    u = gen.haar_u3(rng, 20000)
    a2 = np.abs(u) ** 2
    assert abs(a2.mean() - 1.0 / 3.0) < 5 * a2.std() / np.sqrt(a2.size)
    a4 = a2 ** 2
    assert abs(a4.mean() - 1.0 / 6.0) < 5 * a4.std() / np.sqrt(a4.size)
    ph = np.angle(np.linalg.det(u))
    assert abs(np.mean(np.cos(ph))) < 5 / np.sqrt(ph.size)
    assert abs(np.mean(np.sin(ph))) < 5 / np.sqrt(ph.size)


def test_link_scales_and_phases():
    L = (4, 4, 4, 6)
    U, N = gen.hisq_links(L, seed=3)
    # fat links are 0.9 x (sign) x SU(3), Naik links -1/24 x (sign) x U(3)
    fu = U.reshape(-1, 3, 3) / gen.FAT_SCALE
    fn = N.reshape(-1, 3, 3) / gen.NAIK_SCALE
    eye = np.eye(3)
    assert np.allclose(np.einsum("kij,kil->kjl", fu.conj(), fu), eye, atol=1e-12)
    assert np.allclose(np.einsum("kij,kil->kjl", fn.conj(), fn), eye, atol=1e-12)
    assert np.allclose(np.abs(np.linalg.det(fu)), 1.0, atol=1e-12)
    d = np.linalg.det(fu).real
    assert np.allclose(np.abs(d), 1.0, atol=1e-12)     # det = staggered sign x boundary sign
    assert np.all(np.abs(np.linalg.det(fu).imag) < 1e-12)


def test_sources():
    L = (4, 4, 4, 4)
    z = gen.z2_source(L, 3, seed=1)
    assert z.shape == (3, 128, 3)
    assert np.allclose(np.abs(z.real), 1 / np.sqrt(2)) and np.allclose(np.abs(z.imag), 1 / np.sqrt(2))
    g = gen.gaussian_source(L, 200, seed=2)
    assert abs(g.real.var() - 0.5) < 0.02 and abs(g.imag.var() - 0.5) < 0.02
    assert abs(g.mean()) < 0.02
    # seeded: the same seed gives the same vectors, another seed different ones
    assert np.array_equal(gen.z2_source(L, 3, seed=1), z)
    assert not np.array_equal(gen.z2_source(L, 3, seed=2), z)
