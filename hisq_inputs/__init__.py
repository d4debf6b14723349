"""Seeded synthetic inputs for the HISQ multi-rhs CG: gauge links and sources.

This module is shared by the FP64 oracle and the GPU path. It builds inputs
only; it holds none of the Dslash / CG arithmetic.

The paper measures on HotQCD gauge ensembles (Sec. 3, Fig. 4), which are not
available. Synthetic links stand in for them:

* fat links   U_mu(x) = 0.9    * eta_mu(x) * bc_U(x, mu) * G,  G Haar SU(3)
* Naik links  N_mu(x) = -1/24  * eta_mu(x) * bc_N(x, mu) * W,  W Haar U(3)

with the staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) and an
antiperiodic temporal boundary for the fermion folded into the links: the
sign flips on every hop that wraps from t = Lt-1 to t = 0 (U_3(x) with
x_t = Lt-1, N_3(x) with x_t >= Lt-3).

Haar sampling follows Mezzadri, "How to generate random matrices from the
classical compact groups" (Notices AMS 54, 2007): orthonormalise a complex
Ginibre matrix so that R has a positive real diagonal. Gram-Schmidt on the
columns gives exactly that Q. SU(3) additionally divides by det^(1/3).

Sources: complex Z2 noise (+-1 +- i)/sqrt(2) per colour component with
independent signs, or Gaussian complex noise with Re, Im ~ N(0, 1/2).

Canonical layouts (complex128, C order):

* links    [4][Lt][Lz][Ly][Lx][3][3]  == [4][V][3][3], lexicographic site
           i = x + Lx*(y + Ly*(z + Lz*t)), row-major colour; U[mu][x] is
           the link x -> x+mu, N[mu][x] the link x -> x+3mu.
* spinors  half lattice [V_h][3] per rhs: h = i // 2 over the sites of one
           parity (x+y+z+t) % 2, in lexicographic order.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_volume", "site_coords", "staggered_eta", "antiperiodic_sign",
    "haar_u3", "haar_su3", "hisq_links", "free_field_links",
    "z2_source", "gaussian_source", "random_su3_field",
]

FAT_SCALE = 0.9
NAIK_SCALE = -1.0 / 24.0


def lattice_volume(L) -> int:
    Lx, Ly, Lz, Lt = (int(a) for a in L)
    return Lx * Ly * Lz * Lt


def _check_lattice(L):
    if len(L) != 4:
        raise ValueError("lattice must have four extents (Lx, Ly, Lz, Lt)")
    for a in L:
        if int(a) < 4 or int(a) % 2:
            raise ValueError(f"every extent must be even and >= 4, got {tuple(L)}")


def site_coords(L):
    """Integer coordinate grids (x, y, z, t), each shaped (Lt, Lz, Ly, Lx)."""
    Lx, Ly, Lz, Lt = (int(a) for a in L)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return x, y, z, t


def staggered_eta(L):
    """eta_mu(x) = (-1)^(sum_{nu<mu} x_nu), shaped (4, Lt, Lz, Ly, Lx)."""
    x, y, z, t = site_coords(L)
    eta = np.empty((4,) + x.shape, dtype=np.float64)
    eta[0] = 1.0
    eta[1] = (-1.0) ** x
    eta[2] = (-1.0) ** (x + y)
    eta[3] = (-1.0) ** (x + y + z)
    return eta


def antiperiodic_sign(L, hop: int):
    """Sign of the link x -> x + hop*mu for an antiperiodic fermion in t.

    Returns shape (4, Lt, Lz, Ly, Lx); only mu = 3 hops that cross t = Lt-1 -> 0
    are -1.
    """
    _, _, _, t = site_coords(L)
    Lt = int(L[3])
    s = np.ones((4,) + t.shape, dtype=np.float64)
    s[3] = np.where(t + hop >= Lt, -1.0, 1.0)
    return s


def _ginibre(rng: np.random.Generator, count: int) -> np.ndarray:
    re = rng.standard_normal((count, 3, 3))
    im = rng.standard_normal((count, 3, 3))
    return (re + 1j * im) / np.sqrt(2.0)


def _orthonormalise_columns(z: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt on the three columns: Q of z = QR with diag(R) > 0."""
    q = z.copy()
    for j in range(3):
        for k in range(j):
            proj = np.einsum("ni,ni->n", q[:, :, k].conj(), q[:, :, j])
            q[:, :, j] -= proj[:, None] * q[:, :, k]
        nrm = np.sqrt(np.einsum("ni,ni->n", q[:, :, j].conj(), q[:, :, j]).real)
        q[:, :, j] /= nrm[:, None]
    return q


def haar_u3(rng: np.random.Generator, count: int) -> np.ndarray:
    """count Haar-random U(3) matrices, shape (count, 3, 3)."""
    return _orthonormalise_columns(_ginibre(rng, count))


def haar_su3(rng: np.random.Generator, count: int) -> np.ndarray:
    """count Haar-random SU(3) matrices: U(3) divided by a cube root of det."""
    q = haar_u3(rng, count)
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def hisq_links(L, seed: int, fat_scale: float = FAT_SCALE,
               naik_scale: float = NAIK_SCALE):
    """Synthetic HISQ fat links U and Naik links N, canonical complex128 layout.

    Generation order with numpy Generator(PCG64(seed)): U[mu][site] in
    lexicographic order, then N[mu][site].
    """
    _check_lattice(L)
    Lx, Ly, Lz, Lt = (int(a) for a in L)
    V = lattice_volume(L)
    shape = (4, Lt, Lz, Ly, Lx, 3, 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    G = haar_su3(rng, 4 * V).reshape(shape)
    W = haar_u3(rng, 4 * V).reshape(shape)
    eta = staggered_eta(L)
    U = (fat_scale * eta * antiperiodic_sign(L, 1))[..., None, None] * G
    N = (naik_scale * eta * antiperiodic_sign(L, 3))[..., None, None] * W
    return np.ascontiguousarray(U), np.ascontiguousarray(N)


def free_field_links(L, c1: float = 9.0 / 8.0, c3: float = -1.0 / 24.0):
    """Unit-colour links with phases and boundary signs folded in.

    U_mu(x) = c1 eta_mu(x) bc_U(x,mu) 1 and N_mu(x) = c3 eta_mu(x) bc_N(x,mu) 1.
    """
    _check_lattice(L)
    eta = staggered_eta(L)
    eye = np.eye(3, dtype=np.complex128)
    U = (c1 * eta * antiperiodic_sign(L, 1))[..., None, None] * eye
    N = (c3 * eta * antiperiodic_sign(L, 3))[..., None, None] * eye
    return np.ascontiguousarray(U), np.ascontiguousarray(N)


def random_su3_field(L, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    Lx, Ly, Lz, Lt = (int(a) for a in L)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = haar_su3(rng, lattice_volume(L))
    return g.reshape(Lt, Lz, Ly, Lx, 3, 3)


def z2_source(L, n: int, seed: int) -> np.ndarray:
    """n complex Z2 sources on one parity: shape (n, V_h, 3) complex128."""
    _check_lattice(L)
    vh = lattice_volume(L) // 2
    rng = np.random.Generator(np.random.PCG64(seed))
    sr = rng.integers(0, 2, size=(n, vh, 3)) * 2 - 1
    si = rng.integers(0, 2, size=(n, vh, 3)) * 2 - 1
    return (sr + 1j * si) / np.sqrt(2.0)


def gaussian_source(L, n: int, seed: int) -> np.ndarray:
    """n Gaussian complex sources on one parity: Re, Im ~ N(0, 1/2)."""
    _check_lattice(L)
    vh = lattice_volume(L) // 2
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((n, vh, 3))
    im = rng.standard_normal((n, vh, 3))
    return (re + 1j * im) / np.sqrt(2.0)
