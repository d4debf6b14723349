"""FP64 CPU oracle for the HISQ multi-rhs Dslash and conjugate gradient.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library and imports nothing from it.

Every function is a plain restatement of its definition in the paper
(Kaczmarek, Schmidt, Steinbrecher, Wagner, "Conjugate gradient solvers on
Intel Xeon Phi and NVIDIA GPUs", GPUHEP2014), in complex128, with numpy
array shifts standing in for the site loop. There is no blocking, fusion or
reordering beyond the definition.

Conventions (identical to the canonical input layout):

* full-lattice fields are arrays shaped (..., Lt, Lz, Ly, Lx, 3) for colour
  vectors and (4, Lt, Lz, Ly, Lx, 3, 3) for links; direction mu = 0, 1, 2, 3
  is x, y, z, t and lives on array axis ``3 - mu`` of a site grid;
* half-lattice (one parity) vectors are (n, V_h, 3): h = i // 2 over the
  sites of parity p = (x+y+z+t) % 2, i the lexicographic index
  x + Lx*(y + Ly*(z + Lz*t));
* U[mu][x] is the link x -> x+mu, N[mu][x] the link x -> x+3mu. Staggered
  phases, boundary signs and the Naik coefficient are part of the links.

Readings of the paper taken here (the paper is silent or garbled on them):

* Eq. 3 prints the direction sum as mu = 0..4; a 4-d lattice has four
  directions, read as mu = 0..3.
* Eq. 4 prints v_x in the last slot; read as v_x' like the other rhs.
* The fermion matrix is M = 2m + D (the paper never writes M); the CG system
  is the even-odd normal operator A_e = 4m^2 - D_eo D_oe at mu_chem = 0 and
  the full-lattice M(mu)^dag M(mu) otherwise, with M(mu)^dag = 2m - D(-mu).
* The chemical potential mu_chem multiplies the temporal hops: forward
  U-hop e^{+mu}, backward U^dag-hop e^{-mu}, forward Naik hop e^{+3mu},
  backward Naik hop e^{-3mu} (Eq. 1-2 need derivatives in mu).
* Solving for several vectors together (abstract, Sec. 2) is read as n
  independent CGs sharing each Dslash, not block CG.

Functions without a pin independent of this module are flagged in their
docstrings; every function below is pinned by tests in ``tests/``.
"""
from __future__ import annotations

import numpy as np

FLOAT = np.float64
COMPLEX = np.complex128


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------

def grid_shape(L):
    """Site grid shape (Lt, Lz, Ly, Lx) for L = (Lx, Ly, Lz, Lt)."""
    Lx, Ly, Lz, Lt = (int(a) for a in L)
    return (Lt, Lz, Ly, Lx)


def parity_mask(L, parity: int) -> np.ndarray:
    """Boolean grid of the sites with (x+y+z+t) % 2 == parity."""
    Lt, Lz, Ly, Lx = grid_shape(L)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2) == parity


def to_full(v_half: np.ndarray, L, parity: int) -> np.ndarray:
    """Embed (n, V_h, 3) one-parity vectors into (n, Lt, Lz, Ly, Lx, 3), zero elsewhere.

    Lexicographic order of the sites of one parity equals order in h = i // 2.
    """
    n = v_half.shape[0]
    out = np.zeros((n,) + grid_shape(L) + (3,), dtype=COMPLEX)
    out[:, parity_mask(L, parity)] = v_half
    return out


def to_half(v_full: np.ndarray, L, parity: int) -> np.ndarray:
    """Restrict (n, Lt, Lz, Ly, Lx, 3) full-lattice vectors to one parity: (n, V_h, 3)."""
    return np.ascontiguousarray(v_full[:, parity_mask(L, parity)])


def shift(field: np.ndarray, mu: int, hops: int, site_axis0: int) -> np.ndarray:
    """field(x + hops*mu_hat), periodic in every direction.

    ``site_axis0`` is the array axis of the t coordinate (the first site axis).
    """
    axis = site_axis0 + (3 - mu)
    return np.roll(field, -hops, axis=axis)


def _matvec(links_mu: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(Lt,Lz,Ly,Lx,3,3) x (n,Lt,Lz,Ly,Lx,3) -> (n,Lt,Lz,Ly,Lx,3): sum_j U_ij v_j."""
    return np.einsum("tzyxij,ntzyxj->ntzyxi", links_mu, v)


def _dagger(links_mu: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(links_mu, -1, -2))


# ----------------------------------------------------------------------------
# Dslash (Eq. 3) on a bundle of n right-hand sides (Eq. 4)
# ----------------------------------------------------------------------------

def dslash(U: np.ndarray, N: np.ndarray, v: np.ndarray, mu_chem: float = 0.0) -> np.ndarray:
    """Full-lattice HISQ Dslash applied to n vectors, Eq. 3 and Eq. 4.

    w(x) = sum_{mu=0..3} [ U_mu(x) v(x+mu) - U_mu(x-mu)^dag v(x-mu)
                          + N_mu(x) v(x+3mu) - N_mu(x-3mu)^dag v(x-3mu) ]

    with e^{+-mu_chem} on the temporal one-hop terms and e^{+-3 mu_chem} on the
    temporal Naik terms.

    U, N: (4, Lt, Lz, Ly, Lx, 3, 3) complex; v: (n, Lt, Lz, Ly, Lx, 3) complex.
    """
    v = np.asarray(v, dtype=COMPLEX)
    w = np.zeros_like(v)
    for mu in range(4):
        f1 = np.exp(mu_chem) if mu == 3 else 1.0
        f3 = np.exp(3.0 * mu_chem) if mu == 3 else 1.0
        # forward one-hop: U_mu(x) v(x+mu)
        w += f1 * _matvec(U[mu], shift(v, mu, +1, 1))
        # backward one-hop: U_mu(x-mu)^dag v(x-mu)
        w -= (1.0 / f1) * _matvec(_dagger(shift(U[mu], mu, -1, 0)), shift(v, mu, -1, 1))
        # forward Naik: N_mu(x) v(x+3mu)
        w += f3 * _matvec(N[mu], shift(v, mu, +3, 1))
        # backward Naik: N_mu(x-3mu)^dag v(x-3mu)
        w -= (1.0 / f3) * _matvec(_dagger(shift(N[mu], mu, -3, 0)), shift(v, mu, -3, 1))
    return w


def dslash_at_sites(U: np.ndarray, N: np.ndarray, v: np.ndarray, sites, mu_chem: float = 0.0):
    """Eq. 3 evaluated at single sites, one site at a time, for n vectors.

    ``sites`` is a list of (x, y, z, t); ``v`` is (n, Lt, Lz, Ly, Lx, 3).
    Returns (n, len(sites), 3). Used to check outputs of lattices too large
    for the array form at a sample of sites.
    """
    Lt, Lz, Ly, Lx = v.shape[1:5]
    ext = (Lx, Ly, Lz, Lt)
    out = np.zeros((v.shape[0], len(sites), 3), dtype=COMPLEX)
    for s, site in enumerate(sites):
        for mu in range(4):
            f1 = np.exp(mu_chem) if mu == 3 else 1.0
            f3 = np.exp(3.0 * mu_chem) if mu == 3 else 1.0

            def at(hops):
                c = list(site)
                c[mu] = (c[mu] + hops) % ext[mu]
                return (c[3], c[2], c[1], c[0])

            here = at(0)
            out[:, s] += f1 * (v[(slice(None),) + at(+1)] @ U[mu][here].T)
            out[:, s] -= (1.0 / f1) * (v[(slice(None),) + at(-1)] @ np.conj(U[mu][at(-1)]))
            out[:, s] += f3 * (v[(slice(None),) + at(+3)] @ N[mu][here].T)
            out[:, s] -= (1.0 / f3) * (v[(slice(None),) + at(-3)] @ np.conj(N[mu][at(-3)]))
    return out


def dslash_parity(U, N, v_half: np.ndarray, L, parity: int, mu_chem: float = 0.0) -> np.ndarray:
    """D_{p,1-p}: maps (n, V_h, 3) vectors of parity 1-p to parity p.

    Every one- and three-hop flips parity, so D_{p,1-p} is the block of D
    that takes the opposite parity to p.
    """
    v_full = to_full(v_half, L, 1 - parity)
    return to_half(dslash(U, N, v_full, mu_chem), L, parity)


# ----------------------------------------------------------------------------
# Fermion matrix and CG systems
# ----------------------------------------------------------------------------

def apply_M(U, N, v, mass: float, mu_chem: float = 0.0):
    """M(mu) v = 2m v + D(mu) v on the full lattice."""
    return 2.0 * mass * v + dslash(U, N, v, mu_chem)


def apply_Mdag(U, N, v, mass: float, mu_chem: float = 0.0):
    """M(mu)^dag v = 2m v - D(-mu) v, because D(mu)^dag = -D(-mu)."""
    return 2.0 * mass * v - dslash(U, N, v, -mu_chem)


def apply_MdagM(U, N, v, mass: float, mu_chem: float = 0.0):
    """Full-lattice normal operator M(mu)^dag M(mu) v."""
    return apply_Mdag(U, N, apply_M(U, N, v, mass, mu_chem), mass, mu_chem)


def apply_dM_dmu(U, N, v, mu_chem: float = 0.0):
    """dM/dmu v = dD/dmu v: the temporal terms of Eq. 3 differentiated in mu.

    d/dmu of  e^{mu} U_3(x) v(x+t) - e^{-mu} U_3(x-t)^dag v(x-t)
            + e^{3mu} N_3(x) v(x+3t) - e^{-3mu} N_3(x-3t)^dag v(x-3t).
    """
    return apply_dnM_dmun(U, N, v, mu_chem, 1)


def apply_dnM_dmun(U, N, v, mu_chem: float, order: int):
    """d^k M / dmu^k v for k = order >= 1 (the mu-derivatives that enter Eq. 1-2).

    Only the temporal terms of Eq. 3 depend on mu; the k-th derivative of
    e^{+-mu} is (+-1)^k e^{+-mu} and of e^{+-3mu} is (+-3)^k e^{+-3mu}.
    """
    v = np.asarray(v, dtype=COMPLEX)
    k = int(order)
    mu = 3
    w = np.exp(mu_chem) * _matvec(U[mu], shift(v, mu, +1, 1))
    w -= (-1.0) ** k * np.exp(-mu_chem) * _matvec(_dagger(shift(U[mu], mu, -1, 0)), shift(v, mu, -1, 1))
    w += 3.0 ** k * np.exp(3.0 * mu_chem) * _matvec(N[mu], shift(v, mu, +3, 1))
    w -= (-3.0) ** k * np.exp(-3.0 * mu_chem) * _matvec(_dagger(shift(N[mu], mu, -3, 0)), shift(v, mu, -3, 1))
    return w


def apply_Minv(U, N, v, mass: float, mu_chem: float = 0.0, tol: float = 1e-13):
    """M(mu)^-1 v = (M^dag M)^-1 M^dag v on the full lattice (CG on the normal equations)."""
    x, _ = cg(lambda q: apply_MdagM(U, N, q, mass, mu_chem), apply_Mdag(U, N, v, mass, mu_chem), tol)
    return x


def trace_word_bilinear(U, N, eta, mass: float, mu_chem: float, orders, tol: float = 1e-13):
    """eta_k^dag  d^{n1}M M^-1 d^{n2}M M^-1 ... d^{nj}M M^-1  eta_k, per rhs k (Eq. 2).

    ``orders`` = (n1, ..., nj); each factor d^{n}M M^-1 is applied from the
    right. The mean over noise vectors with E[eta eta^dag] = 1 estimates the
    trace of the word.
    """
    v = np.asarray(eta, dtype=COMPLEX)
    for order in reversed(list(orders)):
        v = apply_Minv(U, N, v, mass, mu_chem, tol)
        v = apply_dnM_dmun(U, N, v, mu_chem, order)
    axes = tuple(range(1, v.ndim))
    return np.sum(np.conj(eta) * v, axis=axes)


def apply_Ae(U, N, v_half, L, mass: float):
    """Even-odd normal operator A_e v = 4m^2 v - D_eo D_oe v on even sites."""
    t_odd = dslash_parity(U, N, v_half, L, 1)
    return 4.0 * mass * mass * v_half - dslash_parity(U, N, t_odd, L, 0)


def cg(apply_A, b: np.ndarray, tol: float, maxiter: int = 100000):
    """Textbook Hestenes-Stiefel CG, run independently for each of the n rhs.

    Solves A x = b for Hermitian positive definite A from x0 = 0. Each rhs has
    its own alpha_k, beta_k and stops when its iterated residual satisfies
    ||r_k|| / ||b_k|| <= tol; a stopped rhs is frozen. ``b`` has the rhs on
    axis 0. Returns (x, iterations per rhs).
    """
    b = np.asarray(b, dtype=COMPLEX)
    n = b.shape[0]
    axes = tuple(range(1, b.ndim))

    def dot(a, c):
        return np.sum(np.conj(a) * c, axis=axes)

    def bcast(s):
        return s.reshape((n,) + (1,) * (b.ndim - 1))

    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = dot(r, r).real
    bb = rr.copy()
    active = bb > 0.0
    iters = np.zeros(n, dtype=np.int64)
    for _ in range(maxiter):
        if not np.any(active):
            break
        Ap = apply_A(p)
        pAp = dot(p, Ap).real
        alpha = np.where(active, rr / np.where(active, pAp, 1.0), 0.0)
        x = x + bcast(alpha) * p
        r = r - bcast(alpha) * Ap
        rr_new = dot(r, r).real
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        p = np.where(bcast(active), r + bcast(beta) * p, p)
        rr = np.where(active, rr_new, rr)
        iters += active
        active = active & (np.sqrt(rr) > tol * np.sqrt(bb))
    return x, iters


def true_relative_residual(apply_A, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """||b - A x|| / ||b|| per rhs (rhs on axis 0), all in FP64."""
    r = np.asarray(b, dtype=COMPLEX) - apply_A(np.asarray(x, dtype=COMPLEX))
    axes = tuple(range(1, r.ndim))
    num = np.sqrt(np.sum(np.abs(r) ** 2, axis=axes))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=axes))
    return num / np.where(den > 0, den, 1.0)


def dense_matrix(apply_op, shape_one) -> np.ndarray:
    """Dense matrix of a linear operator by applying it to every unit vector.

    ``shape_one`` is the shape of one vector without the rhs axis. Only for
    tiny lattices (the 4^4 even-odd system is 384 x 384).
    """
    dim = int(np.prod(shape_one))
    cols = []
    batch = 96
    for start in range(0, dim, batch):
        stop = min(dim, start + batch)
        e = np.zeros((stop - start, dim), dtype=COMPLEX)
        e[np.arange(stop - start), np.arange(start, stop)] = 1.0
        out = apply_op(e.reshape((stop - start,) + tuple(shape_one)))
        cols.append(out.reshape(stop - start, dim))
    return np.concatenate(cols, axis=0).T


# ----------------------------------------------------------------------------
# Link compression (18 -> 12 or 14 reals), Sec. 1: fewer stored reals per
# link, possible for the HISQ Naik links (9 or 13/14 reals in the paper)
# ----------------------------------------------------------------------------
#
# The paper names the float counts but not the encodings. Readings used here:
#   r14: store rows 1 and 2 (12 reals) and one complex z (2 reals); row 3 is
#        z * conj(row1 x row2). Exact for every link c * W with W in U(3) and
#        c real, z = det(W) / c.
#   r12: store rows 1 and 2; row 3 = (sigma / s) * conj(row1 x row2), where
#        sigma = eta_mu(x) * bc(x, mu) is the staggered sign of that link
#        recomputed from coordinates and s is one real scale per field. Exact
#        for links s * sigma * SU(3).

def _cross_conj(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """conj(a x b) for complex 3-vectors on the last axis."""
    c = np.empty(np.broadcast_shapes(a.shape, b.shape), dtype=COMPLEX)
    c[..., 0] = a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1]
    c[..., 1] = a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2]
    c[..., 2] = a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]
    return np.conj(c)


def link_sign(L, hop: int) -> np.ndarray:
    """sigma_mu(x) = eta_mu(x) * bc(x, mu) for hops of length ``hop``, shape (4, Lt, Lz, Ly, Lx).

    eta_mu(x) = (-1)^(x_0+...+x_{mu-1}); bc = -1 for temporal hops that wrap
    from t = Lt-1 to t = 0 (antiperiodic fermion), else +1.
    """
    Lt, Lz, Ly, Lx = grid_shape(L)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    sig = np.ones((4, Lt, Lz, Ly, Lx), dtype=FLOAT)
    sig[1] = np.where(x % 2 == 0, 1.0, -1.0)
    sig[2] = np.where((x + y) % 2 == 0, 1.0, -1.0)
    sig[3] = np.where((x + y + z) % 2 == 0, 1.0, -1.0)
    sig[3] *= np.where(t + hop >= Lt, -1.0, 1.0)
    return sig


def compress_r14(links: np.ndarray) -> np.ndarray:
    """Links (..., 3, 3) -> (..., 14) reals: rows 1, 2 and z with row3 = z conj(row1 x row2).

    z is taken from the largest component of conj(row1 x row2).
    """
    a, b, c = links[..., 0, :], links[..., 1, :], links[..., 2, :]
    cc = _cross_conj(a, b)
    k = np.argmax(np.abs(cc), axis=-1)
    num = np.take_along_axis(c, k[..., None], axis=-1)[..., 0]
    den = np.take_along_axis(cc, k[..., None], axis=-1)[..., 0]
    z = num / den
    out = np.empty(links.shape[:-2] + (14,), dtype=FLOAT)
    out[..., 0:6] = a.view(FLOAT).reshape(a.shape[:-1] + (6,))
    out[..., 6:12] = b.view(FLOAT).reshape(b.shape[:-1] + (6,))
    out[..., 12] = z.real
    out[..., 13] = z.imag
    return out


def reconstruct_r14(packed: np.ndarray) -> np.ndarray:
    """(..., 14) reals -> (..., 3, 3) complex links, row3 = z conj(row1 x row2)."""
    a = packed[..., 0:6:2] + 1j * packed[..., 1:6:2]
    b = packed[..., 6:12:2] + 1j * packed[..., 7:12:2]
    z = packed[..., 12] + 1j * packed[..., 13]
    out = np.empty(packed.shape[:-1] + (3, 3), dtype=COMPLEX)
    out[..., 0, :] = a
    out[..., 1, :] = b
    out[..., 2, :] = z[..., None] * _cross_conj(a, b)
    return out


def compress_r12(links: np.ndarray) -> np.ndarray:
    """(..., 3, 3) -> (..., 12) reals: rows 1 and 2."""
    a, b = links[..., 0, :], links[..., 1, :]
    out = np.empty(links.shape[:-2] + (12,), dtype=FLOAT)
    out[..., 0:6] = np.ascontiguousarray(a).view(FLOAT).reshape(a.shape[:-1] + (6,))
    out[..., 6:12] = np.ascontiguousarray(b).view(FLOAT).reshape(b.shape[:-1] + (6,))
    return out


def reconstruct_r12(packed: np.ndarray, L, scale: float, hop: int = 1) -> np.ndarray:
    """(4, Lt, Lz, Ly, Lx, 12) -> links with row3 = (sigma/s) conj(row1 x row2)."""
    a = packed[..., 0:6:2] + 1j * packed[..., 1:6:2]
    b = packed[..., 6:12:2] + 1j * packed[..., 7:12:2]
    sig = link_sign(L, hop)
    out = np.empty(packed.shape[:-1] + (3, 3), dtype=COMPLEX)
    out[..., 0, :] = a
    out[..., 1, :] = b
    out[..., 2, :] = (sig / scale)[..., None] * _cross_conj(a, b)
    return out


# ----------------------------------------------------------------------------
# Cost model of Table 1 (Sec. 1)
# ----------------------------------------------------------------------------

MATVEC_FLOPS = 9 * 6 + 6 * 2          # 9 complex mul + 6 complex add = 66
DSLASH_FLOPS_PER_SITE_RHS = 16 * MATVEC_FLOPS + 15 * 6   # 16 mat-vecs, 15 vector adds = 1146


def dslash_flops(n: int) -> int:
    """Flops of one Dslash per output site for n rhs: 16 mat-vecs and 15 adds per rhs."""
    return DSLASH_FLOPS_PER_SITE_RHS * int(n)


def dslash_bytes_no_reuse(n: int, naik_reals: int, fat_reals: int = 18,
                          bytes_per_real: int = 4) -> int:
    """Bytes per output site without neighbour reuse (the model behind Table 1).

    Eight fat and eight Naik links are read per site; every rhs reads its 16
    neighbour vectors and writes one result (6 reals each).
    """
    links = 8 * fat_reals + 8 * naik_reals
    spinors = int(n) * (16 * 6 + 6)
    return (links + spinors) * bytes_per_real


def dslash_intensity(n: int, naik_reals: int) -> float:
    """Flop per byte of the single-precision Dslash, Table 1."""
    return dslash_flops(n) / dslash_bytes_no_reuse(n, naik_reals)


def dslash_bytes_algorithmic(n: int, fat_reals: int, naik_reals: int,
                             link_bytes_per_real: int, spinor_bytes_per_real: int) -> int:
    """Minimum bytes per output site of one parity Dslash.

    Every link is read once (8 fat + 8 Naik per output site, since each
    parity's output sites own the forward links of their parity and the
    backward links of the other), every input vector is read once and every
    output vector is written once (6 reals in + 6 reals out per rhs).
    """
    return (8 * (fat_reals + naik_reals) * link_bytes_per_real
            + 12 * int(n) * spinor_bytes_per_real)
