"""Aggregation-based coarse operator (oracle; test infrastructure only).

Sec. 2.2: test vectors are cut over the aggregates; with the spin-preserving
construction each aggregate carries 2*n_tv variables (one orthonormal set of
n_tv vectors per chirality half), and the coarse operator is the Galerkin
product D_c = P^H D P, a nearest-neighbour stencil on the coarse lattice.

Test vectors follow the synthetic recipe: every seeded complex-Gaussian x0 is
refined by one unrestarted 20-step GMRES cycle on D x = 0, i.e. x minimises
||D x|| over x0 + K_20(D, D x0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fine
from .lattice import coordinates, neighbours, volume


def arnoldi_mgs(apply, r0: np.ndarray, steps: int):
    """Alg. 1 with the modified Gram-Schmidt variant of Sec. 3.1.

    Returns (V, Hbar, beta) with V of shape (N, j+1), Hbar (j+1, j), j <= steps
    (j < steps only on breakdown h_{j+1,j} = 0).
    """
    beta = np.linalg.norm(r0)
    V = [r0 / beta]
    H = np.zeros((steps + 1, steps), dtype=complex)
    for j in range(steps):
        w = apply(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return np.array(V).T, H[: j + 2, : j + 1], beta
        V.append(w / H[j + 1, j])
    return np.array(V).T, H, beta


def refine_test_vector(D: sp.spmatrix, x0: np.ndarray, iters: int = 20) -> np.ndarray:
    """x = x0 + V z with z = argmin ||beta e1 - Hbar z||, Krylov space of D from r0 = -D x0."""
    r0 = -(D @ x0)
    V, H, beta = arnoldi_mgs(lambda v: D @ v, r0, iters)
    m = H.shape[1]
    e1 = np.zeros(m + 1, dtype=complex)
    e1[0] = beta
    z = np.linalg.lstsq(H, e1, rcond=None)[0]
    return x0 + V[:, :m] @ z


def mgs_orthonormalise(T: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt on the columns of T, in column order."""
    Q = np.array(T, dtype=complex, copy=True)
    for k in range(Q.shape[1]):
        for i in range(k):
            Q[:, k] -= np.vdot(Q[:, i], Q[:, k]) * Q[:, i]
        Q[:, k] /= np.linalg.norm(Q[:, k])
    return Q


def coarse_dims(fine_dims):
    return tuple(v // 2 for v in fine_dims)


def aggregate_of(fine_dims) -> np.ndarray:
    """Coarse site of every fine site for 2^4 aggregates."""
    c = coordinates(fine_dims) // 2
    cd = coarse_dims(fine_dims)
    return c[:, 0] + cd[0] * (c[:, 1] + cd[1] * (c[:, 2] + cd[2] * c[:, 3]))


def prolongator(test_vectors: np.ndarray, fine_dims) -> sp.csr_matrix:
    """Sparse P of shape (12 V_f, 2 nv V_c).

    Coarse dof (a, h, k) = a*2nv + h*nv + k: test vector k restricted to the
    16 sites of aggregate a, spins of chirality half h (h = 0: spins 0,1 with
    gamma5 = +1; h = 1: spins 2,3), all colours, then orthonormalised.
    """
    nv = test_vectors.shape[0]
    n = 2 * nv
    Vf = volume(fine_dims)
    agg = aggregate_of(fine_dims)
    Vc = Vf // 16
    tv = test_vectors.reshape(nv, Vf, 4, 3)
    rows, cols, vals = [], [], []
    for a in range(Vc):
        sites = np.nonzero(agg == a)[0]
        for h in range(2):
            spins = (0, 1) if h == 0 else (2, 3)
            fine_idx = np.array([12 * x + 3 * s + c for x in sites for s in spins for c in range(3)])
            T = np.array([[tv[k, x, s, c] for k in range(nv)] for x in sites for s in spins for c in range(3)])
            Q = mgs_orthonormalise(T)
            for k in range(nv):
                rows.append(fine_idx)
                cols.append(np.full(fine_idx.shape, a * n + h * nv + k))
                vals.append(Q[:, k])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(12 * Vf, n * Vc)).tocsr()


def galerkin_blocks(U: np.ndarray, fine_dims, P: sp.spmatrix, m0: float, csw: float, nv: int):
    """Self and hop blocks of D_c = P^H D P.

    D is split into its site-diagonal part and its eight hop parts.  The
    product P^H D_d P of the hop part d has nonzero blocks only at (a, a)
    (links inside an aggregate, which belong to the self block) and at
    (a, a +- mu_d) (links crossing the aggregate face, the hop block d).
    Keeping the eight directions apart keeps the forward and backward
    couplings separate even when a coarse extent is 2.
    """
    cd = coarse_dims(fine_dims)
    Vc = volume(cd)
    n = 2 * nv
    nbc = neighbours(cd)
    PH = P.conj().T.tocsr()
    self_b = np.zeros((Vc, n, n), dtype=complex)
    hop_b = np.zeros((Vc, 8, n, n), dtype=complex)
    Dc0 = (PH @ fine.diagonal_part(U, fine_dims, m0, csw) @ P).tocsr()
    for a in range(Vc):
        self_b[a] += Dc0[a * n:(a + 1) * n, a * n:(a + 1) * n].toarray()
    for d in range(8):
        Dd = (PH @ fine.hop_part(U, fine_dims, d) @ P).tocsr()
        for a in range(Vc):
            rs = slice(a * n, (a + 1) * n)
            self_b[a] += Dd[rs, a * n:(a + 1) * n].toarray()
            b = nbc[a, d]
            hop_b[a, d] = Dd[rs, b * n:(b + 1) * n].toarray()
    return self_b, hop_b


def build(U: np.ndarray, fine_dims, nv: int, m0: float, csw: float, starts: np.ndarray, iters: int = 20):
    """Whole setup: returns (D sparse, P sparse, self blocks, hop blocks, test vectors)."""
    D = fine.wilson_clover(U, fine_dims, m0, csw)
    tv = np.array([refine_test_vector(D, s.reshape(-1), iters) for s in starts])
    P = prolongator(tv, fine_dims)
    self_b, hop_b = galerkin_blocks(U, fine_dims, P, m0, csw, nv)
    return D, P, self_b, hop_b, tv
