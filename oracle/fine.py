"""Fine-level Wilson-clover and twisted-mass Dirac operators (oracle; test infrastructure only).

Sec. 2.1, lattice spacing a = 1, periodic boundaries:

    (D psi)(x) = (m0 + 4) psi(x)
                 - 1/2 sum_mu [(I - gamma_mu) (x) U_mu(x)] psi(x + mu)
                 - 1/2 sum_mu [(I + gamma_mu) (x) U_mu(x - mu)^H] psi(x - mu)

clover improvement (replaces the mass term):

    (m0 + 4) I_12 - c_sw/32 sum_{mu,nu} (gamma_mu gamma_nu) (x) (Q_munu(x) - Q_numu(x))

with Q_munu the sum of the four plaquette leaves Q^{+-mu,+-nu}_x,
Q^{mu,nu}_x = U_nu(x) U_mu(x+nu) U_nu(x+mu)^H U_mu(x)^H and U_{-mu}(x) = U_mu(x-mu)^H;
and twisted mass D_TM = D + i mu Gamma5.

A fine spinor is indexed (site, spin, colour) -> 12*x + 3*s + c.  Operators
are returned as scipy.sparse CSR matrices built block by block.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .lattice import gamma5, gammas, neighbours, volume


def link(U: np.ndarray, nb: np.ndarray, d: int, y: np.ndarray) -> np.ndarray:
    """U_{+mu}(y) = U_mu(y) for d = mu < 4; U_{-mu}(y) = U_mu(y - mu)^H for d = mu + 4."""
    mu = d % 4
    if d < 4:
        return U[mu][y]
    return np.conj(np.swapaxes(U[mu][nb[y, d]], -1, -2))


def leaf(U: np.ndarray, nb: np.ndarray, a: int, b: int) -> np.ndarray:
    """Plaquette leaf Q^{a,b}_x for all x (signed directions: 0..3 = +mu, 4..7 = -mu)."""
    x = np.arange(U.shape[1])
    H = lambda m: np.conj(np.swapaxes(m, -1, -2))
    return link(U, nb, b, x) @ link(U, nb, a, nb[x, b]) @ H(link(U, nb, b, nb[x, a])) @ H(link(U, nb, a, x))


def clover_field(U: np.ndarray, nb: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_munu(x): the four plaquette leaves at x in the quadrants (+-mu, +-nu).

    Reading of Sec. 2.1: all four leaves are traversed with the orientation of
    Q^{mu,nu}_x (the clover of Sheikholeslami and Wohlert).  Substituting the
    signed directions literally into the leaf formula would reverse the two
    mixed-sign leaves and cancel the field strength of any abelian field.  A
    mixed-sign leaf is therefore the literal leaf with its two directions
    swapped (path -nu first, then mu becomes mu first, then -nu).
    """
    return (leaf(U, nb, mu, nu) + leaf(U, nb, nu + 4, mu)
            + leaf(U, nb, nu, mu + 4) + leaf(U, nb, mu + 4, nu + 4))


def clover_term(U: np.ndarray, dims, m0: float, csw: float) -> np.ndarray:
    """Site-diagonal 12x12 blocks of the clover-improved mass term, shape (V, 12, 12)."""
    V = volume(dims)
    nb = neighbours(dims)
    g = gammas()
    out = np.zeros((V, 12, 12), dtype=complex)
    out[:] = (m0 + 4.0) * np.eye(12)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = clover_field(U, nb, mu, nu) - clover_field(U, nb, nu, mu)
            gg = g[mu] @ g[nu]
            for x in range(V):
                out[x] -= (csw / 32.0) * np.kron(gg, F[x])
    return out


def wilson_clover(U: np.ndarray, dims, m0: float, csw: float, mu_tm: float = 0.0) -> sp.csr_matrix:
    """Sparse fine operator D (Wilson-clover, plus i*mu_tm*Gamma5 when mu_tm != 0)."""
    V = volume(dims)
    nb = neighbours(dims)
    g = gammas()
    I4 = np.eye(4)
    rows, cols, vals = [], [], []

    def add_block(x, y, blk):
        r = 12 * x + np.arange(12)
        c = 12 * y + np.arange(12)
        rows.append(np.repeat(r, 12))
        cols.append(np.tile(c, 12))
        vals.append(blk.reshape(-1))

    diag = clover_term(U, dims, m0, csw)
    if mu_tm != 0.0:
        diag = diag + 1j * mu_tm * np.kron(gamma5(), np.eye(3))[None]
    for x in range(V):
        add_block(x, x, diag[x])
        for m in range(4):
            add_block(x, nb[x, m], -0.5 * np.kron(I4 - g[m], U[m][x]))
            add_block(x, nb[x, m + 4], -0.5 * np.kron(I4 + g[m], U[m][nb[x, m + 4]].conj().T))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    # duplicates (lattice extent 2: x + mu == x - mu) are summed by the COO -> CSR conversion
    return sp.coo_matrix((v, (r, c)), shape=(12 * V, 12 * V)).tocsr()


def hop_part(U: np.ndarray, dims, d: int) -> sp.csr_matrix:
    """The hop term of D for one direction d alone (d < 4: +mu, d >= 4: -mu)."""
    V = volume(dims)
    nb = neighbours(dims)
    g = gammas()
    I4 = np.eye(4)
    m = d % 4
    rows, cols, vals = [], [], []
    for x in range(V):
        if d < 4:
            blk = -0.5 * np.kron(I4 - g[m], U[m][x])
        else:
            blk = -0.5 * np.kron(I4 + g[m], U[m][nb[x, d]].conj().T)
        rows.append(np.repeat(12 * x + np.arange(12), 12))
        cols.append(np.tile(12 * nb[x, d] + np.arange(12), 12))
        vals.append(blk.reshape(-1))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(12 * V, 12 * V)).tocsr()


def diagonal_part(U: np.ndarray, dims, m0: float, csw: float) -> sp.csr_matrix:
    """Site-diagonal part of D (clover-improved mass term)."""
    return sp.block_diag([sp.csr_matrix(b) for b in clover_term(U, dims, m0, csw)], format="csr")


def Gamma5(dims) -> sp.csr_matrix:
    """Gamma5 = I_V (x) gamma5 (x) I_3."""
    return sp.kron(sp.eye(volume(dims)), np.kron(gamma5(), np.eye(3)), format="csr")
