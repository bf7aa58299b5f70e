"""Coarse nearest-neighbour stencil D_c (oracle; test infrastructure only).

Sec. 2.2: on the coarse lattice D_c couples each site to itself (a dense
n x n self block, n = 2*n_tv) and to its 8 nearest neighbours:

    (D_c v)_x = A_x v_x + sum_{d=0..7} hop[x, d] v_{x +- mu_d}   (+ i mu sigma3 v_x)

where hop[x, d] = D_c[x, x + mu_d] for d < 4 and D_c[x, x - mu_{d-4}] for
d >= 4, and the optional twisted mass enters as i mu sigma3 (the coarse image
of i mu Gamma5, since P^H Gamma5 P = sigma3 for a spin-preserving P).
sigma3 = diag(+1 x n_tv, -1 x n_tv).

Gamma5-hermiticity (Sec. 4.2, Q = Gamma5 D Hermitian) carries over to the
coarse level as sigma3 D_c sigma3 = D_c^H, i.e. blockwise
hop[x, -mu] = sigma3 hop[x - mu, +mu]^H sigma3 and A_x = sigma3 A_x^H sigma3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .lattice import neighbours, volume


def sigma3(nv: int) -> np.ndarray:
    return np.concatenate([np.ones(nv), -np.ones(nv)])


def apply(self_b: np.ndarray, hop_b: np.ndarray, dims, v: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """y = D_c v for v of shape (V*n,) or (V, n)."""
    V, n, _ = self_b.shape
    nb = neighbours(dims)
    vv = v.reshape(V, n)
    y = np.einsum("xij,xj->xi", self_b, vv)
    for d in range(8):
        y += np.einsum("xij,xj->xi", hop_b[:, d], vv[nb[:, d]])
    if mu != 0.0:
        y += 1j * mu * sigma3(n // 2)[None, :] * vv
    return y.reshape(v.shape)


def apply_at(blocks_of, dims, v: np.ndarray, sites, mu: float = 0.0) -> np.ndarray:
    """(D_c v)_x at the listed sites only, by the definition above.

    blocks_of(x) returns (A_x, hop[x]): the n x n self block and the [8, n, n] hop blocks of
    site x, so a caller can hand over the blocks of just the sites asked for.  v is the
    whole vector (V*n,).  Returns [len(sites), n].
    """
    nb = neighbours(dims)
    V = volume(dims)
    vv = v.reshape(V, -1)
    n = vv.shape[1]
    out = np.zeros((len(sites), n), dtype=np.complex128)
    for i, x in enumerate(sites):
        A, hop = blocks_of(int(x))
        y = A @ vv[x]
        for d in range(8):
            y = y + hop[d] @ vv[nb[x, d]]
        if mu != 0.0:
            y = y + 1j * mu * sigma3(n // 2) * vv[x]
        out[i] = y
    return out


def apply_adjoint(self_b, hop_b, dims, v, mu: float = 0.0):
    """y = D_c^H v, from the definition (sum over the transposed couplings)."""
    V, n, _ = self_b.shape
    nb = neighbours(dims)
    vv = v.reshape(V, n)
    y = np.einsum("xji,xj->xi", self_b.conj(), vv)
    for d in range(8):
        # D_c[x, nb(x,d)] contributes conj-transposed to row nb(x,d), column x
        contrib = np.einsum("xji,xj->xi", hop_b[:, d].conj(), vv)
        np.add.at(y, nb[:, d], contrib)
    if mu != 0.0:
        y += -1j * mu * sigma3(n // 2)[None, :] * vv
    return y.reshape(v.shape)


def assemble(self_b: np.ndarray, hop_b: np.ndarray, dims, mu: float = 0.0) -> sp.csr_matrix:
    """Sparse matrix of D_c (duplicate couplings, for an extent of 2, are summed)."""
    V, n, _ = self_b.shape
    nb = neighbours(dims)
    rows, cols, vals = [], [], []
    r_in = np.repeat(np.arange(n), n)
    c_in = np.tile(np.arange(n), n)
    for x in range(V):
        blk = self_b[x].copy()
        if mu != 0.0:
            blk = blk + 1j * mu * np.diag(sigma3(n // 2))
        rows.append(x * n + r_in)
        cols.append(x * n + c_in)
        vals.append(blk.reshape(-1))
        for d in range(8):
            rows.append(x * n + r_in)
            cols.append(nb[x, d] * n + c_in)
            vals.append(hop_b[x, d].reshape(-1))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(V * n, V * n)).tocsr()


def gamma5_defect(self_b: np.ndarray, hop_b: np.ndarray, dims) -> float:
    """max over blocks of || hop[x,-mu] - sigma3 hop[x-mu,+mu]^H sigma3 || / max ||block||,
    including the self blocks (A_x vs sigma3 A_x^H sigma3)."""
    V, n, _ = self_b.shape
    nb = neighbours(dims)
    s = sigma3(n // 2)
    S = s[:, None] * s[None, :]
    scale = max(np.abs(self_b).max(), np.abs(hop_b).max())
    worst = np.abs(self_b - S * np.conj(np.swapaxes(self_b, -1, -2))).max()
    for mu in range(4):
        back = hop_b[:, mu + 4]
        fwd_of_prev = hop_b[nb[:, mu + 4], mu]
        worst = max(worst, np.abs(back - S * np.conj(np.swapaxes(fwd_of_prev, -1, -2))).max())
    return float(worst / scale)


def block_norms(self_b, hop_b):
    return np.sqrt(np.sum(np.abs(self_b) ** 2)), np.sqrt(np.sum(np.abs(hop_b) ** 2))
