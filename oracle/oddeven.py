"""Odd-even reduced coarsest system with block-Jacobi left preconditioning (oracle).

Test infrastructure only: imported by the tests, ``__graft_entry__.smoke`` and the
benchmark's CPU baseline; the product path never calls it.

Sec. 2: with the sites split by parity (x0 + x1 + x2 + x3 even or odd; every hop
then joins opposite parities, which needs even extents), the coarse operator is
    D = [[D_oo, D_oe], [D_eo, D_ee]]
with D_oo, D_ee block diagonal (the self blocks, plus i mu sigma3 for twisted mass)
and D_oe, D_eo the nearest-neighbour hops.  The reduced system is
    (D_ee - D_eo D_oo^{-1} D_oe) psi_e = eta_e - D_eo D_oo^{-1} eta_o,
    psi_o = D_oo^{-1} (eta_o - D_oe psi_e),
and the reduced matrix is applied in this factored form, never assembled.
Sec. 3.2: left block-Jacobi preconditioning with B = the block diagonal of D_ee,
B^{-1} applied as explicit per-site inverses; the polynomial preconditioner is then
built for B^{-1} D_c (Eq. of the system with both preconditioners).  So the operator
the Krylov solver sees is
    S v = D_ee^{-1} (D_ee - D_eo D_oo^{-1} D_oe) v = v - D_ee^{-1} D_eo D_oo^{-1} D_oe v
with right-hand side D_ee^{-1} (eta_e - D_eo D_oo^{-1} eta_o).

Vectors on one parity are compressed: entry k belongs to the k-th site of that parity
in increasing site order.
"""
from __future__ import annotations

import numpy as np

from .coarse import sigma3
from .lattice import coordinates, neighbours


def parity(dims) -> np.ndarray:
    """0 for even sites (x0 + x1 + x2 + x3 even), 1 for odd.  Every extent must be even:
    with an odd periodic extent a hop across the boundary joins two sites of one parity."""
    if any(int(L) % 2 for L in dims):
        raise ValueError(f"odd-even splitting needs even extents, got {tuple(dims)}")
    return coordinates(dims).sum(axis=1) % 2


def sites(dims, p: int) -> np.ndarray:
    """Site indices of parity p in increasing order (the compressed order)."""
    return np.flatnonzero(parity(dims) == p)


def diag_blocks(self_b: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """Per-site diagonal blocks of D: A_x + i mu sigma3."""
    n = self_b.shape[1]
    return self_b + 1j * mu * np.diag(sigma3(n // 2))[None]


def inverses(self_b: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """Explicit per-site inverses of the diagonal blocks (Sec. 3.2)."""
    return np.linalg.inv(diag_blocks(self_b, mu))


def hop(hop_b: np.ndarray, dims, v_src: np.ndarray, dst: int) -> np.ndarray:
    """D_{dst,src} v: for every site x of parity dst, sum over the 8 directions d of
    hop[x, d] v[x +- mu_d]; v_src is compressed on the other parity."""
    V, _, n, _ = hop_b.shape
    par = parity(dims)
    nb = neighbours(dims)
    src_sites = np.flatnonzero(par != dst)
    full = np.zeros((V, n), dtype=np.complex128)
    full[src_sites] = v_src.reshape(-1, n)
    xs = np.flatnonzero(par == dst)
    y = np.zeros((xs.size, n), dtype=np.complex128)
    for d in range(8):
        y += np.einsum("xij,xj->xi", hop_b[xs, d], full[nb[xs, d]])
    return y.reshape(-1)


def block_diag_apply(blocks: np.ndarray, dims, v: np.ndarray, p: int) -> np.ndarray:
    """Per-site blocks of the parity-p sites times a compressed parity-p vector."""
    xs = sites(dims, p)
    n = blocks.shape[1]
    return np.einsum("xij,xj->xi", blocks[xs], v.reshape(-1, n)).reshape(-1)


def schur_apply(self_b, hop_b, dims, v_e: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """S v = v - D_ee^{-1} D_eo D_oo^{-1} D_oe v on a compressed even vector."""
    inv = inverses(self_b, mu)
    t_o = block_diag_apply(inv, dims, hop(hop_b, dims, v_e, 1), 1)
    return v_e - block_diag_apply(inv, dims, hop(hop_b, dims, t_o, 0), 0)


def reduced_rhs(self_b, hop_b, dims, b: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """D_ee^{-1} (b_e - D_eo D_oo^{-1} b_o) from a full right-hand side b."""
    n = self_b.shape[1]
    bb = b.reshape(-1, n)
    b_e, b_o = bb[sites(dims, 0)].reshape(-1), bb[sites(dims, 1)].reshape(-1)
    inv = inverses(self_b, mu)
    w = b_e - hop(hop_b, dims, block_diag_apply(inv, dims, b_o, 1), 0)
    return block_diag_apply(inv, dims, w, 0)


def retrieve(self_b, hop_b, dims, x_e: np.ndarray, b: np.ndarray, mu: float = 0.0) -> np.ndarray:
    """Full solution from the even part: x_o = D_oo^{-1} (b_o - D_oe x_e)."""
    n = self_b.shape[1]
    V = self_b.shape[0]
    bb = b.reshape(-1, n)
    ev, od = sites(dims, 0), sites(dims, 1)
    x_o = block_diag_apply(inverses(self_b, mu), dims, bb[od].reshape(-1) - hop(hop_b, dims, x_e, 1), 1)
    x = np.zeros((V, n), dtype=np.complex128)
    x[ev] = x_e.reshape(-1, n)
    x[od] = x_o.reshape(-1, n)
    return x.reshape(-1)


def schur_at(blocks_of, dims, v_e: np.ndarray, sites_e, mu: float = 0.0, inv_of=None) -> np.ndarray:
    """(S v)_x at the listed even sites only, S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe, from the
    same definition as ``schur_apply``: for each odd neighbour o of x,
    t_o = (A_o + i mu sigma3)^{-1} sum_d hop[o, d] v_{o +- mu_d}, then
    (S v)_x = v_x - (A_x + i mu sigma3)^{-1} sum_d hop[x, d] t_{x +- mu_d}.
    blocks_of(x) returns (A_x, hop[x]) as in coarse.apply_at; v_e is the whole compressed even
    vector.  inv_of(x), if given, supplies the diagonal-block inverse of site x (for instance a
    rounded copy) instead of inverting A_x + i mu sigma3.  Returns [len(sites_e), n]."""
    par = parity(dims)
    nb = neighbours(dims)
    half = np.zeros(par.size, dtype=np.int64)
    for p in (0, 1):
        xs = np.flatnonzero(par == p)
        half[xs] = np.arange(xs.size)
    ve = v_e.reshape(-1, blocks_of(int(sites(dims, 0)[0]))[0].shape[0])
    n = ve.shape[1]

    def diag_inv(x):
        if inv_of is not None:
            return inv_of(x)
        return np.linalg.inv(diag_blocks(blocks_of(x)[0][None], mu)[0])

    out = np.zeros((len(sites_e), n), dtype=np.complex128)
    for i, x in enumerate(sites_e):
        x = int(x)
        if par[x] != 0:
            raise ValueError(f"site {x} is not even")
        hop_x = blocks_of(x)[1]
        acc = np.zeros(n, dtype=np.complex128)
        for d in range(8):
            o = int(nb[x, d])
            hop_o = blocks_of(o)[1]
            w = sum(hop_o[dd] @ ve[half[nb[o, dd]]] for dd in range(8))
            acc = acc + hop_x[d] @ (diag_inv(o) @ w)
        out[i] = ve[half[x]] - diag_inv(x) @ acc
    return out
