"""Adjoint solve and block gradients of L = Re<c, D_c^{-1} b> (oracle; test infrastructure only).

Follows the plain definitions:
    x      = D_c^{-1} b
    lambda = D_c^{-H} c                (solved directly with D_c^H, not through sigma3,
                                        so that the sigma3 identity of Sec. 4.2 is tested)
    dL/db  = lambda
    G_self[x]   = -lambda_x x_x^H
    G_hop[x, d] = -lambda_x x_{x +- mu_d}^H
with the real-gradient convention dL = Re sum conj(G) * dD (the convention of
PyTorch's complex autograd).  Finite differences use central differences on the
real and imaginary part of a single block entry.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import coarse
from .lattice import neighbours


def solve(self_b, hop_b, dims, rhs, mu=0.0):
    return spla.spsolve(coarse.assemble(self_b, hop_b, dims, mu).tocsc(), rhs)


def adjoint_solve(self_b, hop_b, dims, c, mu=0.0):
    Dh = coarse.assemble(self_b, hop_b, dims, mu).conj().T.tocsc()
    return spla.spsolve(Dh, c)


def loss(self_b, hop_b, dims, b, c, mu=0.0) -> float:
    x = solve(self_b, hop_b, dims, b, mu)
    return float(np.real(np.vdot(c, x)))


def block_gradient(lam, x, dims, n):
    V = lam.size // n
    nb = neighbours(dims)
    L = lam.reshape(V, n)
    X = x.reshape(V, n)
    g_self = -np.einsum("xi,xj->xij", L, X.conj())
    g_hop = -np.einsum("xi,xdj->xdij", L, X[nb].conj())
    return g_self, g_hop


def finite_difference(self_b, hop_b, dims, b, c, entry, h=1e-6, mu=0.0) -> complex:
    """dL/dRe + i dL/dIm of one block entry (site, block, row, col); block 0 = self, 1..8 = hop d."""
    site, blk, i, j = (int(v) for v in entry)

    def perturbed(delta):
        s, hp = self_b.copy(), hop_b.copy()
        if blk == 0:
            s[site, i, j] += delta
        else:
            hp[site, blk - 1, i, j] += delta
        return loss(s, hp, dims, b, c, mu)

    dre = (perturbed(h) - perturbed(-h)) / (2 * h)
    dim = (perturbed(1j * h) - perturbed(-1j * h)) / (2 * h)
    return dre + 1j * dim
