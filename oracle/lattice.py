"""Lattice geometry and Dirac gamma matrices (oracle; test infrastructure only).

Sec. 2.1: the gamma_mu are unitary Hermitian generators of the Euclidean
Clifford algebra, gamma_mu gamma_nu + gamma_nu gamma_mu = 2 delta_munu I.
We use a chiral basis with gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 =
diag(1, 1, -1, -1) (the paper's "i gamma_1 gamma_2 gamma_3 gamma_4" carries a
Minkowski-convention factor; its sign only flips the sign of mu in the
twisted-mass term).
"""
from __future__ import annotations

import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
)


def gammas() -> np.ndarray:
    """gamma_0..gamma_3, shape (4, 4, 4)."""
    Z = np.zeros((2, 2), dtype=complex)
    I2 = np.eye(2, dtype=complex)
    out = []
    for k in range(3):
        out.append(np.block([[Z, -1j * SIGMA[k]], [1j * SIGMA[k], Z]]))
    out.append(np.block([[Z, I2], [I2, Z]]))
    return np.array(out)


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def volume(dims) -> int:
    return int(np.prod(dims))


def site_index(c, dims) -> int:
    """x0 + L0*(x1 + L1*(x2 + L2*x3))."""
    return int(c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3])))


def coordinates(dims) -> np.ndarray:
    """Coordinates of every site, shape (V, 4)."""
    V = volume(dims)
    x = np.arange(V)
    out = np.empty((V, 4), dtype=np.int64)
    for mu in range(4):
        out[:, mu] = x % dims[mu]
        x = x // dims[mu]
    return out


def neighbours(dims) -> np.ndarray:
    """nb[x, d] = x + mu_d (d < 4) or x - mu_{d-4} (d >= 4), periodic boundaries."""
    c = coordinates(dims)
    V = c.shape[0]
    nb = np.empty((V, 8), dtype=np.int64)
    for d in range(8):
        mu = d % 4
        step = 1 if d < 4 else -1
        cc = c.copy()
        cc[:, mu] = (cc[:, mu] + step) % dims[mu]
        nb[:, d] = cc[:, 0] + dims[0] * (cc[:, 1] + dims[1] * (cc[:, 2] + dims[2] * cc[:, 3]))
    return nb
