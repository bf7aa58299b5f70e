"""Synthetic SU(3) gauge configurations.

``U = exp(i * eps * H)`` with ``H`` traceless Hermitian built from Gaussian
matrices, ``eps = 0.3`` by default.  These fields stand in for the thermalised
CLS and ETMC ensembles of the paper's Section 4, which are not available
here; they are not QCD configurations, only links with the right group
structure and a tunable roughness.
"""
from __future__ import annotations

import numpy as np
import torch

from . import draws


def lattice_volume(dims) -> int:
    return int(np.prod(dims))


def su3_links(key, dims, eps: float = 0.3, device="cpu") -> torch.Tensor:
    """Links ``U[mu, x]`` as a complex128 tensor of shape (4, V, 3, 3) on ``device``.

    Site index ``x = x0 + L0*(x1 + L1*(x2 + L2*x3))``.
    """
    V = lattice_volume(dims)
    a = torch.from_numpy(draws.gauge_algebra(key, V))  # (V, 4, 3, 3), host
    out = torch.empty((4, V, 3, 3), dtype=torch.complex128)
    # built on the host in chunks (the same arithmetic whatever the target device), then moved
    chunk = 1 << 16
    eye = torch.eye(3, dtype=torch.complex128)
    for s in range(0, V, chunk):
        h = 0.5 * (a[s:s + chunk] + a[s:s + chunk].conj().transpose(-1, -2))
        tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1) / 3.0
        h = h - tr[..., None, None] * eye
        lam, vec = torch.linalg.eigh(h)
        ph = torch.exp(1j * eps * lam.to(torch.complex128))
        u = (vec * ph[..., None, :]) @ vec.conj().transpose(-1, -2)
        out[:, s:s + chunk] = u.permute(1, 0, 2, 3)
    return out.to(device)
