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
    a = torch.from_numpy(draws.gauge_algebra(key, V)).to(device)  # (V, 4, 3, 3)
    h = 0.5 * (a + a.conj().transpose(-1, -2))
    tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1) / 3.0
    h = h - tr[..., None, None] * torch.eye(3, dtype=h.dtype, device=device)
    lam, vec = torch.linalg.eigh(h)
    ph = torch.exp(1j * eps * lam.to(torch.complex128))
    u = (vec * ph[..., None, :]) @ vec.conj().transpose(-1, -2)
    del a, h, vec
    return u.permute(1, 0, 2, 3).contiguous()
