"""Fast (vectorised PyTorch, any device) builder of synthetic coarse operators.

This is the workload generator: it turns the seeded draws of ``draws`` into
the Galerkin blocks that the library ingests.  It follows the same recipe as
the oracle's multigrid setup (fine Wilson-clover operator of Section 2.1,
test vectors, aggregation prolongator and ``D_c = P^H D P`` of Section 2.2),
written independently and vectorised so that a 32^4 fine lattice builds in
seconds on a GPU.  The tests pin it to the oracle's setup block by block.

Output layout (the library's canonical input layout):
    self_blocks  [Vc, n, n]     complex128, row-major, n = 2*nv
    hop_blocks   [Vc, 8, n, n]  hop[x, d] = D_c[x, x + mu_d] for d < 4,
                                 D_c[x, x - mu_{d-4}] for d >= 4
Within a site the nv chirality-+ dofs come first.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import draws
from .gauge import lattice_volume, su3_links


def gamma_chiral(device="cpu") -> torch.Tensor:
    """Euclidean Hermitian gamma_0..gamma_3 in a chiral basis, gamma_5 = diag(1,1,-1,-1)."""
    s = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]
    z = np.zeros((2, 2), complex)
    i2 = np.eye(2, dtype=complex)
    g = [np.block([[z, -1j * s[k]], [1j * s[k], z]]) for k in range(3)]
    g.append(np.block([[z, i2], [i2, z]]))
    return torch.tensor(np.stack(g), dtype=torch.complex128, device=device)


def neighbour_table(dims, device="cpu") -> torch.Tensor:
    """``nb[x, d]``: site x + mu_d (d < 4) or x - mu_{d-4} (d >= 4), periodic."""
    L = list(dims)
    V = lattice_volume(L)
    idx = torch.arange(V, device=device)
    coords = []
    rem = idx.clone()
    for mu in range(4):
        coords.append(rem % L[mu])
        rem = rem // L[mu]
    strides = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]

    def site(c):
        return c[0] + strides[1] * c[1] + strides[2] * c[2] + strides[3] * c[3]

    nb = torch.empty((V, 8), dtype=torch.long, device=device)
    for d in range(8):
        mu, sgn = d % 4, (1 if d < 4 else -1)
        c = list(coords)
        c[mu] = (coords[mu] + sgn) % L[mu]
        nb[:, d] = site(c)
    return nb, coords


@dataclass
class FineOperator:
    dims: tuple
    U: torch.Tensor        # (4, V, 3, 3)
    clover: torch.Tensor   # (V, 12, 12) including (m0 + 4)
    nb: torch.Tensor       # (V, 8)
    coords: list
    gamma: torch.Tensor    # (4, 4, 4)

    def hop(self, d: int, psi: torch.Tensor) -> torch.Tensor:
        """Term of D for hop direction d applied to psi (..., V, 4, 3)."""
        mu = d % 4
        V = psi.shape[-3]
        lead = psi.shape[:-3]
        eye = torch.eye(4, dtype=psi.dtype, device=psi.device)
        if d < 4:
            proj = -0.5 * (eye - self.gamma[mu])
            link = self.U[mu]
        else:
            proj = -0.5 * (eye + self.gamma[mu])
            link = self.U[mu][self.nb[:, d]].conj().transpose(-1, -2)
        src = psi.index_select(-3, self.nb[:, d]).reshape(-1, V, 4, 3)   # (C, V, 4, 3)
        C = src.shape[0]
        x = src.permute(1, 3, 0, 2).reshape(V, 3, C * 4)                # colour-major per site
        t = torch.bmm(link, x).reshape(V, 3, C, 4).permute(2, 0, 3, 1)   # (C, V, 4, 3)
        return torch.matmul(proj, t).reshape(*lead, V, 4, 3)

    def diag(self, psi: torch.Tensor) -> torch.Tensor:
        shp = psi.shape
        out = torch.matmul(self.clover, psi.reshape(-1, shp[-3], 12, 1))
        return out.reshape(shp)

    def apply(self, psi: torch.Tensor) -> torch.Tensor:
        out = self.diag(psi)
        for d in range(8):
            out = out + self.hop(d, psi)
        return out


def _leaf(U, nb, a: int, b: int, x_idx=None):
    """Plaquette leaf Q^{alpha,beta}_x = U_beta(x) U_alpha(x+beta) U_beta(x+alpha)^H U_alpha(x)^H
    for signed directions a, b encoded as 0..3 (+mu) and 4..7 (-mu)."""
    V = U.shape[1]
    x = torch.arange(V, device=U.device)

    def link(d, y):
        mu = d % 4
        if d < 4:
            return U[mu][y]
        return U[mu][nb[y, d]].conj().transpose(-1, -2)

    xb = nb[x, b]
    xa = nb[x, a]
    return link(b, x) @ link(a, xb) @ link(b, xa).conj().transpose(-1, -2) @ link(a, x).conj().transpose(-1, -2)


def clover_blocks(U, nb, gamma, m0: float, csw: float) -> torch.Tensor:
    """Site-diagonal 12x12 blocks (m0 + 4) I - csw/32 sum_{mu,nu} gamma_mu gamma_nu (x) (Q_munu - Q_numu)."""
    V = U.shape[1]
    dev = U.device
    out = torch.zeros((V, 12, 12), dtype=torch.complex128, device=dev)
    out += (m0 + 4.0) * torch.eye(12, dtype=torch.complex128, device=dev)
    if csw == 0.0:
        return out
    Q = {}
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            # four leaves around x, all with the orientation of the (mu, nu) leaf
            Q[(mu, nu)] = (_leaf(U, nb, mu, nu) + _leaf(U, nb, nu + 4, mu)
                           + _leaf(U, nb, nu, mu + 4) + _leaf(U, nb, mu + 4, nu + 4))
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            gg = gamma[mu] @ gamma[nu]
            F = Q[(mu, nu)] - Q[(nu, mu)]
            out -= (csw / 32.0) * torch.einsum("st,vab->vsatb", gg, F).reshape(V, 12, 12)
    return out


def fine_operator(key, dims, m0: float, csw: float, eps: float = 0.3, device="cpu", U=None) -> FineOperator:
    if U is None:
        U = su3_links(key, dims, eps, device)
    nb, coords = neighbour_table(dims, device)
    g = gamma_chiral(device)
    cl = clover_blocks(U, nb, g, m0, csw)
    return FineOperator(tuple(dims), U, cl, nb, coords, g)


def _chunk(count: int, per_item_bytes: int, device) -> int:
    """Items processed together: batched on a GPU (within a memory budget), one at a time on the host."""
    if not str(device).startswith("cuda"):
        return 1
    return max(1, min(count, (24 << 30) // max(per_item_bytes, 1)))


def refine_test_vectors(D: FineOperator, starts: torch.Tensor, iters: int) -> torch.Tensor:
    """Each start x0 -> argmin ||D x|| over x0 + K_iters(D, D x0) (one unrestarted GMRES cycle on D x = 0).

    The starts are processed together in chunks (modified Gram-Schmidt per vector, batched)."""
    nv = starts.shape[0]
    V = starts.shape[1]
    dev = starts.device
    per = (iters + 4) * V * 12 * 16
    ch = _chunk(nv, per, dev)
    out = []
    red = tuple(range(1, starts.dim()))
    for c0 in range(0, nv, ch):
        X0 = starts[c0:c0 + ch]
        nb_ = X0.shape[0]
        r0 = -D.apply(X0)
        beta = torch.linalg.vector_norm(r0, dim=red)
        shape1 = (nb_,) + (1,) * (X0.dim() - 1)
        basis = [r0 / beta.reshape(shape1)]
        H = torch.zeros((nb_, iters + 1, iters), dtype=torch.complex128, device=dev)
        for j in range(iters):
            w = D.apply(basis[j])
            for i in range(j + 1):
                h = (basis[i].conj() * w).sum(dim=red)
                H[:, i, j] = h
                w = w - h.reshape(shape1) * basis[i]
            hn = torch.linalg.vector_norm(w, dim=red)
            H[:, j + 1, j] = hn
            basis.append(w / hn.reshape(shape1))
        rhs = torch.zeros((nb_, iters + 1, 1), dtype=torch.complex128)
        rhs[:, 0, 0] = beta.cpu()
        # small least-squares problems on the host (any device gives the same arithmetic)
        z = torch.linalg.lstsq(H.cpu(), rhs).solution[:, :, 0].to(dev)
        x = X0.clone()
        for i in range(iters):
            x = x + z[:, i].reshape(shape1) * basis[i]
        out.append(x)
        del basis
    return torch.cat(out)


def prolongator(tv: torch.Tensor, dims) -> torch.Tensor:
    """Aggregation prolongator as Pf[x, s, c, k] (fine site, spin, colour, test vector index).

    On each 2^4 aggregate and each chirality half (spins {0,1} and {2,3}) the
    restricted test vectors are orthonormalised in generation order
    (Gram-Schmidt convention: R has a positive real diagonal).
    """
    nv = tv.shape[0]
    L0, L1, L2, L3 = dims
    # tv: (nv, V, 4, 3) -> (L3/2, 2, L2/2, 2, L1/2, 2, L0/2, 2, 2 chir, 2 spin, 3 col, nv)
    t = tv.permute(1, 2, 3, 0).reshape(L3 // 2, 2, L2 // 2, 2, L1 // 2, 2, L0 // 2, 2, 2, 2, 3, nv)
    t = t.permute(0, 2, 4, 6, 8, 1, 3, 5, 7, 9, 10, 11)  # agg(4), chir, local(4), spin, col, nv
    Vc = (L0 // 2) * (L1 // 2) * (L2 // 2) * (L3 // 2)
    shp = t.shape
    dev = t.device
    t = t.reshape(Vc * 2, 96, nv).cpu()   # batched QR on the host
    q, r = torch.linalg.qr(t)
    ph = torch.diagonal(r, dim1=-2, dim2=-1)
    ph = ph / ph.abs()
    q = q * ph[:, None, :]
    q = q.reshape(shp)
    q = q.permute(0, 5, 1, 6, 2, 7, 3, 8, 4, 9, 10, 11)  # back to (L3/2,2,L2/2,2,L1/2,2,L0/2,2,chir,spin,col,nv)
    return q.reshape(L0 * L1 * L2 * L3, 4, 3, nv).to(dev)


def _restrict(Pf: torch.Tensor, w: torch.Tensor, dims) -> torch.Tensor:
    """(P^H w)[a, h*nv + i] for a fine vector w (V, 4, 3)."""
    nv = Pf.shape[-1]
    L0, L1, L2, L3 = dims
    t = torch.einsum("vsck,vsc->vsk", Pf.conj(), w)          # (V, 4, nv)
    t = t.reshape(-1, 2, 2, nv).sum(2)                        # (V, chir, nv)
    t = t.reshape(L3 // 2, 2, L2 // 2, 2, L1 // 2, 2, L0 // 2, 2, 2 * nv).sum((1, 3, 5, 7))
    return t.reshape(-1, 2 * nv)


def galerkin(D: FineOperator, Pf: torch.Tensor):
    """Blocks of D_c = P^H D P, separated into the self block and the 8 hop directions.

    The columns (h, k) of P are pushed through the operator together in chunks."""
    dims = D.dims
    nv = Pf.shape[-1]
    n = 2 * nv
    V = lattice_volume(dims)
    Vc = V // 16
    dev = Pf.device
    self_b = torch.zeros((Vc, n, n), dtype=torch.complex128, device=dev)
    hop_b = torch.zeros((Vc, 8, n, n), dtype=torch.complex128, device=dev)
    chir_of_spin = torch.tensor([0, 0, 1, 1], device=dev)
    ch = _chunk(nv, 8 * V * 12 * 16, dev)
    inside = []
    for d in range(8):
        par = D.coords[d % 4] % 2
        m = (par == 0) if d < 4 else (par == 1)     # x +- mu stays in the aggregate
        inside.append(m.to(torch.complex128)[:, None, None])
    for h in range(2):
        smask = (chir_of_spin == h).to(torch.complex128)[None, None, :, None]
        for k0 in range(0, nv, ch):
            ks = slice(k0, min(nv, k0 + ch))
            phi = Pf[..., ks].permute(3, 0, 1, 2) * smask       # columns (h, k) on every aggregate
            cols = slice(h * nv + k0, h * nv + ks.stop)
            self_b[:, :, cols] += _restrict_many(Pf, D.diag(phi), dims)
            for d in range(8):
                hp = D.hop(d, phi)
                self_b[:, :, cols] += _restrict_many(Pf, hp * inside[d], dims)
                hop_b[:, d, :, cols] += _restrict_many(Pf, hp * (1 - inside[d]), dims)
    return self_b, hop_b


def _restrict_many(Pf: torch.Tensor, w: torch.Tensor, dims) -> torch.Tensor:
    """(P^H w_c) for a stack of fine vectors w (C, V, 4, 3); returns (Vc, n, C)."""
    nv = Pf.shape[-1]
    C = w.shape[0]
    L0, L1, L2, L3 = dims
    # (V, 4, 3*nv)^H-contraction per site, batched over the C vectors
    t = torch.bmm(w.reshape(C, -1, 4, 3).permute(1, 2, 0, 3).reshape(-1, C, 3),
                  Pf.conj().reshape(-1, 3, nv))                    # (V*4, C, nv)
    t = t.reshape(-1, 2, 2, C, nv).sum(2)                          # (V, chir, C, nv)
    t = t.permute(2, 0, 1, 3).reshape(C, L3 // 2, 2, L2 // 2, 2, L1 // 2, 2, L0 // 2, 2, 2 * nv)
    t = t.sum((2, 4, 6, 8)).reshape(C, -1, 2 * nv)                 # (C, Vc, n)
    return t.permute(1, 2, 0)


@dataclass
class CoarseOperator:
    dims: tuple           # coarse lattice
    nv: int
    self_blocks: torch.Tensor
    hop_blocks: torch.Tensor
    mu: float = 0.0       # twisted mass, added on the coarse level as i*mu*sigma3 by the consumer

    @property
    def n(self):
        return 2 * self.nv

    @property
    def volume(self):
        return self.self_blocks.shape[0]


def build_coarse_operator(key, fine_dims, nv: int, m0: float, csw: float = 1.0, eps: float = 0.3,
                          tv_iters: int = 20, device="cpu", mu: float = 0.0) -> CoarseOperator:
    """Whole recipe: SU(3) field -> fine Wilson-clover D -> test vectors -> P -> D_c blocks.

    The twisted mass ``mu`` is not folded into the blocks; it is carried
    alongside (P^H (i mu Gamma5) P = i mu sigma3 exactly for this P).
    """
    fine_dims = tuple(int(v) for v in fine_dims)
    assert all(v % 2 == 0 for v in fine_dims)
    D = fine_operator(key, fine_dims, m0, csw, eps, device)
    V = lattice_volume(fine_dims)
    starts = torch.from_numpy(draws.test_vector_starts(key, V, nv)).to(device)
    tv = refine_test_vectors(D, starts, tv_iters)
    del starts
    Pf = prolongator(tv, fine_dims)
    del tv
    self_b, hop_b = galerkin(D, Pf)
    cdims = tuple(v // 2 for v in fine_dims)
    return CoarseOperator(cdims, nv, self_b, hop_b, mu)
