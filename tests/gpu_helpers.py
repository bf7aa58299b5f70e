"""Shared fixtures of the GPU parity tests: seeded synthetic operators, the oracle side, and the
entry-by-entry error bounds the parity checks use.

Entry-wise bounds.  An output entry y_i = sum_j a_ij x_j evaluated in floating point, with the
block entries rounded to the block precision (relative u_blk per entry, real and imaginary
parts separately) and x rounded to the vector precision (u_x), satisfies to first order
    |fl(y_i) - y_i| <= (u_blk + u_x + (K + 4) u) * sum_j |a_ij| |x_j|,
K the number of complex products summed and u the unit roundoff of the accumulation
(complex products add two roundings each, the +4 covers them and the final store).  The
oracle's own FP64 evaluation adds (K + 4) 2^-53 of the same sum.  The magnitude sums
(|D| |x|)_i come from the oracle applied to |blocks| and |x|.  A wrong term anywhere (one
missing hop, a sign, a transposed block) moves the entry by O(1/sqrt(K)) of that sum, far
above these bounds, even for BF16 blocks.
"""
import numpy as np
import torch

from synthetic import draws
from synthetic.coarse_op import build_coarse_operator

U64, U32, UBF16 = 2.0 ** -53, 2.0 ** -24, 2.0 ** -9
U_ACC = {0: U64, 1: U32, 2: U32}        # accumulation unit roundoff per coarse_precision
U_BLK = {0: 0.0, 1: U32, 2: UBF16}       # rounding of the stored block entries


def make_op(key, fine_dims, nv, m0=-0.4, csw=1.0, device="cpu"):
    return build_coarse_operator(key, fine_dims, nv, m0, csw, device=device)


def to_cuda(op, mu=0.0, precisions=(1, 2), max_nrhs=1):
    from paper_2205_09104_gb300 import CoarseOp
    s = op.self_blocks.to("cuda").contiguous()
    h = op.hop_blocks.to("cuda").contiguous()
    return CoarseOp(s, h, op.dims, op.nv, mu=mu, precisions=precisions, max_nrhs=max_nrhs)


def rhs(key, count, N, index0=0):
    return draws.rhs(key, count, N, index0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def stencil_factor(prec, n, x_prec=None, rounded_operands=False):
    """Entry-wise bound factor of one coarse stencil apply (K = 9n products + the mass term).
    x_prec: precision the kernel rounds x to (default: complex64 for FP32/BF16 applies).
    rounded_operands: the reference already uses the kernel's rounded blocks and vector, so
    only the accumulation differs (a bound tight enough to see a single wrong block entry
    of a BF16 kernel, which the block-rounding term would hide)."""
    ux = {None: 0.0 if prec == 0 else U32, "bf16": UBF16}[x_prec]
    ublk = U_BLK[prec]
    if rounded_operands:
        ux = ublk = 0.0
    K = 9 * n + 1
    return ublk + ux + (K + 4) * U_ACC[prec] + (K + 4) * U64


def bf16(a):
    """Entries rounded to BF16 (real and imaginary parts), returned as complex128."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return torch.complex(re, im).numpy()


def bf16_operator(s, h, dims):
    """The operator a BF16 kernel applies: self and forward hop blocks rounded to BF16, backward
    hops rebuilt from the rounded forward blocks as sigma3 F_{x-mu,mu}^H sigma3."""
    from oracle import coarse as ocoarse
    from oracle.lattice import neighbours
    s3 = ocoarse.sigma3(s.shape[1] // 2)
    nb = neighbours(dims)
    sr, hr = bf16(s), bf16(h)
    for mu in range(4):
        back = hr[nb[:, 4 + mu], mu]
        hr[:, 4 + mu] = s3[None, :, None] * np.conj(np.transpose(back, (0, 2, 1))) * s3[None, None, :]
    return sr, hr


def schur_factor(prec, n, rounded_operands=False):
    """Entry-wise bound factor of S = 1 - B_e^{-1} D_eo B_o^{-1} D_oe: two hop sums of 8n products
    and two inverse-block products of n, each with its block rounding (hops and inverses are
    stored in the block precision).  rounded_operands: the reference uses the kernel's rounded
    hops, inverse blocks and vector, so only the accumulation differs."""
    K = 2 * (8 * n + n) + 8
    ux = 0.0 if prec == 0 else U32
    ublk = U_BLK[prec]
    if rounded_operands:
        ux = ublk = 0.0
    return 4 * ublk + ux + (K + 4) * U_ACC[prec] + (K + 4) * U64


def bf16_schur(s, h, dims, x, mu=0.0):
    """S x as a BF16 kernel computes it, in FP64: BF16-rounded hops (backward hops rebuilt from
    the rounded forward blocks) and BF16-rounded FP64 inverses of the diagonal blocks.
    Returns (S x, the magnitude chain of those operands)."""
    from oracle import oddeven as ooe
    _, hr = bf16_operator(s, h, dims)
    ir = bf16(ooe.inverses(s, mu))
    t = ooe.block_diag_apply(ir, dims, ooe.hop(hr, dims, x, 1), 1)
    y = x - ooe.block_diag_apply(ir, dims, ooe.hop(hr, dims, t, 0), 0)
    ia, ha = np.abs(ir), np.abs(hr)
    ta = ooe.block_diag_apply(ia, dims, ooe.hop(ha, dims, np.abs(x), 1).real, 1).real
    mag = np.abs(x) + ooe.block_diag_apply(ia, dims, ooe.hop(ha, dims, ta, 0).real, 0).real
    return y, mag


def abs_apply(s, h, dims, x, mu=0.0, adjoint=False):
    """(|D_c| |x|)_i, or (|D_c^H| |x|)_i: the sums the stencil bounds scale with."""
    from oracle import coarse as ocoarse
    f = ocoarse.apply_adjoint if adjoint else ocoarse.apply
    return f(np.abs(s), np.abs(h), dims, np.abs(x), 0.0).real + abs(mu) * np.abs(x)


def abs_schur(s, h, dims, x, mu=0.0):
    """|x| + |B_e^{-1}| |D_eo| |B_o^{-1}| |D_oe| |x| on a compressed even vector."""
    from oracle import oddeven as ooe
    inv = np.abs(ooe.inverses(s, mu))
    ha = np.abs(h)
    t = ooe.block_diag_apply(inv, dims, ooe.hop(ha, dims, np.abs(x), 1).real, 1).real
    return np.abs(x) + ooe.block_diag_apply(inv, dims, ooe.hop(ha, dims, t, 0).real, 0).real


def assert_entrywise(y, ref, bound, what=""):
    """Every entry within its own bound; the message names the worst offenders."""
    y, ref, bound = (np.asarray(a).reshape(-1) for a in (y, ref, bound))
    err = np.abs(y - ref)
    bad = np.flatnonzero(err > bound)
    if bad.size:
        worst = bad[np.argsort(-(err[bad] / np.maximum(bound[bad], 1e-300)))][:5]
        detail = ", ".join(f"i={i} err={err[i]:.3e} bound={bound[i]:.3e}" for i in worst)
        raise AssertionError(f"{what}: {bad.size} of {err.size} entries over their bound ({detail})")


def abs_apply_at(blocks_of, dims, x, sites, mu=0.0):
    """(|D_c| |x|) at the listed sites (blocks_of as for oracle.coarse.apply_at)."""
    from oracle import coarse as ocoarse
    absb = lambda s: tuple(np.abs(b) for b in blocks_of(s))
    n = blocks_of(int(sites[0]))[0].shape[0]
    xa = np.abs(x)
    return (ocoarse.apply_at(absb, dims, xa, sites, 0.0).real
            + abs(mu) * xa.reshape(-1, n)[np.asarray(sites)])


def abs_schur_at(blocks_of, dims, v_e, sites_e, mu=0.0, inv_of=None):
    """|v_x| + |B_x^{-1}| sum_d |hop[x,d]| |B_o^{-1}| sum_d' |hop[o,d']| |v| at the listed even sites
    (inv_of as for oracle.oddeven.schur_at)."""
    from oracle import oddeven as ooe
    from oracle.lattice import neighbours
    par = ooe.parity(dims)
    nb = neighbours(dims)
    half = np.zeros(par.size, dtype=np.int64)
    for p in (0, 1):
        xs = np.flatnonzero(par == p)
        half[xs] = np.arange(xs.size)
    n = blocks_of(int(sites_e[0]))[0].shape[0]
    va = np.abs(v_e).reshape(-1, n)
    ainv = lambda s: np.abs(inv_of(s) if inv_of is not None
                            else np.linalg.inv(ooe.diag_blocks(blocks_of(s)[0][None], mu)[0]))
    out = np.zeros((len(sites_e), n))
    for i, x in enumerate(sites_e):
        x = int(x)
        hx = np.abs(blocks_of(x)[1])
        acc = np.zeros(n)
        for d in range(8):
            o = int(nb[x, d])
            ho = np.abs(blocks_of(o)[1])
            w = sum(ho[dd] @ va[half[nb[o, dd]]] for dd in range(8))
            acc += hx[d] @ (ainv(o) @ w)
        out[i] = va[half[x]] + ainv(x) @ acc
    return out


def site_blocks(op, sites):
    """blocks_of(x) over host copies of just the blocks of the listed sites and their neighbours
    (the full block arrays of a large lattice may stay on the device)."""
    from oracle.lattice import neighbours
    nb = neighbours(op.dims)
    need = np.unique(np.concatenate([np.asarray(sites), nb[np.asarray(sites)].reshape(-1)]))
    idx = torch.from_numpy(need).to(op.self_blocks.device)
    s = op.self_blocks[idx].cpu().numpy()
    h = op.hop_blocks[idx].cpu().numpy()
    row = {int(x): i for i, x in enumerate(need)}
    return lambda x: (s[row[x]], h[row[x]])


def bf16_blocks_of(blocks_of, dims):
    """blocks_of for the operator a BF16 kernel applies (as bf16_operator, site by site): the
    backward hop of x is rebuilt from the rounded forward block of its neighbour."""
    from oracle import coarse as ocoarse
    from oracle.lattice import neighbours
    nb = neighbours(dims)

    def f(x):
        A, hop = blocks_of(x)
        s3 = ocoarse.sigma3(A.shape[0] // 2)
        hr = bf16(hop)
        for mu in range(4):
            fwd = bf16(blocks_of(int(nb[x, 4 + mu]))[1][mu])
            hr[4 + mu] = s3[:, None] * np.conj(fwd.T) * s3[None, :]
        return bf16(A), hr
    return f


def check_schur_entrywise(y, x, s, h, dims, prec, mu=0.0, what="S"):
    """S x from a kernel of precision prec against the oracle, entry by entry: the worst-case
    bound around the exact S, and for BF16 also the accumulation-only bound around S on the
    kernel's rounded operands.  x is the complex64 (or complex128) input the kernel received."""
    from oracle import oddeven as ooe
    x = np.asarray(x).astype(np.complex128)
    ref = ooe.schur_apply(s, h, dims, x, mu)
    assert_entrywise(y, ref, schur_factor(prec, s.shape[1]) * abs_schur(s, h, dims, x, mu), f"{what} prec {prec}")
    if prec == 2:
        ref_r, mag_r = bf16_schur(s, h, dims, x, mu)
        assert_entrywise(y, ref_r, schur_factor(2, s.shape[1], rounded_operands=True) * mag_r,
                         f"{what} bf16 rounded operands")


def bf16_inv_of(blocks_of, mu=0.0):
    """The diagonal-block inverses a BF16 odd-even kernel uses: FP64 inverses rounded to BF16."""
    from oracle import oddeven as ooe
    return lambda x: bf16(np.linalg.inv(ooe.diag_blocks(blocks_of(x)[0][None], mu)[0]))


def sampled_apply_check(dev, op, mu, x, sites, precs=(0, 1, 2), what=""):
    """coarse_apply at the listed sites against the oracle's per-site stencil, entry by entry
    (BF16 also on its rounded operands).  op's blocks may stay on the device."""
    from oracle import coarse as ocoarse
    blocks_of = site_blocks(op, sites)
    ref = ocoarse.apply_at(blocks_of, op.dims, x, sites, mu)
    mag = abs_apply_at(blocks_of, op.dims, x, sites, mu)
    for prec in precs:
        dt = torch.complex128 if prec == 0 else torch.complex64
        xin = torch.from_numpy(x).to(dt)
        y = dev.apply(xin.to("cuda"), precision=prec).cpu().numpy().reshape(op.volume, op.n)[sites]
        assert_entrywise(y, ref, stencil_factor(prec, op.n) * mag, f"{what} sampled apply prec {prec}")
        if prec == 2:
            x32 = xin.numpy().astype(np.complex128)
            rb = bf16_blocks_of(blocks_of, op.dims)
            ref_r = ocoarse.apply_at(rb, op.dims, x32, sites, mu)
            mag_r = abs_apply_at(rb, op.dims, x32, sites, mu)
            assert_entrywise(y, ref_r, stencil_factor(2, op.n, rounded_operands=True) * mag_r,
                             f"{what} sampled apply, bf16 rounded operands")


def schur_site_blocks(op, sites_e):
    """blocks_of over the even sites listed, their odd neighbours and those neighbours' neighbours
    (what the per-site S needs)."""
    from oracle.lattice import neighbours
    nb = neighbours(op.dims)
    first = np.unique(np.concatenate([np.asarray(sites_e), nb[np.asarray(sites_e)].reshape(-1)]))
    return site_blocks(op, first)


def sampled_schur_check(dev, op, mu, v_e, sites_e, precs=(0, 1, 2), what=""):
    """coarse_schur_apply at the listed even sites against the oracle's per-site S, entry by entry
    (BF16 also on its rounded hops and inverse blocks)."""
    from oracle import oddeven as ooe
    blocks_of = schur_site_blocks(op, sites_e)
    ev = ooe.sites(op.dims, 0)
    pos = np.searchsorted(ev, np.asarray(sites_e))
    ref = ooe.schur_at(blocks_of, op.dims, v_e, sites_e, mu)
    mag = abs_schur_at(blocks_of, op.dims, v_e, sites_e, mu)
    for prec in precs:
        dt = torch.complex128 if prec == 0 else torch.complex64
        xin = torch.from_numpy(v_e).to(dt)
        y = dev.schur(xin.to("cuda"), precision=prec).cpu().numpy().reshape(-1, op.n)[pos]
        assert_entrywise(y, ref, schur_factor(prec, op.n) * mag, f"{what} sampled S prec {prec}")
        if prec == 2:
            x32 = xin.numpy().astype(np.complex128)
            rb = bf16_blocks_of(blocks_of, op.dims)
            ri = bf16_inv_of(blocks_of, mu)
            ref_r = ooe.schur_at(rb, op.dims, x32, sites_e, mu, inv_of=ri)
            mag_r = abs_schur_at(rb, op.dims, x32, sites_e, mu, inv_of=ri)
            assert_entrywise(y, ref_r, schur_factor(2, op.n, rounded_operands=True) * mag_r,
                             f"{what} sampled S, bf16 rounded operands")
