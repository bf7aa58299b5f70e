"""The entry-wise bounds of the GPU parity tests (gpu_helpers) on the CPU: an emulation of each
kernel's rounding stays inside them, and planted mistakes in one site (one hop dropped, one hop
block transposed, one block entry of the wrong sign) leave them.  A single wrong block entry is
below the BF16 block-rounding bound, so BF16 kernels are also compared with the oracle applied
to their BF16-rounded operands, where only the FP32 accumulation differs; that bound sees it."""
import numpy as np
import pytest
import torch

from gpu_helpers import (abs_apply, abs_schur, assert_entrywise, bf16_operator, bf16_schur, schur_factor,
                         stencil_factor)
from oracle import coarse as ocoarse
from oracle import oddeven as ooe
from oracle.lattice import neighbours
from synthetic import draws


def _bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return torch.complex(re, im).numpy()


def _c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


@pytest.fixture(scope="module")
def op24():
    from synthetic.coarse_op import build_coarse_operator
    return build_coarse_operator((906, 0), (4, 6, 4, 4), 24, -0.4, 1.0)


def _planted(s, h, dims, x, site, kind):
    """The oracle's apply with one mistake at one site (planted on the CPU)."""
    y = ocoarse.apply(s, h, dims, x).reshape(s.shape[0], -1).copy()
    nb = neighbours(dims)
    xv = x.reshape(s.shape[0], -1)
    blk = h[site, 2]
    if kind == "drop":
        y[site] -= blk @ xv[nb[site, 2]]
    elif kind == "transpose":
        y[site] += (blk.T - blk) @ xv[nb[site, 2]]
    elif kind == "sign":
        i, j = 3, 5
        y[site, i] -= 2 * blk[i, j] * xv[nb[site, 2], j]
    return y.reshape(-1)


def test_rounding_emulations_inside_bounds(op24):
    s, h, dims = op24.self_blocks.numpy(), op24.hop_blocks.numpy(), op24.dims
    n = op24.n
    x = draws.rhs((906, 1), 1, s.shape[0] * n)[0]
    ref = ocoarse.apply(s, h, dims, x)
    mag = abs_apply(s, h, dims, x)
    # FP32 blocks and vector, sums in complex64
    s32, h32, x32 = (a.astype(np.complex64) for a in (s, h, x))
    y32 = ocoarse.apply(s32, h32, dims, x32).astype(np.complex128)
    assert_entrywise(y32, ref, stencil_factor(1, n) * mag, "fp32 emulation")
    # BF16 blocks, complex64 vector, complex64 sums
    yb = ocoarse.apply(_bf16(s).astype(np.complex64), _bf16(h).astype(np.complex64), dims, x32)
    assert_entrywise(yb.astype(np.complex128), ref, stencil_factor(2, n) * mag, "bf16 emulation")
    # BF16 vector too (the tensor-core path)
    yt = ocoarse.apply(_bf16(s), _bf16(h), dims, _bf16(_c64(x)))
    assert_entrywise(yt, ref, stencil_factor(2, n, x_prec="bf16") * mag, "bf16 operands emulation")


@pytest.mark.parametrize("kind", ["drop", "transpose", "sign"])
@pytest.mark.parametrize("prec", [1, 2])
def test_planted_mistake_leaves_bound(op24, kind, prec):
    s, h, dims = op24.self_blocks.numpy(), op24.hop_blocks.numpy(), op24.dims
    x = draws.rhs((906, 2), 1, s.shape[0] * op24.n)[0]
    if prec == 2:   # BF16 kernels: compared on their rounded operands
        s, h = bf16_operator(s, h, dims)
        x = _c64(x)
    ref = ocoarse.apply(s, h, dims, x)
    bad = _planted(s, h, dims, x, 7, kind)
    bound = stencil_factor(prec, op24.n, rounded_operands=prec == 2) * abs_apply(s, h, dims, x)
    with pytest.raises(AssertionError):
        assert_entrywise(bad, ref, bound, kind)


def test_bf16_rounded_operand_emulation_inside_bound(op24):
    s, h, dims = op24.self_blocks.numpy(), op24.hop_blocks.numpy(), op24.dims
    sr, hr = bf16_operator(s, h, dims)
    x32 = draws.rhs((906, 3), 1, s.shape[0] * op24.n)[0].astype(np.complex64)
    ref = ocoarse.apply(sr, hr, dims, x32.astype(np.complex128))
    y = ocoarse.apply(sr.astype(np.complex64), hr.astype(np.complex64), dims, x32).astype(np.complex128)
    bound = stencil_factor(2, op24.n, rounded_operands=True) * abs_apply(sr, hr, dims, x32)
    assert_entrywise(y, ref, bound, "bf16 rounded-operand emulation")


def test_schur_bound_emulation_and_planted():
    from synthetic.coarse_op import build_coarse_operator
    op = build_coarse_operator((907, 0), (8, 4, 4, 8), 16, -0.4, 1.0)
    s, h, dims = op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims
    n = op.n
    x = _c64(draws.rhs((907, 1), 1, s.shape[0] * n // 2)[0])
    ref = ooe.schur_apply(s, h, dims, x)
    mag = abs_schur(s, h, dims, x)
    # BF16 hops and inverse blocks, complex64 vectors and sums: inside the block-rounding bound,
    # and inside the accumulation-only bound around the oracle on the same rounded operands
    _, hr = bf16_operator(s, h, dims)
    inv = ooe.inverses(s)
    hb, ib, x32 = hr.astype(np.complex64), _bf16(inv).astype(np.complex64), x.astype(np.complex64)
    t = ooe.block_diag_apply(ib, dims, ooe.hop(hb, dims, x32, 1).astype(np.complex64), 1).astype(np.complex64)
    y = (x32 - ooe.block_diag_apply(ib, dims, ooe.hop(hb, dims, t, 0).astype(np.complex64), 0)).astype(np.complex128)
    assert_entrywise(y, ref, schur_factor(2, n) * mag, "bf16 schur emulation")
    ref_r, mag_r = bf16_schur(s, h, dims, x)
    assert_entrywise(y, ref_r, schur_factor(2, n, rounded_operands=True) * mag_r, "bf16 schur, rounded operands")
    # planted: one even site misses one hop of its second pass
    ev = ooe.sites(dims, 0)
    nb = neighbours(dims)
    xs = ev[5]
    od = ooe.sites(dims, 1)
    half = {int(o): i for i, o in enumerate(od)}
    for r, m, f in ((ref, mag, schur_factor(1, n)), (ref_r, mag_r, schur_factor(2, n, rounded_operands=True))):
        tt = ooe.block_diag_apply(inv, dims, ooe.hop(h, dims, x, 1), 1).reshape(-1, n)
        wrong = r.reshape(-1, n).copy()
        wrong[5] += inv[xs] @ (h[xs, 1] @ tt[half[int(nb[xs, 1])]])
        with pytest.raises(AssertionError):
            assert_entrywise(wrong.reshape(-1), r, f * m, "planted schur")
