"""GPU parity of the multi-right-hand-side tensor-core apply Y = D_c X (Eq. 6 per column;
BF16 blocks and vector fragments, FP32 accumulation) against the FP64 oracle.

Two bars per column:
  * against the exact operator: 1e-2 relative (block and vector entries rounded to 2^-9);
  * against the oracle applied, in FP64, to the BF16-rounded forward blocks (backward hops rebuilt
    from them by sigma3 F^H sigma3, as the kernel does) and the BF16-rounded vector, plus the
    twisted-mass term i mu sigma3 x taken from the unrounded (complex64) vector as the kernel's
    epilogue does: 2e-5 relative, and entry by entry (9n + 5) 2^-24 of (|D_c| |x|)_i on those
    operands.  Only the FP32 accumulation differs there (9n-term sums at 2^-24), so an index,
    sign or transposition error anywhere in the fragment layout is an O(1) difference.
Column counts cover one partial tile (2, 5), full passes (12) and a second pass (13, 24).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import abs_apply, assert_entrywise, make_op, rel, rhs, stencil_factor
from oracle import coarse as ocoarse
from oracle.lattice import neighbours

pytestmark = pytest.mark.gpu


def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return torch.complex(re, im).numpy()


@pytest.fixture(scope="module")
def ops():
    out = {}
    for nv, fdims in [(8, (6, 4, 4, 6)), (16, (6, 4, 4, 6)), (24, (4, 6, 4, 4))]:
        op = make_op((510, nv), fdims, nv)
        s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
        n = op.n
        s3 = ocoarse.sigma3(n // 2)
        nb = neighbours(op.dims)
        sr, hr = bf16(s), bf16(h)
        for mu in range(4):  # backward hop of x = s3 F_{x-mu,mu}^H s3 of the rounded forward block
            back = hr[nb[:, 4 + mu], mu]
            hr[:, 4 + mu] = s3[None, :, None] * np.conj(np.transpose(back, (0, 2, 1))) * s3[None, None, :]
        out[nv] = (op, s, h, sr, hr)
    return out


@pytest.mark.parametrize("nv", [8, 16, 24])
@pytest.mark.parametrize("nrhs", [2, 5, 12, 13, 24])
@pytest.mark.parametrize("mu", [0.0, 0.03])
@pytest.mark.parametrize("adjoint", [False, True])
def test_mrhs_matches_oracle(ops, nv, nrhs, mu, adjoint):
    from paper_2205_09104_gb300 import CoarseOp
    op, s, h, sr, hr = ops[nv]
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(2,),
                   max_nrhs=24)
    N = op.volume * op.n
    X = rhs((510, nv, nrhs), nrhs, N)
    Xd = torch.from_numpy(X).to("cuda", torch.complex64)
    Y = dev.apply(Xd, precision=2, adjoint=adjoint).cpu().numpy().astype(np.complex128)
    X32 = Xd.cpu().numpy().astype(np.complex128)
    Xr = bf16(X32)
    f = ocoarse.apply_adjoint if adjoint else ocoarse.apply
    s3 = np.tile(ocoarse.sigma3(op.n // 2), op.volume)
    for c in range(nrhs):
        exact = f(s, h, op.dims, X[c], mu)
        assert rel(Y[c], exact) <= 1e-2, (c, rel(Y[c], exact))
        rounded = f(sr, hr, op.dims, Xr[c], 0.0) + (-1j if adjoint else 1j) * mu * s3 * X32[c]
        assert rel(Y[c], rounded) <= 2e-5, (c, rel(Y[c], rounded))
        mag = abs_apply(sr, hr, op.dims, Xr[c], 0.0, adjoint=adjoint) + mu * np.abs(X32[c])
        assert_entrywise(Y[c], rounded, stencil_factor(2, op.n, rounded_operands=True) * mag,
                         f"nv={nv} nrhs={nrhs} mu={mu} adjoint={adjoint} column {c}")
    dev.close()


def test_mrhs_columns_independent(ops):
    """Column q of a 12-column apply equals the same column applied in a 2-column pass (no
    cross-talk between the columns of a tile or between tiles)."""
    from paper_2205_09104_gb300 import CoarseOp
    op = ops[16][0]
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, precisions=(2,), max_nrhs=12)
    N = op.volume * op.n
    X = torch.from_numpy(rhs((511, 0), 12, N)).to("cuda", torch.complex64)
    Y12 = dev.apply(X, precision=2)
    for q in (0, 5, 11):
        pair = torch.stack([X[q], X[(q + 1) % 12]])
        Y2 = dev.apply(pair, precision=2)
        assert rel(Y2[0].cpu().numpy(), Y12[q].cpu().numpy()) <= 1e-6
    dev.close()
