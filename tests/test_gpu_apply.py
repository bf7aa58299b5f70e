"""GPU parity of the coarse stencil apply (Sec. 2.2) against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic):
  FP64 blocks, FP64 accumulation : 1e-12 relative (norm-wise)
  FP32 blocks, FP32 accumulation : 2e-6 relative (9n-term sums of products rounded to 2^-24)
  BF16 blocks, FP32 accumulation : 1e-2 relative (entries rounded to 2^-9, random-sign sums)
and, entry by entry, |y_i - ref_i| <= c (|D_c| |x|)_i with c from gpu_helpers.stencil_factor
(block rounding + vector rounding + (9n + 5) accumulation roundings); BF16 applies also entry by
entry against the oracle on their BF16-rounded blocks, where only the FP32 accumulation differs.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import (abs_apply, abs_apply_at, assert_entrywise, bf16, bf16_blocks_of, bf16_operator, make_op, rel,
                         rhs, site_blocks, stencil_factor, to_cuda)
from oracle import coarse as ocoarse

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6, 2: 1e-2}


@pytest.fixture(scope="module")
def ops():
    out = {}
    # ragged coarse lattices (3x2x2x3 = 36 sites: not a multiple of the 4 sites per CTA)
    for nv, fdims in [(8, (6, 4, 4, 6)), (16, (6, 4, 4, 6)), (24, (4, 6, 4, 4))]:
        out[nv] = make_op((500, nv), fdims, nv)
    return out


@pytest.mark.parametrize("nv", [8, 16, 24])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("mu", [0.0, 0.01])
def test_apply_matches_oracle(ops, nv, prec, mu):
    op = ops[nv]
    dev = to_cuda(op, mu=mu, max_nrhs=3)
    N = op.volume * op.n
    X = rhs((500, nv, 1), 3, N)
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = dev.apply(torch.from_numpy(X).to("cuda", dt), precision=prec).cpu().numpy()
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    s3v = np.tile(ocoarse.sigma3(op.n // 2), op.volume)
    for c in range(3):
        ref = ocoarse.apply(s, h, op.dims, X[c], mu)
        assert rel(y[c], ref) <= TOL[prec], (nv, prec, mu, c)
        # three BF16 columns run the tensor-core multi-right-hand-side kernel, which also rounds x to BF16
        xp = "bf16" if prec == 2 else None
        bound = stencil_factor(prec, op.n, x_prec=xp) * abs_apply(s, h, op.dims, X[c], mu)
        assert_entrywise(y[c], ref, bound, f"nv={nv} prec={prec} mu={mu} column {c}")
        if prec == 2:
            sr, hr = bf16_operator(s, h, op.dims)
            x32 = X[c].astype(np.complex64).astype(np.complex128)
            ref_r = ocoarse.apply(sr, hr, op.dims, bf16(x32), 0.0) + 1j * mu * s3v * x32
            bound = stencil_factor(2, op.n, rounded_operands=True) * (abs_apply(sr, hr, op.dims, bf16(x32))
                                                                      + mu * np.abs(x32))
            assert_entrywise(y[c], ref_r, bound, f"nv={nv} bf16 rounded operands mu={mu} column {c}")


@pytest.mark.parametrize("nv", [8, 24])
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_adjoint_matches_oracle(ops, nv, prec):
    op = ops[nv]
    mu = 0.02
    dev = to_cuda(op, mu=mu)
    N = op.volume * op.n
    x = rhs((501, nv), 1, N)[0]
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = dev.apply(torch.from_numpy(x).to("cuda", dt), precision=prec, adjoint=True).cpu().numpy()
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    ref = ocoarse.apply_adjoint(s, h, op.dims, x, mu)
    assert rel(y, ref) <= TOL[prec]
    bound = stencil_factor(prec, op.n) * abs_apply(s, h, op.dims, x, mu, adjoint=True)
    assert_entrywise(y, ref, bound, f"adjoint nv={nv} prec={prec}")


def test_apply_full_size_sampled_sites():
    """Wilson-clover 8^4 coarse lattice, n = 32 (the 131072-unknown workload): sampled sites one by one."""
    op = make_op((2, 0), (16, 16, 16, 16), 16, m0=-0.42, device="cuda")
    _sampled_sites(op, 0.0, (2, 0, 9), 64)


def _sampled_sites(op, mu, key, count):
    dev = to_cuda(op, mu=mu)
    N = op.volume * op.n
    x = rhs(key, 1, N)[0]
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([[0, op.volume - 1], rng.integers(0, op.volume, count - 2)]))
    blocks_of = site_blocks(op, sites)
    ref = ocoarse.apply_at(blocks_of, op.dims, x, sites, mu)
    mag = abs_apply_at(blocks_of, op.dims, x, sites, mu)
    x32 = x.astype(np.complex64).astype(np.complex128)
    rb = bf16_blocks_of(blocks_of, op.dims)
    ref_r = ocoarse.apply_at(rb, op.dims, x32, sites, mu)
    mag_r = abs_apply_at(rb, op.dims, x32, sites, mu)
    for prec in (0, 1, 2):
        dt = torch.complex128 if prec == 0 else torch.complex64
        y = dev.apply(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy().reshape(op.volume, op.n)
        assert_entrywise(y[sites], ref, stencil_factor(prec, op.n) * mag, f"sampled sites prec {prec}")
        if prec == 2:
            assert_entrywise(y[sites], ref_r, stencil_factor(2, op.n, rounded_operands=True) * mag_r,
                             "sampled sites, bf16 rounded operands")
    dev.close()


def test_gamma5_violation_rejected(ops):
    from paper_2205_09104_gb300 import CoarseError, CoarseOp
    op = ops[8]
    h = op.hop_blocks.clone()
    h[3, 5, 1, 2] += 0.1
    with pytest.raises(CoarseError) as e:
        CoarseOp(op.self_blocks.cuda(), h.cuda(), op.dims, op.nv)
    assert e.value.code == -8


def test_invalid_arguments(ops):
    from paper_2205_09104_gb300 import CoarseError
    op = ops[8]
    dev = to_cuda(op, precisions=())
    N = op.volume * op.n
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    with pytest.raises(CoarseError):
        dev.apply(x, precision=1)            # FP32 copy not enabled
    with pytest.raises(CoarseError):
        dev.apply(torch.zeros(2 * N, dtype=torch.complex128, device="cuda"))  # nrhs > max_nrhs
