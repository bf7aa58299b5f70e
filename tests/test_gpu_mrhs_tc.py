"""GPU parity of the tcgen05 multi-right-hand-side apply (csrc/mrhs_tc.cu: BF16 operands read by
the tensor core from shared memory, FP32 accumulators in tensor memory) for n = 32 and 48, with
each launch configuration the autotuner may pick fixed in turn through coarse_autotune_set:
one to three CTAs per SM, all stages that fit or a 2- / 3-stage ring, and passes of 1 to 16
columns (13-16 columns: one pass of four column tiles, which only this kernel runs).

The bar is the one of the mma.sync kernel: against the oracle applied in FP64 to the BF16-rounded
forward blocks (backward hops rebuilt from them by sigma3 F^H sigma3) and the BF16-rounded
columns, plus the twisted-mass term from the unrounded columns, entry by entry within
(9n + 5) 2^-24 of (|D_c| |x|)_i.  Only the FP32 accumulation differs there, so a wrong core
matrix, a transposed plane, a sign of sigma3 or a column from the wrong accumulator is an O(1)
difference.

On the small lattices every CTA gets one site, so with 2 stages per ring (self / forward hops,
backward hops) each ring wraps two or three times per site; on the
coarse 8^4 lattice (4096 sites over 152 to 456 CTAs) every CTA walks 9-27 sites, so both tensor
memory accumulator sets are reused many times and the stage phases flip throughout.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import (abs_apply, abs_apply_at, assert_entrywise, bf16, bf16_blocks_of, make_op, rhs, site_blocks,
                         stencil_factor)
from oracle import coarse as ocoarse
from oracle.lattice import neighbours

pytestmark = pytest.mark.gpu

# (100 + CTAs per SM, stages (0: all that fit)); 3 CTAs per SM exist only for passes of up to 8
# columns (their tensor memory), so passes of 9-16 columns run that one with 2
CONFIGS = [(101, 0), (102, 0), (101, 2), (102, 3), (103, 0), (103, 2)]


def _keys(n, V):
    vb = V.bit_length() - 1
    return [(t, f"mrhs/n{n}/t{t}/v{vb}") for t in (1, 2, 3, 4)]


def _fix(n, V, cfg):
    from paper_2205_09104_gb300 import autotune_set
    for t, k in _keys(n, V):
        autotune_set(k, cfg[0] if t <= 2 else min(cfg[0], 102), *cfg[1:])


def _forget(n, V):
    from paper_2205_09104_gb300 import autotune_set
    for _, k in _keys(n, V):
        autotune_set(k, -1)


@pytest.fixture(scope="module")
def small():
    out = {}
    for nv, fdims in [(16, (6, 4, 4, 6)), (24, (4, 6, 4, 4))]:
        op = make_op((530, nv), fdims, nv)
        s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
        s3 = ocoarse.sigma3(op.n // 2)
        nb = neighbours(op.dims)
        sr, hr = bf16(s), bf16(h)
        for mu in range(4):
            back = hr[nb[:, 4 + mu], mu]
            hr[:, 4 + mu] = s3[None, :, None] * np.conj(np.transpose(back, (0, 2, 1))) * s3[None, None, :]
        out[nv] = (op, sr, hr)
    return out


@pytest.mark.parametrize("nv", [16, 24])
@pytest.mark.parametrize("cfg", CONFIGS)
@pytest.mark.parametrize("nrhs", [2, 7, 12, 13, 16, 19])
@pytest.mark.parametrize("adjoint", [False, True])
def test_tc_small_lattices(small, nv, cfg, nrhs, adjoint):
    from paper_2205_09104_gb300 import CoarseOp
    op, sr, hr = small[nv]
    mu = 0.03
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(2,), max_nrhs=24)
    _fix(op.n, op.volume, cfg)
    try:
        N = op.volume * op.n
        Xd = torch.from_numpy(rhs((530, nv, nrhs), nrhs, N)).to("cuda", torch.complex64)
        Y = dev.apply(Xd, precision=2, adjoint=adjoint).cpu().numpy().astype(np.complex128)
    finally:
        _forget(op.n, op.volume)
        dev.close()
    X32 = Xd.cpu().numpy().astype(np.complex128)
    Xr = bf16(X32)
    f = ocoarse.apply_adjoint if adjoint else ocoarse.apply
    s3 = np.tile(ocoarse.sigma3(op.n // 2), op.volume)
    for c in range(nrhs):
        ref = f(sr, hr, op.dims, Xr[c], 0.0) + (-1j if adjoint else 1j) * mu * s3 * X32[c]
        mag = abs_apply(sr, hr, op.dims, Xr[c], 0.0, adjoint=adjoint) + mu * np.abs(X32[c])
        assert_entrywise(Y[c], ref, stencil_factor(2, op.n, rounded_operands=True) * mag,
                         f"tcgen05 nv={nv} cfg={cfg} nrhs={nrhs} adjoint={adjoint} column {c}")


@pytest.fixture(scope="module")
def coarse8():
    out = {}
    for nv in (16, 24):
        out[nv] = make_op((531, nv), (16, 16, 16, 16), nv, device="cuda")
    return out


@pytest.mark.parametrize("nv", [16, 24])
@pytest.mark.parametrize("cfg", CONFIGS)
def test_tc_many_sites_per_cta(coarse8, nv, cfg):
    """Coarse 8^4: 12 columns plain and adjoint, 5 columns plain, on sampled sites."""
    from paper_2205_09104_gb300 import CoarseOp
    op = coarse8[nv]
    mu = 0.02
    V, n = op.volume, op.n
    rng = np.random.default_rng(40 + nv)
    sites = np.unique(np.concatenate([[0, V - 1], rng.integers(0, V, 30)]))
    rb = bf16_blocks_of(site_blocks(op, sites), op.dims)
    s3 = ocoarse.sigma3(n // 2)
    dev = CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=mu, precisions=(2,), max_nrhs=16)
    _fix(n, V, cfg)
    try:
        for nrhs, adjoint in ((12, False), (12, True), (5, False), (8, True), (16, False), (14, True)):
            Xd = torch.from_numpy(rhs((531, nv, nrhs), nrhs, V * n)).to("cuda", torch.complex64)
            Y = dev.apply(Xd, precision=2, adjoint=adjoint).cpu().numpy().astype(np.complex128)
            X32 = Xd.cpu().numpy().astype(np.complex128)
            Xr = bf16(X32)
            for c in range(nrhs):
                xs = X32[c].reshape(V, n)[sites]
                if adjoint:   # D^H = sigma3 D(-mu) sigma3
                    w = (Xr[c].reshape(V, n) * s3[None, :]).reshape(-1)
                    ref = s3[None, :] * ocoarse.apply_at(rb, op.dims, w, sites, 0.0) - 1j * mu * s3[None, :] * xs
                else:
                    ref = ocoarse.apply_at(rb, op.dims, Xr[c], sites, 0.0) + 1j * mu * s3[None, :] * xs
                mag = abs_apply_at(rb, op.dims, Xr[c], sites, 0.0) + mu * np.abs(xs)
                got = Y[c].reshape(V, n)[sites]
                assert_entrywise(got, ref, stencil_factor(2, n, rounded_operands=True) * mag,
                                 f"tcgen05 8^4 nv={nv} cfg={cfg} nrhs={nrhs} adjoint={adjoint} column {c}")
    finally:
        _forget(n, V)
        dev.close()
