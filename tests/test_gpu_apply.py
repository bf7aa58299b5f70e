"""GPU parity of the coarse stencil apply (Sec. 2.2) against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic):
  FP64 blocks, FP64 accumulation : 1e-12 relative (norm-wise)
  FP32 blocks, FP32 accumulation : 2e-6 relative (9n-term sums of products rounded to 2^-24)
  BF16 blocks, FP32 accumulation : 1e-2 relative (entries rounded to 2^-9, random-sign sums)
"""
import numpy as np
import pytest
import torch

from gpu_helpers import make_op, rel, rhs, to_cuda
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
    for c in range(3):
        ref = ocoarse.apply(s, h, op.dims, X[c], mu)
        assert rel(y[c], ref) <= TOL[prec], (nv, prec, mu, c)


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
    ref = ocoarse.apply_adjoint(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    assert rel(y, ref) <= TOL[prec]


def test_apply_full_size_sampled_sites():
    """Wilson-clover 8^4 coarse lattice, n = 32 (the 131072-unknown workload): sampled sites one by one."""
    op = make_op((2, 0), (16, 16, 16, 16), 16, m0=-0.42, device="cuda")
    op.self_blocks, op.hop_blocks = op.self_blocks.cpu(), op.hop_blocks.cpu()
    dev = to_cuda(op)
    N = op.volume * op.n
    x = rhs((2, 0, 9), 1, N)[0]
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    from oracle.lattice import neighbours
    nb = neighbours(op.dims)
    xs = x.reshape(op.volume, op.n)
    rng = np.random.default_rng(3)
    sites = np.concatenate([[0, op.volume - 1], rng.integers(0, op.volume, 62)])
    for prec in (0, 1, 2):
        dt = torch.complex128 if prec == 0 else torch.complex64
        y = dev.apply(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy().reshape(op.volume, op.n)
        for site in sites:
            ref = s[site] @ xs[site] + sum(h[site, d] @ xs[nb[site, d]] for d in range(8))
            bound = TOL[0] if prec == 0 else 10 * TOL[prec]   # one site: fewer terms averaged
            assert rel(y[site], ref) <= bound


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
