"""GPU parity of the odd-even reduced system with block-Jacobi left preconditioning (Sec. 2,
Sec. 3.2): S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe against the oracle, and solves through it
(COARSE_ODD_EVEN) against the oracle's direct solution of the full system.

Tolerances: FP64 1e-12 (as the FP64 stencil); FP32 1e-5 (two hop passes and two inverse
blocks of 9n-term FP32 sums); BF16 3e-2 (block entries rounded to 2^-9 in four products)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from gpu_helpers import check_schur_entrywise, make_op, rel, rhs
from oracle import coarse as ocoarse
from oracle import oddeven as ooe

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-2}


@pytest.fixture(scope="module")
def ops():
    # coarse 4^4 (n = 16), 4x2x2x4 (n = 32), 2x4x2x2 (n = 48): extents 2 make x+mu = x-mu
    return {8: make_op((530, 8), (8, 8, 8, 8), 8), 16: make_op((530, 16), (8, 4, 4, 8), 16),
            24: make_op((530, 24), (4, 8, 4, 4), 24)}


def _dev(op, mu, precisions=(1, 2)):
    from paper_2205_09104_gb300 import CoarseOp
    return CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=precisions)


@pytest.mark.parametrize("nv", [8, 16, 24])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("mu", [0.0, 0.03])
def test_schur_apply_matches_oracle(ops, nv, prec, mu):
    op = ops[nv]
    dev = _dev(op, mu)
    N2 = op.volume * op.n // 2
    x = rhs((531, nv), 1, N2)[0]
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = dev.schur(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy()
    ref = ooe.schur_apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    assert rel(y, ref) <= TOL[prec], rel(y, ref)
    xin = torch.from_numpy(x).to(dt).numpy()
    check_schur_entrywise(y, xin, op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, prec, mu, f"nv={nv} mu={mu}")
    dev.close()


def _solve(op, dev, b, flags, prec=1, d=4, k=8):
    from paper_2205_09104_gb300 import COARSE_ZERO_GUESS, solve_params
    p = solve_params(m=30, tol=1e-10, precision=prec, poly_degree=d, defl_k=k, recycle_updates=5,
                     inner_tol=1e-5 if prec == 1 else 1e-2, max_ir=40, flags=COARSE_ZERO_GUESS | flags)
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
    return x.cpu().numpy(), info[0]


@pytest.mark.parametrize("nv,mu", [(8, 0.0), (16, 0.0), (8, 0.03), (24, 0.0)])
@pytest.mark.parametrize("prec", [1, 2])
def test_odd_even_solve_matches_direct(ops, nv, mu, prec):
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN
    op = ops[nv]
    dev = _dev(op, mu)
    N = op.volume * op.n
    A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu).tocsc()
    for i, b in enumerate(rhs((532, nv), 2, N)):
        x, info = _solve(op, dev, b, COARSE_ODD_EVEN, prec=prec)
        assert info["status"] == 0, info
        res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert res <= 1e-10, res
        assert rel(x, spla.spsolve(A, b)) <= 1e-9
        assert abs(info["rel_residual"] - res) <= 1e-6 * res + 1e-13
    dev.close()


def test_odd_even_needs_fewer_iterations(ops):
    """The reduced, block-Jacobi preconditioned system converges in fewer Arnoldi steps."""
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN, COARSE_POLY_BF16
    op = ops[8]
    dev = _dev(op, 0.0)
    N = op.volume * op.n
    b = rhs((533, 0), 1, N)[0]
    _, full = _solve(op, dev, b, COARSE_POLY_BF16, k=0)
    _, red = _solve(op, dev, b, COARSE_ODD_EVEN | COARSE_POLY_BF16, k=0)
    assert red["status"] == 0 and full["status"] == 0
    assert red["iterations"] < full["iterations"], (red["iterations"], full["iterations"])
    dev.close()


def test_odd_extent_rejected():
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN, CoarseError
    op = make_op((534, 0), (6, 4, 4, 6), 8)  # coarse 3x2x2x3
    dev = _dev(op, 0.0)
    with pytest.raises(CoarseError):
        dev.schur(torch.zeros(op.volume * op.n // 2, dtype=torch.complex64, device="cuda"), precision=1)
    with pytest.raises(CoarseError):
        _solve(op, dev, rhs((534, 1), 1, op.volume * op.n)[0], COARSE_ODD_EVEN)
    dev.close()


@pytest.mark.parametrize("mu", [0.0, 0.03])
def test_odd_even_adjoint_solve(ops, mu):
    """D_c^H lambda = c through the reduced system of sigma3 D_c(-mu) sigma3 (its own inverses and
    solver for mu != 0), interleaved with forward solves on the same handle."""
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN, COARSE_ZERO_GUESS, solve_params
    op = ops[16]
    dev = _dev(op, mu)
    N = op.volume * op.n
    A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu).tocsc()
    p = solve_params(m=30, tol=1e-10, precision=1, poly_degree=4, defl_k=8, recycle_updates=5, inner_tol=2e-6,
                     max_ir=40, flags=COARSE_ZERO_GUESS | COARSE_ODD_EVEN)
    for i, c in enumerate(rhs((535, 0), 3, N)):
        lam, info = dev.solve(torch.from_numpy(c).cuda(), params=p, adjoint=True)
        lam = lam.cpu().numpy()
        assert info[0]["status"] == 0, info[0]
        res = np.linalg.norm(c - A.conj().T @ lam) / np.linalg.norm(c)
        assert res <= 1e-10, res
        x, info = dev.solve(torch.from_numpy(c).cuda(), params=p)          # forward in between
        assert np.linalg.norm(c - A @ x.cpu().numpy()) / np.linalg.norm(c) <= 1e-10
    dev.close()
