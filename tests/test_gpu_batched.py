"""GPU parity of coarse_solve_batched: uneven operators (n = 16, 32, 48) with several
right-hand sides each, advanced in lockstep (one launch per phase; the whole solve one CUDA
graph whose conditional loops the device drives).  Every column is checked against the FP64 oracle's direct solution and the
true FP64 residual is recomputed by the oracle.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from gpu_helpers import make_op, rel, rhs
from oracle import coarse as ocoarse

pytestmark = pytest.mark.gpu

CASES = [  # key, fine dims, nv, mu, nrhs
    ((800, 0), (4, 4, 4, 4), 8, 0.0, 2),
    ((801, 0), (6, 4, 4, 6), 16, 0.0, 3),
    ((802, 0), (4, 6, 4, 4), 24, 0.01, 1),
    ((803, 0), (8, 8, 8, 8), 8, 0.0, 2),
]


@pytest.fixture(scope="module")
def problems():
    out = []
    for key, fdims, nv, mu, nr in CASES:
        op = make_op(key, fdims, nv, m0=-0.4)
        N = op.volume * op.n
        B = rhs((*key, 5), nr, N)
        A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu).tocsc()
        lu = spla.splu(A)
        X = np.stack([lu.solve(B[c]) for c in range(nr)])
        out.append((op, mu, B, X, A))
    return out


@pytest.mark.parametrize("prec,chain_bf16", [(1, False), (2, False), (1, True)])
def test_batched_matches_oracle(problems, prec, chain_bf16):
    """chain_bf16: FP32 inner solves whose polynomial-chain phases read BF16 blocks."""
    from paper_2205_09104_gb300 import COARSE_POLY_BF16, COARSE_ZERO_GUESS, CoarseOp, solve_batched, solve_params
    ops, bs, xs = [], [], []
    for op, mu, B, X, A in problems:
        ops.append(CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(1, 2),
                            max_nrhs=4))
        bs.append(torch.from_numpy(B).cuda().contiguous())
        xs.append(torch.zeros_like(bs[-1]))
    p = solve_params(m=20, tol=1e-10, precision=prec, poly_degree=4, defl_k=4, recycle_updates=10,
                     inner_tol=1e-5 if prec == 1 else 1e-2, max_restarts=50, max_ir=40,
                     flags=COARSE_ZERO_GUESS | (COARSE_POLY_BF16 if chain_bf16 else 0))
    infos = solve_batched(ops, bs, xs, p)
    q = 0
    for (op, mu, B, X, A), x in zip(problems, xs):
        xg = x.cpu().numpy()
        for c in range(B.shape[0]):
            res = np.linalg.norm(B[c] - A @ xg[c]) / np.linalg.norm(B[c])
            assert res <= 1e-10, (q, res, infos[q])
            assert rel(xg[c], X[c]) <= 1e-9, (q, infos[q])
            assert infos[q]["status"] == 0
            assert abs(infos[q]["rel_residual"] - res) <= 1e-6 * max(res, 1e-12) + 1e-13
            q += 1
    for o in ops:
        o.close()


def test_batched_equals_single_operator_path(problems):
    """Same columns through coarse_solve (one operator at a time): both meet the bar."""
    from paper_2205_09104_gb300 import CoarseOp, solve_batched, solve_params
    op, mu, B, X, A = problems[1]
    p = solve_params(m=20, tol=1e-10, precision=1, poly_degree=4, defl_k=4, inner_tol=1e-5)
    d1 = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, max_nrhs=4)
    xa, _ = d1.solve(torch.from_numpy(B).cuda().contiguous(), params=p)
    d2 = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, max_nrhs=4)
    xb = torch.zeros(B.shape, dtype=torch.complex128, device="cuda")
    solve_batched([d2], [torch.from_numpy(B).cuda().contiguous()], [xb], p)
    assert rel(xa.cpu().numpy(), X) <= 1e-9
    assert rel(xb.cpu().numpy(), X) <= 1e-9
    d1.close()
    d2.close()


def test_batched_bounds_and_statistics(problems):
    """The batched solve is one graph whose loops the device ends: with max_ir = 1 and
    max_restarts = 1 it stops after one cycle of at most m steps per solve and reports the
    solves as not converged; a zero right-hand side is done before any step; the statistics of a
    converged run (cycles, Arnoldi steps, refinement steps) are those of real work."""
    from paper_2205_09104_gb300 import COARSE_ZERO_GUESS, CoarseOp, solve_batched, solve_params
    ops, bs, xs = [], [], []
    for op, mu, B, X, A in problems[:2]:
        ops.append(CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(1, 2),
                            max_nrhs=4))
        b = torch.from_numpy(B).cuda().contiguous()
        bs.append(b)
        xs.append(torch.zeros_like(b))
    bs[1][0].zero_()   # a zero right-hand side
    m = 6
    p = solve_params(m=m, tol=1e-10, precision=1, poly_degree=2, defl_k=0, inner_tol=1e-5, max_restarts=1, max_ir=1,
                     flags=COARSE_ZERO_GUESS)
    infos = solve_batched(ops, bs, xs, p, allow_not_converged=True)
    assert infos[2]["status"] == 0 and infos[2]["iterations"] == 0 and infos[2]["ir_steps"] == 0
    for q in (0, 1, 3, 4):
        assert infos[q]["status"] == -4, infos[q]
        assert infos[q]["ir_steps"] == 1 and infos[q]["cycles"] == 1 and 1 <= infos[q]["iterations"] <= m
        assert 0.0 < infos[q]["rel_residual"] < 1.0
    for x in xs:
        assert torch.isfinite(torch.view_as_real(x)).all()
    p = solve_params(m=20, tol=1e-10, precision=1, poly_degree=4, defl_k=0, inner_tol=1e-5, max_restarts=50, max_ir=40,
                     flags=COARSE_ZERO_GUESS)
    infos = solve_batched(ops, bs, xs, p)
    for q, inf in enumerate(infos):
        if q == 2:
            continue
        assert inf["status"] == 0 and inf["ir_steps"] >= 2 and inf["cycles"] >= inf["ir_steps"]
        assert inf["iterations"] >= inf["cycles"]
    for o in ops:
        o.close()


EO_CASES = [  # even coarse extents: key, fine dims, nv, mu, nrhs
    ((810, 0), (4, 4, 4, 4), 8, 0.0, 2),
    ((811, 0), (8, 4, 4, 8), 16, 0.0, 3),
    ((812, 0), (4, 8, 4, 4), 24, 0.01, 1),
    ((813, 0), (8, 8, 8, 8), 8, 0.02, 2),
]


@pytest.fixture(scope="module")
def eo_problems():
    out = []
    for key, fdims, nv, mu, nr in EO_CASES:
        op = make_op(key, fdims, nv, m0=-0.4)
        N = op.volume * op.n
        B = rhs((*key, 5), nr, N)
        A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu).tocsc()
        lu = spla.splu(A)
        X = np.stack([lu.solve(B[c]) for c in range(nr)])
        out.append((op, mu, B, X, A))
    return out


@pytest.mark.parametrize("prec,chain_bf16,k", [(1, False, 4), (1, True, 4), (2, False, 0), (1, True, 0)])
def test_batched_odd_even_matches_oracle(eo_problems, prec, chain_bf16, k):
    """COARSE_ODD_EVEN in the batched engine (Sec. 2, Sec. 3.2): every solve's inner system is the
    block-Jacobi preconditioned reduced S on the even sites, the odd sites retrieved per
    refinement step; every column against the oracle's direct solution of the full system."""
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_ZERO_GUESS, CoarseOp, solve_batched,
                                        solve_params)
    ops, bs, xs = [], [], []
    for op, mu, B, X, A in eo_problems:
        ops.append(CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(1, 2),
                            max_nrhs=4))
        bs.append(torch.from_numpy(B).cuda().contiguous())
        xs.append(torch.zeros_like(bs[-1]))
    p = solve_params(m=20, tol=1e-10, precision=prec, poly_degree=4, defl_k=k, recycle_updates=10,
                     inner_tol=1e-5 if prec == 1 else 1e-2, max_restarts=50, max_ir=40,
                     flags=COARSE_ZERO_GUESS | COARSE_ODD_EVEN | (COARSE_POLY_BF16 if chain_bf16 else 0))
    infos = solve_batched(ops, bs, xs, p)
    q = 0
    for (op, mu, B, X, A), x in zip(eo_problems, xs):
        xg = x.cpu().numpy()
        for c in range(B.shape[0]):
            res = np.linalg.norm(B[c] - A @ xg[c]) / np.linalg.norm(B[c])
            assert res <= 1e-10, (q, res, infos[q])
            assert rel(xg[c], X[c]) <= 1e-9, (q, infos[q])
            assert infos[q]["status"] == 0
            assert abs(infos[q]["rel_residual"] - res) <= 1e-6 * max(res, 1e-12) + 1e-13
            q += 1
    for o in ops:
        o.close()


def test_batched_odd_even_rejects_odd_extents(problems):
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN, COARSE_ZERO_GUESS, CoarseError, CoarseOp, solve_batched, solve_params
    op, mu, B, X, A = problems[1]                      # coarse 3x2x2x3
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, max_nrhs=4)
    b = torch.from_numpy(B).cuda().contiguous()
    p = solve_params(m=20, tol=1e-10, precision=1, poly_degree=4, inner_tol=1e-5,
                     flags=COARSE_ZERO_GUESS | COARSE_ODD_EVEN)
    with pytest.raises(CoarseError) as e:
        solve_batched([dev], [b], [torch.zeros_like(b)], p)
    assert e.value.code == -1
    dev.close()
