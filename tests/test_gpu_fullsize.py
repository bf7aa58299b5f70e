"""Full-size checks in the benchmark's own configuration: the Wilson-clover 8^4 coarse lattice
(n = 32, 131072 unknowns, fine 16^4, m0 = -0.42), solved exactly as the benchmark solves it
(FP32 inner solves on the odd-even reduced, block-Jacobi preconditioned system, polynomial
chain on BF16 blocks, Arnoldi-step chunks replayed as CUDA graphs, FP64 refinement), with the
true residual recomputed by the FP64 oracle; and the reduced operator S at that size against
the oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import check_schur_entrywise, make_op, rel, rhs
from oracle import coarse as ocoarse
from oracle import oddeven as ooe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wilson8():
    op = make_op((2, 0), (16, 16, 16, 16), 16, m0=-0.42, device="cuda")
    op.self_blocks, op.hop_blocks = op.self_blocks.cpu(), op.hop_blocks.cpu()
    return op


def test_full_size_solves_in_benchmark_configuration(wilson8):
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_ZERO_GUESS, CoarseOp, solve_params)
    op = wilson8
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, precisions=(1, 2))
    N = op.volume * op.n
    p = solve_params(m=50, tol=1e-10, precision=1, poly_degree=4, defl_k=16, recycle_updates=10, inner_tol=2e-6,
                     max_restarts=100, max_ir=20, flags=COARSE_ZERO_GUESS | COARSE_POLY_BF16 | COARSE_ODD_EVEN)
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    # several right-hand sides: the first cycles run eagerly, the later ones replay step graphs
    for b in rhs((2, 0, 77), 4, N):
        x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
        x = x.cpu().numpy()
        res = np.linalg.norm(b - ocoarse.apply(s, h, op.dims, x)) / np.linalg.norm(b)
        assert info[0]["status"] == 0, info[0]
        assert res <= 1e-10, res
        assert abs(info[0]["rel_residual"] - res) <= 1e-6 * res + 1e-13
    dev.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (2, 3e-2)])
def test_full_size_schur(wilson8, prec, tol):
    from paper_2205_09104_gb300 import CoarseOp
    op = wilson8
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, precisions=(1, 2))
    x = rhs((2, 0, 78), 1, op.volume * op.n // 2)[0]
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = dev.schur(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy()
    ref = ooe.schur_apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x)
    assert rel(y, ref) <= tol, rel(y, ref)
    check_schur_entrywise(y, torch.from_numpy(x).to(dt).numpy(), op.self_blocks.numpy(), op.hop_blocks.numpy(),
                          op.dims, prec, 0.0, "8^4 n=32")
    dev.close()


def test_full_size_forward_error_ill_conditioned():
    """Wilson-clover 8^4, n = 32 at the most ill-conditioned sweep point m0 = -0.44: the solution of
    the benchmark's configuration against the oracle's own FP64 GCRO-DR solution at a 1e-13
    residual, forward error <= 1e-9."""
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_ZERO_GUESS, CoarseOp, solve_params)
    from oracle import krylov
    from synthetic import draws
    op = make_op((2, 0), (16, 16, 16, 16), 16, m0=-0.44, device="cuda")
    op.self_blocks, op.hop_blocks = op.self_blocks.cpu(), op.hop_blocks.cpu()
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, precisions=(1, 2))
    N = op.volume * op.n
    b = rhs((2, 0, 79), 1, N)[0]
    p = solve_params(m=50, tol=1e-10, precision=1, poly_degree=4, defl_k=16, recycle_updates=10, inner_tol=2e-6,
                     max_restarts=100, max_ir=20, flags=COARSE_ZERO_GUESS | COARSE_POLY_BF16 | COARSE_ODD_EVEN)
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
    x = x.cpu().numpy()
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    A = lambda v: ocoarse.apply(s, h, op.dims, v)
    theta, _ = krylov.poly_setup(A, draws.poly_start((2, 0, 80), N), 4)
    xs, oinfo, _ = krylov.gcrodr(A, b, m=50, k=16, tol=1e-13, precond=lambda v: krylov.poly_apply(A, theta, v))
    assert oinfo.converged
    res = np.linalg.norm(b - A(x)) / np.linalg.norm(b)
    assert info[0]["status"] == 0 and res <= 1e-10, (res, info[0])
    err = rel(x, xs)
    print(f"m0=-0.44: forward error {err:.3e}, residual {res:.3e}, {info[0]['iterations']} Arnoldi steps")
    assert err <= 1e-9, err
    dev.close()
