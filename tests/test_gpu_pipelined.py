"""GPU parity of latency-1 pipelined GMRES / GCRO-DR (Sec. 3.5, COARSE_PIPELINED) against the
oracle (oracle/pipelined.py) and against the library's classical cycles, through the C ABI.

In exact arithmetic the pipelined process produces the classical Arnoldi basis and Hessenberg
matrix, so in FP64 the pipelined solver takes the same Arnoldi steps as the classical one (the
oracle's pipelined solver counts them the same way) and reaches the same solution.  The
breakdown branch (t = ||v^a||^2 - sum |h|^2 - sum |b|^2 < 0) is driven deterministically by
installing a planted recycle space whose columns repeat one vector w, chosen so that the first
step's t is -3 (||A v0||^2 - |v0^H A v0|^2): the cycle must end with a reported breakdown and no
update; the proper space installed afterwards makes the same solve converge.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from gpu_helpers import make_op, rel, rhs, to_cuda
from oracle import coarse as ocoarse
from oracle import krylov
from oracle import pipelined as opl
from synthetic import draws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wilson4():
    return make_op((1, 0), (8, 8, 8, 8), 8, m0=-0.4)


def _params(**kw):
    from paper_2205_09104_gb300 import solve_params
    return solve_params(**kw)


def _lu(op, b, mu=0.0):
    A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu).tocsc()
    return spla.spsolve(A, b)


def _resid(op, x, b, mu=0.0):
    y = ocoarse.apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    return np.linalg.norm(b - y) / np.linalg.norm(b)


def test_pipelined_gmres_fp64_matches_classical_and_oracle(wilson4):
    from paper_2205_09104_gb300 import COARSE_PIPELINED, COARSE_ZERO_GUESS, PREC_FP64
    op = wilson4
    N = op.volume * op.n
    v0 = draws.poly_start((1, 21), N)
    b = rhs((1, 22), 1, N)[0]
    its = {}
    for flags in (0, COARSE_PIPELINED):
        dev = to_cuda(op, precisions=())
        p = _params(m=12, tol=1e-10, precision=PREC_FP64, poly_degree=4, defl_k=0, max_restarts=200,
                    poly_start=torch.from_numpy(v0).cuda(), flags=COARSE_ZERO_GUESS | flags)
        x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
        x = x.cpu().numpy()
        assert info[0]["status"] == 0 and info[0]["breakdowns"] == 0, info[0]
        assert _resid(op, x, b) <= 1e-10
        assert rel(x, _lu(op, b)) <= 1e-9
        its[flags] = (info[0]["iterations"], info[0]["cycles"])
        dev.close()
    assert abs(its[0][0] - its[COARSE_PIPELINED][0]) <= 1, its
    # the oracle's pipelined GMRES on the same operator and polynomial start
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    D = lambda v: ocoarse.apply(s, h, op.dims, v)
    theta, _ = krylov.poly_setup(D, v0, 4)
    _, oinfo, bd = opl.p1_gmres(D, b, 12, 1e-10, precond=lambda v: krylov.poly_apply(D, theta, v))
    assert oinfo.converged and bd == 0
    assert abs(oinfo.iterations - its[COARSE_PIPELINED][0]) <= 2, (oinfo.iterations, its)


def test_pipelined_gcrodr_fp64_matches_classical(wilson4):
    """GCRO-DR(12, k = 4) over three right-hand sides with recycling, classical and pipelined."""
    from paper_2205_09104_gb300 import COARSE_PIPELINED, COARSE_ZERO_GUESS, PREC_FP64
    op = wilson4
    N = op.volume * op.n
    v0 = draws.poly_start((1, 23), N)
    bs = rhs((1, 24), 3, N)
    its = {}
    for flags in (0, COARSE_PIPELINED):
        dev = to_cuda(op, precisions=())
        p = _params(m=12, tol=1e-10, precision=PREC_FP64, poly_degree=4, defl_k=4, recycle_updates=10,
                    max_restarts=200, poly_start=torch.from_numpy(v0).cuda(), flags=COARSE_ZERO_GUESS | flags)
        its[flags] = []
        for b in bs:
            x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
            x = x.cpu().numpy()
            assert info[0]["status"] == 0 and info[0]["breakdowns"] == 0, info[0]
            assert _resid(op, x, b) <= 1e-10
            assert rel(x, _lu(op, b)) <= 1e-9
            its[flags].append(info[0]["iterations"])
        dev.close()
    for a, c in zip(its[0], its[COARSE_PIPELINED]):
        assert abs(a - c) <= 2, its


@pytest.mark.parametrize("odd_even", [False, True])
def test_pipelined_mixed_precision_reaches_tolerance(wilson4, odd_even):
    """FP32 inner solves (chain on BF16 blocks), pipelined pp-GMRES and pipelined GCRO-DR, with and
    without the odd-even reduction: true residual 1e-10 (the oracle's), forward error 1e-9."""
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_PIPELINED, COARSE_POLY_BF16, COARSE_RECYCLE_FULL_CYCLE,
                                        COARSE_ZERO_GUESS, PREC_FP32)
    op = wilson4
    N = op.volume * op.n
    dev = to_cuda(op, precisions=(1, 2))
    base = COARSE_ZERO_GUESS | COARSE_POLY_BF16 | COARSE_PIPELINED | (COARSE_ODD_EVEN if odd_even else 0)
    bs = rhs((1, 25), 4, N)
    for i, (k, extra) in enumerate(((0, 0), (8, COARSE_RECYCLE_FULL_CYCLE), (8, 0), (8, 0))):
        p = _params(m=30, tol=1e-10, precision=PREC_FP32, poly_degree=4, defl_k=k, recycle_updates=4,
                    inner_tol=1e-5, max_ir=30, flags=base | extra)
        x, info = dev.solve(torch.from_numpy(bs[i]).cuda(), params=p)
        x = x.cpu().numpy()
        assert info[0]["status"] == 0, info[0]
        assert _resid(op, x, bs[i]) <= 1e-10
        assert rel(x, _lu(op, bs[i])) <= 1e-9
    assert dev.recycle_check(PREC_FP32, odd_even=odd_even)["k"] == 8
    dev.close()


def test_pipelined_breakdown_on_planted_recycle_space(wilson4):
    from paper_2205_09104_gb300 import COARSE_PIPELINED, COARSE_ZERO_GUESS, PREC_FP64
    op = wilson4
    N = op.volume * op.n
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    v0 = draws.poly_start((1, 26), N)
    b = rhs((1, 27), 2, N)
    dev = to_cuda(op, precisions=())
    kw = dict(m=12, tol=1e-10, precision=PREC_FP64, poly_degree=4, defl_k=4, recycle_updates=10, max_restarts=200,
              poly_start=torch.from_numpy(v0).cuda())
    # a classical solve creates the solver, its polynomial and a proper recycle space
    dev.solve(torch.from_numpy(b[0]).cuda(), params=_params(flags=COARSE_ZERO_GUESS, **kw))
    U, C = dev.recycle_get(PREC_FP64)
    assert U.shape[0] == 4
    # planted: 4 copies of w, w _|_ b so the cycle starts from v0 = b/||b||, and w the part of
    # A v0 orthogonal to v0: t = ||a||^2 - 4 (||a||^2 - |h00|^2) - |h00|^2 < 0 at the first step
    D = lambda v: ocoarse.apply(s, h, op.dims, v)
    theta = dev.poly(PREC_FP64)
    Aop = lambda v: D(krylov.poly_apply(D, theta, v))
    v = b[1] / np.linalg.norm(b[1])
    a = Aop(v)
    w = a - v * np.vdot(v, a)
    w /= np.linalg.norm(w)
    Wt = torch.from_numpy(np.stack([w] * 4)).cuda().contiguous()
    dev.recycle_set(PREC_FP64, U.contiguous(), Wt, updates=10)
    p = _params(flags=COARSE_ZERO_GUESS | COARSE_PIPELINED, max_ir=3, **dict(kw, max_restarts=3))
    x, info = dev.solve(torch.from_numpy(b[1]).cuda(), params=p, allow_not_converged=True)
    assert info[0]["breakdowns"] >= 1, info[0]
    assert info[0]["status"] == -4, info[0]
    assert np.all(np.isfinite(x.cpu().numpy()))
    assert dev.recycle_check(PREC_FP64)["chc_minus_i"] >= 0.5     # the planted space is not orthonormal
    # the proper space back: the same solve converges without a breakdown
    dev.recycle_set(PREC_FP64, U.contiguous(), C.contiguous(), updates=10)
    chk = dev.recycle_check(PREC_FP64)
    assert chk["au_minus_c"] <= 1e-10 and chk["chc_minus_i"] <= 1e-12
    x, info = dev.solve(torch.from_numpy(b[1]).cuda(), params=_params(flags=COARSE_ZERO_GUESS | COARSE_PIPELINED, **kw))
    assert info[0]["status"] == 0 and info[0]["breakdowns"] == 0, info[0]
    assert _resid(op, x.cpu().numpy(), b[1]) <= 1e-10
    dev.close()
