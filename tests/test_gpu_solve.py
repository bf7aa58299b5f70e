"""GPU parity of the coarsest-level solver against the FP64 oracle, through the C ABI.

Bars: true FP64 relative residual <= 1e-10 (recomputed by the oracle), forward
error vs the oracle's direct solution <= max(1e-9, kappa * 1e-10 * 10) where kappa
is computed densely for the small cases.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from gpu_helpers import make_op, rel, rhs, to_cuda
from oracle import coarse as ocoarse
from oracle import krylov

pytestmark = pytest.mark.gpu


def _lu(op, b, mu=0.0, adjoint=False):
    A = ocoarse.assemble(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, mu)
    if adjoint:
        A = A.conj().T
    return spla.spsolve(A.tocsc(), b), A


def _resid(op, x, b, mu=0.0):
    y = ocoarse.apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    return np.linalg.norm(b - y) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def wilson4():
    """Fine 8^4 Wilson-clover, c_sw = 1, m0 = -0.4, Nv = 8: coarse 4^4, 16 dof/site (4096 unknowns)."""
    return make_op((1, 0), (8, 8, 8, 8), 8, m0=-0.4)


@pytest.fixture(scope="module")
def small():
    return make_op((600, 0), (6, 4, 4, 6), 8, m0=-0.4)


def _params(**kw):
    from paper_2205_09104_gb300 import solve_params
    return solve_params(**kw)


def test_plain_fp64_gmres_wilson4(wilson4):
    from paper_2205_09104_gb300 import PREC_FP64
    dev = to_cuda(wilson4, precisions=())
    N = wilson4.volume * wilson4.n
    b = rhs((1, 0), 1, N)[0]
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=_params(m=30, tol=1e-10, precision=PREC_FP64))
    x = x.cpu().numpy()
    assert info[0]["status"] == 0
    assert _resid(wilson4, x, b) <= 1e-10
    xs, A = _lu(wilson4, b)
    assert rel(x, xs) <= 1e-9
    assert info[0]["rel_residual"] <= 1e-10


def test_fp64_residual_entry_point(wilson4):
    dev = to_cuda(wilson4, precisions=())
    N = wilson4.volume * wilson4.n
    b = rhs((1, 0), 2, N)
    r, rn, bn = dev.residual(torch.from_numpy(b[0]).cuda(), torch.from_numpy(b[1]).cuda())
    ref = b[0] - ocoarse.apply(wilson4.self_blocks.numpy(), wilson4.hop_blocks.numpy(), wilson4.dims, b[1])
    assert rel(r.cpu().numpy(), ref) <= 1e-13
    assert abs(rn - np.linalg.norm(ref)) <= 1e-12 * rn
    assert abs(bn - np.linalg.norm(b[0])) <= 1e-12 * bn


@pytest.mark.parametrize("d", [1, 4, 8])
def test_poly_roots_match_oracle(small, d):
    """Harmonic Ritz values of d Arnoldi steps from the same start vector (Sec. 3.3), FP64 on both sides."""
    from paper_2205_09104_gb300 import PREC_FP64
    dev = to_cuda(small, precisions=())
    N = small.volume * small.n
    from synthetic import draws
    v0 = draws.poly_start((600, 1), N)
    b = rhs((600, 2), 1, N)[0]
    p = _params(m=10, tol=1e-10, precision=PREC_FP64, poly_degree=d, poly_start=torch.from_numpy(v0).cuda())
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
    theta_gpu = dev.poly(PREC_FP64)
    A = lambda v: ocoarse.apply(small.self_blocks.numpy(), small.hop_blocks.numpy(), small.dims, v)
    theta_ref, _ = krylov.poly_setup(A, v0, d)
    assert len(theta_gpu) == d
    for t in theta_gpu:
        assert np.abs(theta_ref - t).min() <= 1e-8 * abs(t)
    # Leja order: the first root has the largest modulus; each next maximises the distance product
    assert abs(theta_gpu[0]) >= np.abs(theta_gpu).max() * (1 - 1e-12)
    assert _resid(small, x.cpu().numpy(), b) <= 1e-10


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_gcrodr_poly_mixed_wilson4(wilson4, prec):
    """GMRES(30) + degree-4 polynomial + k = 8 deflation, FP64 / FP32-IR / BF16-IR."""
    dev = to_cuda(wilson4)
    N = wilson4.volume * wilson4.n
    bs = rhs((1, 5), 3, N)
    p = _params(m=30, tol=1e-10, precision=prec, poly_degree=4, defl_k=8, recycle_updates=10,
                inner_tol=1e-5 if prec == 1 else 1e-2)
    its = []
    for i in range(3):
        x, info = dev.solve(torch.from_numpy(bs[i]).cuda(), params=p)
        x = x.cpu().numpy()
        assert info[0]["status"] == 0, info
        assert _resid(wilson4, x, bs[i]) <= 1e-10
        xs, _ = _lu(wilson4, bs[i])
        assert rel(x, xs) <= 1e-9
        its.append(info[0]["iterations"])
    assert its[-1] <= its[0]  # recycling across right-hand sides does not hurt


def test_twisted_mass_and_adjoint(wilson4):
    mu = 3e-3
    dev = to_cuda(wilson4, mu=mu)
    N = wilson4.volume * wilson4.n
    b = rhs((1, 9), 1, N)[0]
    p = _params(m=30, tol=1e-10, precision=1, poly_degree=4, defl_k=8)
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
    xs, _ = _lu(wilson4, b, mu)
    assert rel(x.cpu().numpy(), xs) <= 1e-9
    lam, info = dev.solve(torch.from_numpy(b).cuda(), params=p, adjoint=True)
    ls, _ = _lu(wilson4, b, mu, adjoint=True)
    assert rel(lam.cpu().numpy(), ls) <= 1e-9


def test_nonfinite_rhs_reported(small):
    from paper_2205_09104_gb300 import CoarseError
    dev = to_cuda(small)
    N = small.volume * small.n
    b = torch.from_numpy(rhs((600, 3), 1, N)[0]).cuda()
    b[7] = float("nan")
    with pytest.raises(CoarseError) as e:
        dev.solve(b, params=_params(m=10, precision=1))
    assert e.value.code == -6


def test_not_converged_keeps_best_iterate(wilson4):
    from paper_2205_09104_gb300 import PREC_FP64
    dev = to_cuda(wilson4, precisions=())
    N = wilson4.volume * wilson4.n
    b = rhs((1, 0), 1, N)[0]
    x, info = dev.solve(torch.from_numpy(b).cuda(), params=_params(m=4, max_restarts=2, max_ir=1, precision=PREC_FP64),
                        allow_not_converged=True)
    assert info[0]["status"] == -4
    assert info[0]["rel_residual"] < 1.0
    assert abs(_resid(wilson4, x.cpu().numpy(), b) - info[0]["rel_residual"]) <= 1e-6


def test_bf16_polynomial_chain(wilson4):
    """COARSE_POLY_BF16: the polynomial q (Sec. 3.3) evaluated with the BF16 blocks while the
    Krylov operator keeps FP32 blocks.  Same 1e-10 true residual and forward error; switching
    the flag on one handle rebuilds the recycle space for the new q, so every order converges."""
    from paper_2205_09104_gb300 import COARSE_POLY_BF16, COARSE_ZERO_GUESS
    dev = to_cuda(wilson4, precisions=(1, 2))
    N = wilson4.volume * wilson4.n
    b = rhs((1, 7), 3, N)
    its = {}
    for i, flag in enumerate((COARSE_POLY_BF16, 0, COARSE_POLY_BF16)):
        p = _params(m=30, tol=1e-10, precision=1, poly_degree=4, defl_k=8, recycle_updates=5, inner_tol=1e-5,
                    flags=COARSE_ZERO_GUESS | flag)
        x, info = dev.solve(torch.from_numpy(b[i]).cuda(), params=p)
        x = x.cpu().numpy()
        assert info[0]["status"] == 0, info[0]
        assert _resid(wilson4, x, b[i]) <= 1e-10
        xs, _ = _lu(wilson4, b[i])
        assert rel(x, xs) <= 1e-9
        its.setdefault(flag, []).append(info[0]["iterations"])
    # the BF16 chain changes the preconditioner by the block rounding only
    assert max(its[COARSE_POLY_BF16]) <= 1.3 * its[0][0] + 4, its
