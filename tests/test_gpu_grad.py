"""GPU parity of the differentiable solve: CoarseSolve (autograd.Function) with its
hand-written backward (adjoint solve through sigma3 D_c(-mu) sigma3, block gradients
-lambda_x x_y^H), against the FP64 oracle's gradient and central finite differences.

Bar: relative error 1e-6 (FP32 inner solves inside FP64 refinement to 1e-12).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import make_op, rel
from oracle import coarse as ocoarse
from oracle import gradient as ograd
from oracle import krylov
from synthetic import draws

pytestmark = pytest.mark.gpu


def _autograd(op, b, c, mu=0.0, tol=1e-12):
    from paper_2205_09104_gb300 import CoarseOp, CoarseSolve, solve_params
    S = op.self_blocks.cuda().requires_grad_()
    H = op.hop_blocks.cuda().requires_grad_()
    dev = CoarseOp(S.detach(), H.detach(), op.dims, op.nv, mu=mu, precisions=(1,))
    p = solve_params(m=30, tol=tol, precision=1, poly_degree=4, defl_k=8, inner_tol=1e-5)
    bt = torch.from_numpy(b).cuda().requires_grad_()
    ct = torch.from_numpy(c).cuda()
    x = CoarseSolve.apply(bt, S, H, dev, p)
    L = (ct.conj() * x).sum().real
    L.backward()
    out = (x.detach().cpu().numpy(), bt.grad.cpu().numpy(), S.grad.cpu().numpy(), H.grad.cpu().numpy(), float(L.detach()))
    dev.close()
    return out


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_gradient_small_vs_oracle_and_fd(mu):
    op = make_op((700, 0), (6, 4, 4, 6), 16, m0=-0.4)     # 36 sites, n = 32
    n, V = op.n, op.volume
    N = n * V
    c, b, ent = draws.grad_draws((700, 1), N, V, n, 64)
    x, gb, gs, gh, L = _autograd(op, b, c, mu)
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    xs = ograd.solve(s, h, op.dims, b, mu)
    lam = ograd.adjoint_solve(s, h, op.dims, c, mu)
    rs, rh = ograd.block_gradient(lam, xs, op.dims, n)
    assert rel(x, xs) <= 1e-9
    assert rel(gb, lam) <= 1e-6
    assert rel(gs, rs) <= 1e-6
    assert rel(gh, rh) <= 1e-6
    for e in ent:
        site, blk, i, j = e
        an = gs[site, i, j] if blk == 0 else gh[site, blk - 1, i, j]
        fd = ograd.finite_difference(s, h, op.dims, b, c, e, h=1e-6, mu=mu)
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-2 * np.abs(rs).max())


def test_gradient_differentiation_workload_sampled():
    """Coarse 8^4, nv = 16, m0 = -0.42 (131072 unknowns): 64 sampled block entries and dL/db
    against the oracle's gradient from its own FP64 GCRO-DR solves."""
    op = make_op((5, 0), (16, 16, 16, 16), 16, m0=-0.42, device="cuda")
    op.self_blocks, op.hop_blocks = op.self_blocks.cpu(), op.hop_blocks.cpu()
    n, V = op.n, op.volume
    N = n * V
    c, b, ent = draws.grad_draws((5, 1), N, V, n, 64)
    x, gb, gs, gh, L = _autograd(op, b, c)
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    A = lambda v: ocoarse.apply(s, h, op.dims, v)
    Ah = lambda v: ocoarse.apply_adjoint(s, h, op.dims, v)
    theta, _ = krylov.poly_setup(A, draws.poly_start((5, 2), N), 4)
    xs, _, _ = krylov.gcrodr(A, b, m=50, k=16, tol=1e-12, precond=lambda v: krylov.poly_apply(A, theta, v))
    theta_h, _ = krylov.poly_setup(Ah, draws.poly_start((5, 3), N), 4)
    lam, _, _ = krylov.gcrodr(Ah, c, m=50, k=16, tol=1e-12, precond=lambda v: krylov.poly_apply(Ah, theta_h, v))
    assert rel(x, xs) <= 1e-9
    assert rel(gb, lam) <= 1e-6
    from oracle.lattice import neighbours
    nb = neighbours(op.dims)
    Lm, Xm = lam.reshape(V, n), xs.reshape(V, n)
    scale = np.abs(Lm).max() * np.abs(Xm).max()
    for site, blk, i, j in ent:
        src = site if blk == 0 else nb[site, blk - 1]
        ref = -Lm[site, i] * np.conj(Xm[src, j])
        got = gs[site, i, j] if blk == 0 else gh[site, blk - 1, i, j]
        assert abs(got - ref) <= 1e-6 * max(abs(ref), 1e-3 * scale)


def test_gradient_with_odd_even_forward():
    """The forward solve on the odd-even reduced system with the BF16 chain; the backward's
    adjoint solve falls back to the full operator: gradients as the oracle's."""
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_ZERO_GUESS, CoarseOp, CoarseSolve,
                                        solve_params)
    op = make_op((701, 0), (8, 4, 4, 8), 16, m0=-0.4)     # coarse 4x2x2x4 (even extents), n = 32
    n, V = op.n, op.volume
    c, b, _ = draws.grad_draws((701, 1), n * V, V, n, 4)
    S = op.self_blocks.cuda().requires_grad_()
    H = op.hop_blocks.cuda().requires_grad_()
    dev = CoarseOp(S.detach(), H.detach(), op.dims, op.nv, precisions=(1, 2))
    p = solve_params(m=30, tol=1e-12, precision=1, poly_degree=4, defl_k=8, inner_tol=2e-6, max_ir=30,
                     flags=COARSE_ZERO_GUESS | COARSE_ODD_EVEN | COARSE_POLY_BF16)
    bt = torch.from_numpy(b).cuda().requires_grad_()
    x = CoarseSolve.apply(bt, S, H, dev, p)
    (torch.from_numpy(c).cuda().conj() * x).sum().real.backward()
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    xs = ograd.solve(s, h, op.dims, b)
    lam = ograd.adjoint_solve(s, h, op.dims, c)
    rs, rh = ograd.block_gradient(lam, xs, op.dims, n)
    assert rel(x.detach().cpu().numpy(), xs) <= 1e-9
    assert rel(bt.grad.cpu().numpy(), lam) <= 1e-6
    assert rel(S.grad.cpu().numpy(), rs) <= 1e-6
    assert rel(H.grad.cpu().numpy(), rh) <= 1e-6
    dev.close()


@pytest.mark.parametrize("hop_dirs", [8, 4])
def test_block_grad_kernel_entrywise(hop_dirs):
    """coarse_block_grad on given lambda and x, every entry against the oracle's -lambda_x x_y^H
    (hop_dirs = 4: plus the backward-hop gradient of x + mu folded onto F_{x,mu} as
    sigma3 G^H sigma3) within 8 u of the products' magnitudes."""
    from gpu_helpers import U64, assert_entrywise, to_cuda
    from oracle.lattice import neighbours
    op = make_op((702, 0), (6, 4, 4, 6), 16, m0=-0.4)
    n, V = op.n, op.volume
    dev = to_cuda(op, precisions=())
    g = np.random.default_rng(5)
    lam = g.standard_normal(V * n) + 1j * g.standard_normal(V * n)
    x = g.standard_normal(V * n) + 1j * g.standard_normal(V * n)
    gs, gh = dev.block_grad(torch.from_numpy(lam).cuda(), torch.from_numpy(x).cuda(), hop_dirs=hop_dirs)
    gs, gh = gs.cpu().numpy(), gh.cpu().numpy()
    rs, rh = ograd.block_gradient(lam, x, op.dims, n)
    nb = neighbours(op.dims)
    L, X = np.abs(lam.reshape(V, n)), np.abs(x.reshape(V, n))
    ms = L[:, :, None] * X[:, None, :]
    mh = L[:, None, :, None] * X[nb][:, :, None, :]
    assert_entrywise(gs, rs, 8 * U64 * ms, "g_self")
    if hop_dirs == 8:
        assert_entrywise(gh, rh, 8 * U64 * mh, "g_hop")
        return
    s3 = ocoarse.sigma3(n // 2)
    want = rh[:, :4].copy()
    mag = mh[:, :4].copy()
    for mu in range(4):
        back = rh[nb[:, mu], 4 + mu]          # gradient of D[x + mu, x] = sigma3 F_{x,mu}^H sigma3
        want[:, mu] += s3[None, :, None] * np.conj(np.transpose(back, (0, 2, 1))) * s3[None, None, :]
        mag[:, mu] += np.transpose(mh[nb[:, mu], 4 + mu], (0, 2, 1))
    assert_entrywise(gh, want, 8 * U64 * mag, "g_hop folded")


def test_gradient_gamma5_compressed_input_vs_fd():
    """CoarseSolve on a gamma5-compressed operator (hop blocks [V, 4, n, n], backward hops
    derived): the gradient with respect to the forward blocks against central finite
    differences of the oracle's loss with the backward hops rebuilt from the perturbed block."""
    from paper_2205_09104_gb300 import CoarseOp, CoarseSolve, solve_params
    from oracle.lattice import neighbours
    op = make_op((703, 0), (6, 4, 4, 6), 8, m0=-0.4)
    n, V = op.n, op.volume
    N = n * V
    c, b, ent = draws.grad_draws((703, 1), N, V, n, 16)
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    S = op.self_blocks.cuda().requires_grad_()
    H4 = op.hop_blocks[:, :4].contiguous().cuda().requires_grad_()
    dev = CoarseOp(S.detach(), H4.detach(), op.dims, op.nv, precisions=(1,), assume_gamma5=True)
    p = solve_params(m=30, tol=1e-12, precision=1, poly_degree=4, defl_k=8, inner_tol=1e-5)
    bt = torch.from_numpy(b).cuda().requires_grad_()
    x = CoarseSolve.apply(bt, S, H4, dev, p)
    (torch.from_numpy(c).cuda().conj() * x).sum().real.backward()
    assert H4.grad.shape == H4.shape
    gh = H4.grad.cpu().numpy()
    nb = neighbours(op.dims)
    s3 = ocoarse.sigma3(n // 2)

    def loss_with(site, mu, i, j, delta):
        hp = h.copy()
        hp[site, mu, i, j] += delta
        y = nb[site, mu]
        hp[y, 4 + mu] = s3[:, None] * np.conj(hp[site, mu].T) * s3[None, :]
        return ograd.loss(s, hp, op.dims, b, c)

    scale = np.abs(gh).max()
    for k, (site, blk, i, j) in enumerate(ent):
        mu = int(blk) % 4
        eps = 1e-6
        fd = ((loss_with(site, mu, i, j, eps) - loss_with(site, mu, i, j, -eps))
              + 1j * (loss_with(site, mu, i, j, 1j * eps) - loss_with(site, mu, i, j, -1j * eps))) / (2 * eps)
        assert abs(gh[site, mu, i, j] - fd) <= 1e-6 * max(abs(fd), 1e-2 * scale), (k, gh[site, mu, i, j], fd)
    dev.close()
