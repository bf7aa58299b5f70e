"""Full-size checks on the twisted-mass workload: coarse 16^4 lattice (65536 sites), nv = 24
(n = 48, 3,145,728 unknowns), fine 32^4 with 2^4 aggregates, m0 = -0.42, mu = 3e-3.

At this size each CTA of the persistent kernels (the TMA-staged stencil, the streamed odd-even
layout) walks hundreds of sites, so their rings wrap many times.  The oracle cannot hold the
whole operator on the host, so it is evaluated site by site on sampled sites (blocks copied from
the device one site at a time), entry by entry; every launch configuration the autotuner may
choose is fixed in turn with coarse_autotune_set.  The solve runs exactly as the benchmark runs
it; its true residual is the library's FP64 residual, whose entries are checked against the
oracle's per-site residual on sampled sites.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import U64, assert_entrywise, make_op, rhs, sampled_apply_check, sampled_schur_check, site_blocks

pytestmark = pytest.mark.gpu

MU = 3e-3
KEY = (3, 0)


@pytest.fixture(scope="module")
def tm16():
    from paper_2205_09104_gb300 import CoarseOp
    op = make_op(KEY, (32, 32, 32, 32), 24, m0=-0.42, device="cuda")   # blocks stay on the device
    dev = CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=MU, precisions=(1, 2))
    yield op, dev
    dev.close()


def _sites(V, count, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, V - 1], rng.integers(0, V, count - 2)]))


def test_tm16_solve_in_benchmark_configuration(tm16):
    """Odd-even + block-Jacobi, degree-8 polynomial on BF16 blocks, GCRO-DR k = 32 (recycle space
    built by a full first cycle), FP32 inner solves to 2e-6, FP64 refinement to 1e-10."""
    from paper_2205_09104_gb300 import (COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_RECYCLE_FULL_CYCLE,
                                        COARSE_ZERO_GUESS, PREC_FP32, solve_params)
    from oracle import coarse as ocoarse
    op, dev = tm16
    N = op.volume * op.n
    kw = dict(m=50, tol=1e-10, precision=PREC_FP32, poly_degree=8, defl_k=32, recycle_updates=10, inner_tol=2e-6,
              max_restarts=100, max_ir=20)
    flags = COARSE_ZERO_GUESS | COARSE_POLY_BF16 | COARSE_ODD_EVEN
    bs = rhs((*KEY, 60), 3, N)
    _, info = dev.solve(torch.from_numpy(bs[0]).cuda(), params=solve_params(flags=flags | COARSE_RECYCLE_FULL_CYCLE, **kw))
    assert info[0]["status"] == 0 and info[0]["recycle_updates"] >= 1, info[0]
    chk = dev.recycle_check(PREC_FP32, odd_even=True)
    assert chk["k"] == 32 and chk["au_minus_c"] <= 2e-5 and chk["chc_minus_i"] <= 1e-5, chk
    sites = _sites(op.volume, 48, 11)
    blocks_of = site_blocks(op, sites)
    for b in bs[1:]:
        bd = torch.from_numpy(b).cuda()
        x, info = dev.solve(bd, params=solve_params(flags=flags, **kw))
        assert info[0]["status"] == 0, info[0]
        r, rn, bn = dev.residual(bd, x)
        assert rn / bn <= 1e-10, (rn / bn, info[0])
        assert abs(info[0]["rel_residual"] - rn / bn) <= 1e-6 * rn / bn + 1e-14
        # the residual's entries at sampled sites against the oracle's per-site b - D x
        xh = x.cpu().numpy()
        ref = b.reshape(op.volume, op.n)[sites] - ocoarse.apply_at(blocks_of, op.dims, xh, sites, MU)
        mag = np.abs(b.reshape(op.volume, op.n)[sites]) + ocoarse.apply_at(
            lambda s: tuple(np.abs(t) for t in blocks_of(s)), op.dims, np.abs(xh), sites).real \
            + MU * np.abs(xh.reshape(op.volume, op.n)[sites])
        got = r.cpu().numpy().reshape(op.volume, op.n)[sites]
        assert_entrywise(got, ref, (2 * (9 * op.n + 6)) * U64 * mag, "residual at sampled sites")


@pytest.mark.parametrize("variant", [0, 1])
def test_tm16_apply_sampled_sites_every_kernel(tm16, variant):
    """TMA-staged persistent stencil (0) and register push-pull stencil (1) for FP32 and BF16."""
    from paper_2205_09104_gb300 import autotune_set
    op, dev = tm16
    vb = op.volume.bit_length() - 1
    for p in (1, 2):
        autotune_set(f"apply/p{p}/n{op.n}/v{vb}", variant)
    try:
        x = rhs((*KEY, 61), 1, op.volume * op.n)[0]
        sampled_apply_check(dev, op, MU, x, _sites(op.volume, 96, 12 + variant), what=f"tm16 apply variant {variant}")
    finally:
        for p in (1, 2):
            autotune_set(f"apply/p{p}/n{op.n}/v{vb}", -1)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_tm16_schur_sampled_sites_every_layout(tm16, variant):
    """Every odd-even half-apply layout (6 = the streamed persistent one, whose CTAs walk about
    215 sites per half here) in FP64, FP32 and BF16."""
    from paper_2205_09104_gb300 import autotune_set
    from oracle import oddeven as ooe
    op, dev = tm16
    vb = op.volume.bit_length() - 1
    for p in (0, 1, 2):
        autotune_set(f"eo/p{p}/n{op.n}/v{vb}", variant)
    try:
        v = rhs((*KEY, 62), 1, op.volume * op.n // 2)[0]
        ev = ooe.sites(op.dims, 0)
        rng = np.random.default_rng(20 + variant)
        pick = np.unique(np.concatenate([[0, len(ev) - 1], rng.integers(0, len(ev), 30)]))
        sampled_schur_check(dev, op, MU, v, ev[pick], what=f"tm16 layout {variant}")
    finally:
        for p in (0, 1, 2):
            autotune_set(f"eo/p{p}/n{op.n}/v{vb}", -1)
