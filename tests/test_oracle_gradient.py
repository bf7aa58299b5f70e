"""Pins of the oracle's adjoint solve and block gradient against FD and the sigma3 identity."""
import numpy as np
import pytest

from oracle import coarse, gradient
from oracle.lattice import volume


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_adjoint_via_sigma3(small_setup, mu):
    """D_c^{-H} c = sigma3 D_c(-mu)^{-1} sigma3 c (Gamma5-hermiticity; Sec. 4.2)."""
    st = small_setup
    n = 2 * st["nv"]
    N = volume(st["cdims"]) * n
    rng = np.random.default_rng(3)
    c = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    lam = gradient.adjoint_solve(st["self"], st["hop"], st["cdims"], c, mu)
    s3 = np.tile(coarse.sigma3(st["nv"]), volume(st["cdims"]))
    via = s3 * gradient.solve(st["self"], st["hop"], st["cdims"], s3 * c, -mu)
    assert np.linalg.norm(lam - via) / np.linalg.norm(lam) < 1e-12


def test_block_gradient_matches_fd(small_setup):
    from synthetic import draws
    st = small_setup
    n = 2 * st["nv"]
    V = volume(st["cdims"])
    c, b, ent = draws.grad_draws((*st["key"], 5), V * n, V, n, 12)
    x = gradient.solve(st["self"], st["hop"], st["cdims"], b)
    lam = gradient.adjoint_solve(st["self"], st["hop"], st["cdims"], c)
    gs, gh = gradient.block_gradient(lam, x, st["cdims"], n)
    for e in ent:
        site, blk, i, j = e
        an = gs[site, i, j] if blk == 0 else gh[site, blk - 1, i, j]
        fd = gradient.finite_difference(st["self"], st["hop"], st["cdims"], b, c, e)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)
