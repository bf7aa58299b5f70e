"""Pins of the odd-even reduced, block-Jacobi preconditioned oracle (Sec. 2, Sec. 3.2).

Each pin reaches the same quantity by an independent route: dense Schur-complement algebra
on the assembled sparse matrix, the reconstruction of a known full solution of D x = b, and
the Schur determinant identity det D = det D_oo det D_ee det S."""
import numpy as np
import pytest

from oracle import coarse as oc
from oracle import oddeven as oe
from oracle.lattice import neighbours

from synthetic import draws


class _Op:
    """The oracle-built coarse operator of a conftest setup (coarse 2^4, n = 8)."""

    def __init__(self, setup):
        self.s, self.h, self.dims = setup["self"], setup["hop"], setup["cdims"]
        self.n = self.s.shape[1]
        self.volume = self.s.shape[0]


@pytest.fixture(scope="module")
def op(small_setup):
    return _Op(small_setup)


def _dense_parts(op, mu):
    A = oc.assemble(op.s, op.h, op.dims, mu).toarray()
    par = np.repeat(oe.parity(op.dims), op.n)
    ev, od = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    return A, A[np.ix_(ev, ev)], A[np.ix_(ev, od)], A[np.ix_(od, ev)], A[np.ix_(od, od)], ev, od


def _dense_S(op, mu):
    A, Aee, Aeo, Aoe, Aoo, ev, od = _dense_parts(op, mu)
    S = Aee - Aeo @ np.linalg.solve(Aoo, Aoe)
    return np.linalg.solve(Aee, S), A, Aee, Aoo, ev, od


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 4), (4, 4, 4, 4)])
def test_hops_join_opposite_parities(dims):
    par = oe.parity(dims)
    nb = neighbours(dims)
    for d in range(8):
        assert np.all(par[nb[:, d]] != par)
    assert (par == 0).sum() == (par == 1).sum()


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        oe.parity((3, 2, 2, 2))


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_schur_matches_dense_complement(op, mu):
    Sd, *_ = _dense_S(op, mu)
    N2 = Sd.shape[0]
    gen = draws.rng((700, 0), 0)
    v = draws.complex_gaussian(gen, (N2,))
    s = oe.schur_apply(op.s, op.h, op.dims, v, mu)
    assert np.linalg.norm(s - Sd @ v) <= 1e-12 * np.linalg.norm(Sd @ v)


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_reduced_system_reproduces_full_solution(op, mu):
    s_b, h_b = op.s, op.h
    Sd, *_ = _dense_S(op, mu)
    gen = draws.rng((701, 0), 0)
    x_true = draws.complex_gaussian(gen, (op.volume * op.n,))
    b = oc.apply(s_b, h_b, op.dims, x_true, mu)
    x_e = np.linalg.solve(Sd, oe.reduced_rhs(s_b, h_b, op.dims, b, mu))
    x = oe.retrieve(s_b, h_b, op.dims, x_e, b, mu)
    assert np.linalg.norm(x - x_true) <= 1e-10 * np.linalg.norm(x_true)


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_schur_determinant_identity(op, mu):
    Sd, A, Aee, Aoo, ev, od = _dense_S(op, mu)
    sD, lD = np.linalg.slogdet(A)
    parts = [np.linalg.slogdet(M) for M in (Aoo, Aee, Sd)]
    sP = np.prod([p[0] for p in parts])
    lP = sum(p[1] for p in parts)
    assert abs(lD - lP) <= 1e-9 * abs(lD)
    assert abs(sD - sP) <= 1e-8


def test_block_inverses(op):
    inv = oe.inverses(op.s, 0.05)
    blk = oe.diag_blocks(op.s, 0.05)
    eye = np.eye(op.n)
    assert max(np.linalg.norm(blk[x] @ inv[x] - eye) for x in range(op.volume)) <= 1e-12


def test_schur_at_equals_whole_lattice_schur():
    """The per-site evaluation of S (for sampled sites of large lattices) equals the factored
    whole-lattice S, which the dense Schur algebra pins."""
    from synthetic.coarse_op import build_coarse_operator
    from synthetic import draws
    op = build_coarse_operator((905, 0), (8, 4, 4, 8), 4, -0.4, 1.0)
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    N2 = s.shape[0] * s.shape[1] // 2
    v = draws.rhs((905, 1), 1, N2)[0]
    ev = oe.sites(op.dims, 0)
    for mu in (0.0, 0.05):
        full = oe.schur_apply(s, h, op.dims, v, mu).reshape(len(ev), -1)
        at = oe.schur_at(lambda x: (s[x], h[x]), op.dims, v, ev, mu)
        assert np.abs(at - full).max() <= 1e-12 * np.abs(full).max()
