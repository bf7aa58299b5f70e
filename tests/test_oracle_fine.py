"""Pins of the oracle's fine-level operator (Sec. 2.1) against closed forms and identities."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fine
from oracle.lattice import gamma5, gammas, neighbours, volume
from synthetic.gauge import su3_links


def test_clifford_and_gamma5():
    g = gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.array_equal(anti, 2.0 * (mu == nu) * np.eye(4))
    g5 = gamma5()
    assert np.array_equal(g5, np.diag([1, 1, -1, -1]).astype(complex))
    for mu in range(4):
        assert np.array_equal(g5 @ g[mu] + g[mu] @ g5, np.zeros((4, 4)))


def test_links_are_su3():
    U = su3_links((7, 0), (2, 2, 2, 2)).numpy()
    UhU = np.einsum("mxba,mxbc->mxac", U.conj(), U)
    assert np.abs(UhU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


def _free_field_closed_form(dims, m0):
    """lambda = m0 + sum(1 - cos p) +- i sqrt(sum sin^2 p), each sign with multiplicity 6."""
    vals = []
    for n0 in range(dims[0]):
        for n1 in range(dims[1]):
            for n2 in range(dims[2]):
                for n3 in range(dims[3]):
                    p = 2 * np.pi * np.array([n0, n1, n2, n3]) / np.array(dims)
                    re = m0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    vals += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(vals)


def _same_multiset(a, b, tol):
    a = np.sort_complex(np.round(a, 9))
    b = np.sort_complex(np.round(b, 9))
    return np.abs(a - b).max() < tol


@pytest.mark.parametrize("dims", [(3, 4, 2, 3), (4, 4, 3, 2)])
def test_free_field_spectrum(dims):
    V = volume(dims)
    U = np.tile(np.eye(3, dtype=complex), (4, V, 1, 1))
    m0 = -0.37
    D = fine.wilson_clover(U, dims, m0, csw=1.0).toarray()
    ev = np.linalg.eigvals(D)
    assert _same_multiset(ev, _free_field_closed_form(dims, m0), 1e-8)


def test_gamma5_hermiticity_and_clover():
    dims = (4, 2, 4, 2)
    U = su3_links((11, 0), dims).numpy()
    D = fine.wilson_clover(U, dims, -0.4, 1.0)
    G5 = fine.Gamma5(dims)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    y = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    # <y, G5 D G5 x> == <D y, x>  (Gamma5 D Gamma5 = D^H)
    lhs = np.vdot(y, G5 @ (D @ (G5 @ x)))
    rhs = np.vdot(D @ y, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    cl = fine.clover_term(U, dims, -0.4, 1.0)
    assert np.abs(cl - np.conj(np.swapaxes(cl, -1, -2))).max() < 1e-13
    g5 = np.kron(gamma5(), np.eye(3))
    assert np.abs(cl @ g5 - g5 @ cl).max() < 1e-13
    # clover term is not trivial for a random field
    assert np.abs(cl - (3.6) * np.eye(12)).max() > 1e-2


def test_clover_constant_abelian_field():
    """Constant U(1) flux B in the (0,1) plane: clover eigenvalues (m0+4) +- (c_sw/2) sin B."""
    dims = (4, 3, 2, 2)
    V = volume(dims)
    B = 2 * np.pi / (dims[0] * dims[1])
    c = np.stack(np.meshgrid(*[np.arange(L) for L in dims], indexing="ij"), -1)
    c = np.transpose(c, (3, 2, 1, 0, 4)).reshape(V, 4)   # site-major, x0 fastest
    U = np.tile(np.eye(3, dtype=complex), (4, V, 1, 1))
    ph1 = np.exp(1j * B * c[:, 0])                        # U_1(x) = exp(i B x0)
    ph0 = np.where(c[:, 0] == dims[0] - 1, np.exp(-1j * B * dims[0] * c[:, 1]), 1.0)
    U[1] *= ph1[:, None, None]
    U[0] *= ph0[:, None, None]
    m0, csw = -0.2, 1.3
    cl = fine.clover_term(U, dims, m0, csw)
    expect = np.array([m0 + 4 + 0.5 * csw * np.sin(B)] * 6 + [m0 + 4 - 0.5 * csw * np.sin(B)] * 6)
    for x in range(V):
        ev = np.sort(np.linalg.eigvalsh(cl[x]))
        assert np.abs(ev - np.sort(expect)).max() < 1e-13


def test_gauge_covariance():
    """D[U^Omega] = Omega D[U] Omega^H with U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^H."""
    dims = (2, 4, 2, 4)
    V = volume(dims)
    U = su3_links((12, 0), dims).numpy()
    Om = su3_links((13, 0), dims).numpy()[0]
    nb = neighbours(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = Om @ U[mu] @ np.conj(np.swapaxes(Om[nb[:, mu]], -1, -2))
    D = fine.wilson_clover(U, dims, -0.3, 1.0).toarray()
    Dg = fine.wilson_clover(Ug, dims, -0.3, 1.0).toarray()
    import scipy.sparse as sp
    Omega = sp.block_diag([np.kron(np.eye(4), Om[x]) for x in range(V)]).toarray()
    assert np.abs(Dg - Omega @ D @ Omega.conj().T).max() < 1e-13


def test_twisted_mass_singular_values():
    """sigma(D + i mu Gamma5) = sqrt(lambda(Gamma5 D)^2 + mu^2) (Sec. 4.2)."""
    dims = (2, 2, 2, 4)
    U = su3_links((14, 0), dims).numpy()
    mu = 0.05
    D = fine.wilson_clover(U, dims, -0.5, 1.0).toarray()
    Dtm = fine.wilson_clover(U, dims, -0.5, 1.0, mu_tm=mu).toarray()
    G5 = fine.Gamma5(dims).toarray()
    lam = np.linalg.eigvalsh(G5 @ D)
    sv = np.linalg.svd(Dtm, compute_uv=False)
    assert np.abs(np.sort(sv) - np.sort(np.sqrt(lam ** 2 + mu ** 2))).max() < 1e-12
