"""Pins of the oracle's Krylov methods (Sec. 3) against exact identities, brute force and dense LU."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import coarse, krylov

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _op(st, mu=0.0):
    return lambda v: coarse.apply(st["self"], st["hop"], st["cdims"], v, mu)


def _rhs(st, idx=0):
    from synthetic import draws
    N = st["self"].shape[0] * st["self"].shape[1]
    return draws.rhs((*st["key"], 77), 1, N, idx)[0]


def _lu_solution(st, b, mu=0.0):
    A = coarse.assemble(st["self"], st["hop"], st["cdims"], mu).tocsc()
    return spla.spsolve(A, b), A


def test_gmres_matches_dense_lu(ragged_setup):
    st = ragged_setup
    b = _rhs(st)
    xs, A = _lu_solution(st, b)
    x, info = krylov.gmres(_op(st), b, m=12, tol=1e-11)
    assert info.converged
    r = b - A @ x
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-11
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-11
    assert info.cycles > 1   # restarts were exercised


@pytest.mark.parametrize("d", [1, 2, 4, 8])
def test_residual_polynomial_equals_gmres_residual(ragged_setup, d):
    """r_d = p_d(A) r0 with p_d(t) = prod(1 - t/theta_i), theta the harmonic Ritz values."""
    st = ragged_setup
    A = _op(st)
    r0 = _rhs(st, 3)
    V, H, beta = krylov.arnoldi(A, r0, d)
    theta = krylov.harmonic_ritz(H)
    # independent d-step GMRES residual: minimise ||r0 - A K c|| over the monomial Krylov basis
    K = [r0]
    for _ in range(d - 1):
        K.append(A(K[-1]))
    AK = np.array([A(k) for k in K]).T
    c = np.linalg.lstsq(AK, r0, rcond=None)[0]
    rd = r0 - AK @ c
    got = krylov.residual_poly_apply(A, theta, r0)
    assert np.linalg.norm(got - rd) / np.linalg.norm(r0) < 1e-10
    # and q interpolates 1/theta at its nodes: x_d = q(A) r0 gives r_d = r0 - A q(A) r0
    q = krylov.poly_apply(A, krylov.leja_order(theta), r0)
    assert np.linalg.norm(r0 - A(q) - rd) / np.linalg.norm(r0) < 1e-9


def test_q_interpolates_inverse_and_degree_one():
    theta = np.array([2.0 + 1j, -0.5 + 0.2j, 1.5 - 0.7j, 0.3 + 0.9j])
    for t in theta:
        val = krylov.poly_apply(lambda v: t * v, theta, np.array([1.0 + 0j]))[0]
        assert abs(val - 1 / t) < 1e-13
    one = krylov.poly_apply(lambda v: 5 * v, theta[:1], np.array([1.0 + 0j]))[0]
    assert abs(one - 1 / theta[0]) < 1e-15


def test_q_independent_of_ordering(ragged_setup):
    st = ragged_setup
    A = _op(st)
    theta = np.array([2.0 + 0.5j, 1.0 - 0.3j, 3.5 + 0.1j])
    v = _rhs(st, 5)
    a = krylov.poly_apply(A, theta, v)
    b = krylov.poly_apply(A, theta[[2, 0, 1]], v)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_lucky_breakdown_gives_exact_roots():
    """h_{d+1,d} = 0: theta are eigenvalues of A and p_d(A) r0 = 0."""
    rng = np.random.default_rng(4)
    lam = np.array([1.0 + 0.5j, 2.0 - 1j, 0.5 + 0.1j, 3.0 + 0j, 4.0 + 2j, 1.5 - 0.2j])
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    M = Q @ np.diag(lam) @ Q.conj().T
    r0 = Q[:, :3] @ np.array([1.0, 2.0 - 1j, 0.5j])
    V, H, beta = krylov.arnoldi(lambda v: M @ v, r0, 3)
    assert abs(H[3, 2]) < 1e-12
    theta = krylov.harmonic_ritz(H)
    assert np.abs(np.sort_complex(theta) - np.sort_complex(lam[:3])).max() < 1e-10
    assert np.linalg.norm(krylov.residual_poly_apply(lambda v: M @ v, theta, r0)) < 1e-10


def _read_golden(name):
    sections = {}
    cur = None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("input", "ordered"):
            cur = sections.setdefault(line, [])
            continue
        re, im = map(float, line.split())
        cur.append(re + 1j * im)
    return {k: np.array(v) for k, v in sections.items()}


def test_leja_golden_example():
    g = _read_golden("leja_example.txt")
    assert np.array_equal(krylov.leja_order(g["input"]), g["ordered"])


def test_leja_is_permutation_with_greedy_property():
    rng = np.random.default_rng(6)
    theta = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    out = krylov.leja_order(theta)
    assert np.array_equal(np.sort_complex(out), np.sort_complex(theta))
    assert abs(out[0]) >= np.abs(theta).max() * (1 - 1e-15)
    for k in range(1, len(out)):
        prod = lambda t: np.prod(np.abs(t - out[:k]))
        assert all(prod(out[k]) >= prod(t) - 1e-12 for t in out[k:])


def test_pp_gmres_solves(ragged_setup):
    st = ragged_setup
    A = _op(st)
    b = _rhs(st, 1)
    xs, Am = _lu_solution(st, b)
    rng_start = np.random.default_rng(8)
    v0 = rng_start.standard_normal(b.size) + 1j * rng_start.standard_normal(b.size)
    theta, _ = krylov.poly_setup(A, v0, 4)
    x, info = krylov.gmres(A, b, m=8, tol=1e-11, precond=lambda v: krylov.poly_apply(A, theta, v))
    x0, info0 = krylov.gmres(A, b, m=8, tol=1e-11)
    assert info.converged and info0.converged
    assert info.iterations < info0.iterations              # fewer Arnoldi steps (Sec. 3.3)
    assert np.linalg.norm(b - Am @ x) / np.linalg.norm(b) <= 1e-11


def test_gcrodr_k0_equals_gmres(ragged_setup):
    st = ragged_setup
    b = _rhs(st, 2)
    x1, i1 = krylov.gmres(_op(st), b, m=10, tol=1e-10)
    x2, i2, rec = krylov.gcrodr(_op(st), b, m=10, k=0, tol=1e-10)
    assert rec.U is None
    assert i1.cycles == i2.cycles and i1.iterations == i2.iterations
    assert np.abs(np.array(i1.history) - np.array(i2.history)).max() < 1e-12
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-11


def test_gcrodr_first_cycle_is_gmres(ragged_setup):
    st = ragged_setup
    b = _rhs(st, 2)
    _, i1 = krylov.gmres(_op(st), b, m=10, tol=1e-10, max_restarts=1)
    _, i2, _ = krylov.gcrodr(_op(st), b, m=10, k=4, tol=1e-10, max_cycles=1)
    assert abs(i1.history[1] - i2.history[1]) < 1e-13


def test_gcrodr_invariants_and_solution(ragged_setup):
    st = ragged_setup
    A = _op(st)
    b = _rhs(st, 4)
    xs, Am = _lu_solution(st, b)
    diag = []
    x, info, rec = krylov.gcrodr(A, b, m=10, k=4, tol=1e-11, diagnostics=diag)
    assert info.converged
    assert np.linalg.norm(b - Am @ x) / np.linalg.norm(b) <= 1e-11
    kappa = np.linalg.cond(Am.toarray())
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-11
    # C^H C = I and A U = C
    assert np.abs(rec.C.conj().T @ rec.C - np.eye(4)).max() < 1e-12
    AU = np.array([A(u) for u in rec.U.T]).T
    assert np.linalg.norm(AU - rec.C) / np.linalg.norm(rec.C) < 1e-10
    # Arnoldi relation A Vhat = What G of every recycled cycle (eq. gcrodr_Arn_relation)
    assert diag
    for dgn in diag:
        AV = np.array([dgn["A"](v) for v in dgn["Vhat"].T]).T
        assert np.linalg.norm(AV - dgn["What"] @ dgn["G"]) / np.linalg.norm(AV) < 1e-10
    # minimal residual over a growing augmented space: residuals never increase
    h = np.array(info.history)
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))


def test_gcrodr_recycling_across_rhs_and_poly(ragged_setup):
    """Second right-hand side reuses U, C; combined with the polynomial preconditioner."""
    st = ragged_setup
    A = _op(st)
    rng = np.random.default_rng(9)
    v0 = rng.standard_normal(st["self"].shape[0] * st["self"].shape[1]) * (1 + 0j)
    theta, _ = krylov.poly_setup(A, v0, 4)
    M = lambda v: krylov.poly_apply(A, theta, v)
    b1, b2 = _rhs(st, 10), _rhs(st, 11)
    x1, i1, rec = krylov.gcrodr(A, b1, m=8, k=3, tol=1e-11, precond=M, u_limit=10)
    x2, i2, rec = krylov.gcrodr(A, b2, m=8, k=3, tol=1e-11, precond=M, recycle=rec, u_limit=10)
    xs, Am = _lu_solution(st, b2)
    assert i1.converged and i2.converged
    assert np.linalg.norm(b2 - Am @ x2) / np.linalg.norm(b2) <= 1e-11
    assert rec.updates <= 10
