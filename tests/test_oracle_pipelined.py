"""Pins of the latency-1 pipelined GMRES / GCRO-DR oracle (Sec. 3.5, Alg. "pipe1fgmres" and
"pipe1gcrodr") against what mathematics fixes: the pipelined process builds the same basis and
Hessenberg matrix as the classical Arnoldi process (modified Gram-Schmidt, an independent
algorithm) on A, or on (I - C C^H) A with a recycle space; its solves reach the dense solution;
an invariant Krylov space (t = 0) ends a cycle with the exact solution; a loss of orthogonality
(t < 0) is reported as a breakdown and the restarted solver still converges; pipelined and
classical GCRO-DR agree cycle by cycle.

The comparisons use short cycles (4-5 steps): with sigma = 0 the pipelined recurrences amplify
rounding by about ||h|| / h_{i+1,i} per step (the instability the paper mentions), so a long
cycle drifts away from the classical one by far more than rounding.
"""
import numpy as np
import pytest

from oracle import krylov as kr
from oracle import pipelined as pl


def _matrix(seed, N=48, rad=0.5):
    """Complex non-Hermitian test matrix, eigenvalues in a disc of radius ~rad around 1."""
    rng = np.random.default_rng(seed)
    A0 = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(2 * N) * rad + np.eye(N)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return A0, r


def test_pipelined_arnoldi_equals_classical():
    A0, r = _matrix(1)
    cyc = pl.p1_arnoldi(lambda v: A0 @ v, r, 4)
    V, H, beta = kr.arnoldi(lambda v: A0 @ v, r, 4)
    assert cyc.status == "ok"
    assert np.abs(H.imag).max() > 0.05            # complex entries: |h|^2, not h^2, decides t
    assert np.abs(cyc.H - H).max() <= 1e-12 * np.abs(H).max()
    assert np.abs(cyc.V - V).max() <= 1e-12
    assert abs(cyc.beta - beta) <= 1e-14 * beta
    # Arnoldi relation and orthonormality, independently of the classical process
    assert np.abs(A0 @ cyc.V[:, :4] - cyc.V @ cyc.H).max() <= 1e-12
    assert np.abs(cyc.V.conj().T @ cyc.V - np.eye(5)).max() <= 1e-12


def test_pipelined_arnoldi_uses_steps_plus_one_products():
    A0, r = _matrix(2)
    D = kr.Counter(lambda v: A0 @ v)
    pl.p1_arnoldi(D, r, 5)
    assert D.count == 6


def test_pipelined_arnoldi_with_recycle_space_equals_projected_arnoldi():
    A0, r = _matrix(3)
    rng = np.random.default_rng(33)
    C, _ = np.linalg.qr(rng.standard_normal((A0.shape[0], 3)) + 1j * rng.standard_normal((A0.shape[0], 3)))
    r = r - C @ (C.conj().T @ r)        # a GCRO-DR cycle starts from a residual orthogonal to C
    A = lambda v: A0 @ v
    VC = A0 @ C
    cyc = pl.p1_arnoldi(A, r, 4, C, VC)
    # classical Arnoldi on (I - C C^H) A from the same start vector
    P = lambda v: A0 @ v - C @ (C.conj().T @ (A0 @ v))
    V, H, _ = kr.arnoldi(P, r, 4)
    assert cyc.status == "ok"
    assert np.abs(cyc.H - H).max() <= 1e-11 * np.abs(H).max()
    assert np.abs(cyc.V - V).max() <= 1e-11
    assert np.abs(cyc.B - C.conj().T @ A0 @ cyc.V[:, :4]).max() <= 1e-12 * np.abs(cyc.B).max()
    # the GCRO-DR relation A V_j = C B + V_{j+1} H
    assert np.abs(A0 @ cyc.V[:, :4] - C @ cyc.B - cyc.V @ cyc.H).max() <= 1e-11


def test_pipelined_gmres_reaches_dense_solution():
    A0, b = _matrix(4)
    x, info, _ = pl.p1_gmres(lambda v: A0 @ v, b, 6, 1e-10)
    assert info.converged
    assert np.linalg.norm(b - A0 @ x) / np.linalg.norm(b) <= 1e-10
    xs = np.linalg.solve(A0, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-9


def test_pipelined_gmres_cycle_equals_classical_cycle():
    A0, b = _matrix(5)
    M0 = np.eye(A0.shape[0]) + 0.1 * np.diag(np.linspace(0, 1, A0.shape[0]))   # a right preconditioner
    x1, i1, _ = pl.p1_gmres(lambda v: A0 @ v, b, 4, 1e-14, max_restarts=1, precond=lambda v: M0 @ v)
    x2, i2 = kr.gmres(lambda v: A0 @ v, b, 4, 1e-14, max_restarts=1, precond=lambda v: M0 @ v)
    assert i1.iterations == i2.iterations == 4
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) <= 1e-11
    assert abs(i1.history[-1] - i2.history[-1]) <= 1e-9 * i2.history[-1]


def test_invariant_subspace_gives_exact_solution():
    # A = lambda I: A v_0 is parallel to v_0, t = 0 at the first step
    _, b = _matrix(6)
    lam = 2.0 - 1.0j
    x, info, bd = pl.p1_gmres(lambda v: lam * v, b, 8, 1e-13)
    assert info.converged and info.cycles == 1 and bd == 0
    assert np.abs(x - b / lam).max() <= 1e-14 * np.abs(b / lam).max()
    # b in a two-dimensional invariant subspace: exact after two steps
    N = 20
    A0 = np.diag(np.arange(1.0, N + 1.0)).astype(complex)
    A0[:2, :2] = [[1.0 + 1.0j, 0.5], [-0.25, 2.0 - 0.5j]]
    b = np.zeros(N, dtype=complex)
    b[:2] = [1.0, 1.0j]
    cyc = pl.p1_arnoldi(lambda v: A0 @ v, b, 6)
    assert cyc.status == "invariant" and cyc.H.shape == (3, 2) and cyc.H[2, 1] == 0.0
    x, info, _ = pl.p1_gmres(lambda v: A0 @ v, b, 6, 1e-13)
    assert info.cycles == 1 and np.linalg.norm(A0 @ x - b) <= 1e-13 * np.linalg.norm(b)


def test_negative_t_is_reported_as_breakdown():
    # planted: a "recycle space" with a repeated column is not orthonormal, so the subtracted
    # squares exceed ||v^a||^2 and t < 0 at the first step
    A0, r = _matrix(7)
    c = A0 @ (r / np.linalg.norm(r))
    c = c / np.linalg.norm(c)
    C = np.stack([c, c], axis=1)
    cyc = pl.p1_arnoldi(lambda v: A0 @ v, r, 4, C, A0 @ C)
    assert cyc.status == "breakdown" and cyc.H.shape == (1, 0)


def test_restarted_solver_recovers_from_a_breakdown():
    # loss of orthogonality in a long cycle (clustered spectrum, sigma = 0) ends the cycle; the
    # steps before it are applied and the next cycle restarts from the true residual
    A0, b = _matrix(7, N=50, rad=0.2)
    x, info, bd = pl.p1_gmres(lambda v: A0 @ v, b, 30, 1e-10)
    assert bd >= 1
    assert info.converged and np.linalg.norm(b - A0 @ x) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("k", [2, 3])
def test_pipelined_gcrodr_matches_gcrodr(k):
    A0, b1 = _matrix(8, N=64, rad=0.9)
    rng = np.random.default_rng(88)
    b2 = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    A = lambda v: A0 @ v
    rec_p, rec_c = kr.Recycle(), kr.Recycle()
    for b in (b1, b2):
        xp, ip, rec_p, bd = pl.p1_gcrodr(A, b, 7, k, 1e-10, recycle=rec_p)
        xc, ic, rec_c = kr.gcrodr(A, b, 7, k, 1e-10, recycle=rec_c)
        assert bd == 0
        assert ip.converged and ic.converged
        assert ip.cycles == ic.cycles and ip.iterations == ic.iterations
        h_p, h_c = np.array(ip.history), np.array(ic.history)
        assert np.all(np.abs(h_p - h_c) <= 1e-6 * h_c + 1e-14)
        xs = np.linalg.solve(A0, b)
        assert np.linalg.norm(xp - xs) / np.linalg.norm(xs) <= 1e-9
