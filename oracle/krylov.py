"""Krylov solvers of the coarsest level (oracle; test infrastructure only).

Follows Sec. 3 of the paper:
    arnoldi          Alg. 1 (Arnoldi process) with modified Gram-Schmidt (Sec. 3.1)
    gmres            restarted GMRES(m): x_m = x_0 + V_m z, z = argmin ||beta e1 - Hbar_m z|| (Sec. 3.1)
    harmonic_ritz    eigenvalues of H_d + h_{d+1,d}^2 f e_d^T, f = H_d^{-H} e_d (Sec. 3.3)
    leja_order       Alg. 2 (Leja ordering of harmonic Ritz values)
    poly_apply       q_{d-1}(A) v = sum_i (1/theta_i) prod_{j<i} (I - A/theta_j) v (Sec. 3.3, eq. q)
    poly_setup       Alg. 3, steps 1-3 (Arnoldi from a random vector, harmonic Ritz, Leja)
    gcrodr           GCRO-DR with recycling (Sec. 3.4; steps reconstructed from the
                     high-level description there, see the function docstring)

Right preconditioning throughout: A = D M, x = x0 + M (...).
All arithmetic is complex128; small least-squares problems use numpy.linalg.lstsq
and eigenproblems numpy/scipy eig (library primitives as single steps).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


def _ls(H: np.ndarray, rhs: np.ndarray):
    z = np.linalg.lstsq(H, rhs, rcond=None)[0]
    return z, float(np.linalg.norm(rhs - H @ z))


def arnoldi(apply, v0: np.ndarray, steps: int, stop=None):
    """Arnoldi with MGS from v0 (normalised inside).

    ``stop(H_partial, beta)`` may end the process early (returns True).
    Returns (V (N x (j+1)), Hbar ((j+1) x j), beta).
    """
    beta = float(np.linalg.norm(v0))
    V = [v0 / beta]
    H = np.zeros((steps + 1, steps), dtype=complex)
    j = 0
    for j in range(steps):
        w = apply(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            V.append(np.zeros_like(w))
            return np.array(V).T, H[: j + 2, : j + 1], beta
        V.append(w / H[j + 1, j])
        if stop is not None and stop(H[: j + 2, : j + 1], beta):
            return np.array(V).T, H[: j + 2, : j + 1], beta
    return np.array(V).T, H, beta


@dataclass
class SolveInfo:
    converged: bool = False
    cycles: int = 0
    iterations: int = 0            # Arnoldi steps
    matvecs: int = 0               # applications of D
    history: list = field(default_factory=list)   # true relative residual after each cycle
    rel_residual: float = np.inf


class Counter:
    """Wraps a D_c apply to count matrix-vector products."""

    def __init__(self, apply):
        self._apply = apply
        self.count = 0

    def __call__(self, v):
        self.count += 1
        return self._apply(v)


def gmres(apply, b, m: int, tol: float, max_restarts: int = 10000, x0=None, precond=None):
    """Restarted GMRES(m) with optional right preconditioner ``precond`` (x = x0 + M V z).

    Convergence is judged on the true residual ||b - D x|| / ||b||, recomputed
    at every restart; inside a cycle the least-squares residual estimate ends
    the cycle early.
    """
    D = Counter(apply)
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: D(M(v))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = float(np.linalg.norm(b))
    r = b - D(x) if x0 is not None else b.copy()
    info = SolveInfo()
    info.history.append(float(np.linalg.norm(r)) / bnorm)
    while info.history[-1] > tol and info.cycles < max_restarts:
        stop = lambda H, beta: _ls(H, beta * np.eye(H.shape[0], 1)[:, 0])[1] <= tol * bnorm
        V, H, beta = arnoldi(A, r, m, stop)
        j = H.shape[1]
        info.iterations += j
        z, _ = _ls(H, beta * np.eye(j + 1, 1)[:, 0])
        x = x + M(V[:, :j] @ z)
        r = b - D(x)
        info.cycles += 1
        info.history.append(float(np.linalg.norm(r)) / bnorm)
    info.matvecs = D.count
    info.rel_residual = info.history[-1]
    info.converged = info.rel_residual <= tol
    return x, info


def harmonic_ritz(Hbar: np.ndarray) -> np.ndarray:
    """Harmonic Ritz values: eig(H_d + |h_{d+1,d}|^2 f e_d^T) with f = H_d^{-H} e_d.

    If h_{d+1,d} = 0 (the Krylov space is invariant) or H_d is singular, the
    Ritz values eig(H_d) are returned instead.
    """
    d = Hbar.shape[1]
    H = Hbar[:d, :d]
    h = Hbar[d, d - 1] if Hbar.shape[0] > d else 0.0
    if h == 0.0:
        return np.linalg.eigvals(H)
    e = np.zeros(d, dtype=complex)
    e[-1] = 1.0
    try:
        f = np.linalg.solve(H.conj().T, e)
    except np.linalg.LinAlgError:
        return np.linalg.eigvals(H)
    return np.linalg.eigvals(H + abs(h) ** 2 * np.outer(f, e))


def _better(a, b, ia, ib, sa, sb):
    """Leja tie-break: larger score, then larger real part, larger imaginary part, lower index."""
    if sa != sb:
        return sa > sb
    if a.real != b.real:
        return a.real > b.real
    if a.imag != b.imag:
        return a.imag > b.imag
    return ia < ib


def leja_order(theta: np.ndarray) -> np.ndarray:
    """Alg. 2: first the value of largest modulus, then repeatedly the value that
    maximises the product of distances to the values already chosen.

    Products are compared as sums of logarithms (a zero distance scores -inf).
    """
    theta = np.asarray(theta, dtype=complex)
    left = list(range(len(theta)))
    chosen = []

    def pick(score):
        best = left[0]
        for i in left[1:]:
            if _better(theta[i], theta[best], i, best, score(i), score(best)):
                best = i
        return best

    first = pick(lambda i: abs(theta[i]))
    chosen.append(first)
    left.remove(first)
    while left:
        def score(i):
            s = 0.0
            for j in chosen:
                dist = abs(theta[i] - theta[j])
                if dist == 0.0:
                    return -np.inf
                s += np.log(dist)
            return s
        nxt = pick(score)
        chosen.append(nxt)
        left.remove(nxt)
    return theta[chosen]


def poly_apply(apply, theta: np.ndarray, v: np.ndarray) -> np.ndarray:
    """q_{d-1}(A) v via the Newton-like form: d-1 applications of A."""
    s = v
    acc = s / theta[0]
    for i in range(1, len(theta)):
        s = s - apply(s) / theta[i - 1]
        acc = acc + s / theta[i]
    return acc


def residual_poly_apply(apply, theta: np.ndarray, v: np.ndarray) -> np.ndarray:
    """p_d(A) v = prod_i (I - A/theta_i) v (Sec. 3.3, eq. gmres_pol_loe)."""
    s = v
    for t in theta:
        s = s - apply(s) / t
    return s


def poly_setup(apply, v0: np.ndarray, d: int):
    """Alg. 3, steps 1-3: d Arnoldi steps from v0, harmonic Ritz values, Leja order."""
    V, H, beta = arnoldi(apply, v0, d)
    theta = harmonic_ritz(H)
    return leja_order(theta), H


@dataclass
class Recycle:
    """GCRO-DR recycle space: A U = C with C^H C = I (A = D M)."""
    U: np.ndarray | None = None
    C: np.ndarray | None = None
    updates: int = 0


def _first_cycle_pk(H: np.ndarray, k: int) -> np.ndarray:
    """k harmonic Ritz vectors of smallest |theta| from a plain Arnoldi cycle."""
    m = H.shape[1]
    Hm = H[:m, :m]
    e = np.zeros(m, dtype=complex)
    e[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, e)
    theta, Z = np.linalg.eig(Hm + abs(H[m, m - 1]) ** 2 * np.outer(f, e))
    idx = np.argsort(np.abs(theta), kind="stable")[:k]
    return Z[:, idx]


def _gcrodr_pk(G: np.ndarray, WhV: np.ndarray, k: int) -> np.ndarray:
    """k harmonic Ritz vectors of smallest |theta|: G^H G z = theta G^H (W^H V) z (QZ)."""
    theta, Z = sla.eig(G.conj().T @ G, G.conj().T @ WhV)
    mag = np.where(np.isfinite(theta), np.abs(theta), np.inf)
    idx = np.argsort(mag, kind="stable")[:k]
    return Z[:, idx]


def gcrodr(apply, b, m: int, k: int, tol: float, max_cycles: int = 10000, x0=None,
           precond=None, recycle: Recycle | None = None, u_limit: int = 10**9, diagnostics=None):
    """GCRO-DR(m, k) with right preconditioner and a recycle space kept across solves.

    Steps (Sec. 3.4; the full listing the paper points to is not reproduced there,
    so the cycle is reconstructed from its four-step description):
      0. r = b - D x; if U, C exist: x += M U (C^H r), r -= C (C^H r).
      1. Without U, C: one GMRES cycle of length m on A = D M; then the k harmonic
         Ritz vectors of smallest |theta| give P_k, [Q, R] = qr(Hbar P_k),
         C = V_{m+1} Q, U = V_m P_k R^{-1}.
      2. Otherwise m-k Arnoldi steps on (I - C C^H) A from r/||r||, recording
         B_k = C^H A V; with D_k = diag(1/||u_i||), Vhat = [U D_k, V],
         What = [C, V_{m-k+1}], G = [[D_k, B_k], [0, Hbar]] one has A Vhat = What G.
      3. y = argmin ||What^H r - G y||, x += M Vhat y, r -= What G y.
      4. While fewer than u_limit updates were made: G^H G z = theta G^H What^H Vhat z,
         k smallest |theta| -> P_k, [Q, R] = qr(G P_k), C = What Q, U = Vhat P_k R^{-1}.
    A cycle also ends early once its least-squares residual reaches tol.
    The true residual b - D x is recomputed after every cycle.
    """
    D = Counter(apply)
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: D(M(v))
    rec = recycle if recycle is not None else Recycle()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = float(np.linalg.norm(b))
    r = b - D(x) if x0 is not None else b.copy()
    info = SolveInfo()
    info.history.append(float(np.linalg.norm(r)) / bnorm)
    while float(np.linalg.norm(r)) / bnorm > tol and info.cycles < max_cycles:
        if rec.U is not None:
            # keep r orthogonal to range(C): x += M U (C^H r), r -= C (C^H r)
            c = rec.C.conj().T @ r
            x = x + M(rec.U @ c)
            r = r - rec.C @ c
        if rec.U is None:
            stop = lambda H, beta: _ls(H, beta * np.eye(H.shape[0], 1)[:, 0])[1] <= tol * bnorm
            V, H, beta = arnoldi(A, r, m, stop)
            j = H.shape[1]
            info.iterations += j
            z, _ = _ls(H, beta * np.eye(j + 1, 1)[:, 0])
            x = x + M(V[:, :j] @ z)
            r = r - V @ (H @ z)
            if k > 0 and j > k and rec.updates < u_limit and H[j, j - 1] != 0.0:
                Pk = _first_cycle_pk(H, k)
                Q, R = np.linalg.qr(H @ Pk)
                rec.C = V @ Q
                rec.U = V[:, :j] @ Pk @ np.linalg.inv(R)
                rec.updates += 1
        else:
            U, C = rec.U, rec.C
            kk = U.shape[1]
            dk = 1.0 / np.linalg.norm(U, axis=0)
            Ut = U * dk[None, :]
            beta = float(np.linalg.norm(r))
            Vs = [r / beta]
            steps = m - kk
            H = np.zeros((steps + 1, steps), dtype=complex)
            B = np.zeros((kk, steps), dtype=complex)
            j = 0
            for j in range(steps):
                w = A(Vs[j])
                B[:, j] = C.conj().T @ w
                w = w - C @ B[:, j]
                for i in range(j + 1):
                    H[i, j] = np.vdot(Vs[i], w)
                    w = w - H[i, j] * Vs[i]
                H[j + 1, j] = np.linalg.norm(w)
                Vs.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else np.zeros_like(w))
                G = _gcrodr_G(dk, B[:, : j + 1], H[: j + 2, : j + 1])
                rhs = np.concatenate([C.conj().T @ r, beta * np.eye(j + 2, 1)[:, 0]])
                _, est = _ls(G, rhs)
                if est <= tol * bnorm or H[j + 1, j] == 0.0:
                    break
            j = j + 1
            info.iterations += j
            Vm = np.array(Vs[: j + 1]).T
            G = _gcrodr_G(dk, B[:, :j], H[: j + 1, :j])
            Vhat = np.concatenate([Ut, Vm[:, :j]], axis=1)
            What = np.concatenate([C, Vm], axis=1)
            rhs = What.conj().T @ r
            y, _ = _ls(G, rhs)
            x = x + M(Vhat @ y)
            r = r - What @ (G @ y)
            if diagnostics is not None:
                diagnostics.append({"Vhat": Vhat, "What": What, "G": G, "A": A})
            if rec.updates < u_limit:
                Pk = _gcrodr_pk(G, What.conj().T @ Vhat, kk)
                Q, R = np.linalg.qr(G @ Pk)
                rec.C = What @ Q
                rec.U = Vhat @ Pk @ np.linalg.inv(R)
                rec.updates += 1
        info.cycles += 1
        r = b - D(x)
        info.history.append(float(np.linalg.norm(r)) / bnorm)
    info.matvecs = D.count
    info.rel_residual = float(np.linalg.norm(b - apply(x))) / bnorm
    info.converged = info.rel_residual <= tol
    return x, info, rec


def _gcrodr_G(dk, B, H):
    kk = dk.shape[0]
    j = H.shape[1]
    G = np.zeros((kk + j + 1, kk + j), dtype=complex)
    G[:kk, :kk] = np.diag(dk)
    G[:kk, kk:] = B
    G[kk:, kk:] = H
    return G
