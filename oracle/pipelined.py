"""Latency-1 pipelined GMRES and GCRO-DR (Sec. 3.5; oracle, test infrastructure only).

Imported by the tests only; the product path never calls it.

Pipelining (Sec. 3.5, after Ghysels et al.) decouples the matrix-vector product of an Arnoldi
step from its inner products: next to the orthonormal basis v_j the method carries
v^a_j = A v_j (shift sigma_j = 0, as the paper chooses), so that the product for step i,
w = A v^a_{i-1}, no longer waits for the orthogonalisation of step i-1 and the inner products
(v_j, v^a_{i-1}) with the squared norm ||v^a_{i-1}||^2 form one reduction.  The new
subdiagonal entry comes from that norm instead of a second reduction:
    h_{i,i-1}^2 = ||v^a_{i-1}||^2 - sum_j |h_{j,i-1}|^2  (- sum_j |b_{j,i-1}|^2 with recycling),
and a negative value is a breakdown (loss of orthogonality).  Both recurrences are updated with
the same coefficients:
    v_i   = (v^a_{i-1} - sum_j v_j h_{j,i-1}   - sum_j c_j b_{j,i-1})   / h_{i,i-1}
    v^a_i = (w         - sum_j v^a_j h_{j,i-1} - sum_j v^c_j b_{j,i-1}) / h_{i,i-1}
with v^c_j = A c_j for the recycle vectors c_j (Alg. "pipe1gcrodr"); without recycling the
c-terms vanish (Alg. "pipe1fgmres").  Mathematically the basis and the Hessenberg matrix are
those of the classical Arnoldi process on (I - C C^H) A.

A = D M is the right-preconditioned operator (M the polynomial preconditioner), as in
krylov.py; the block-Jacobi factor, when used, is part of the D the caller passes.

Readings taken where the algorithms are terse:
  * h^2 and b^2 in the formula for t are the squared moduli |h|^2, |b|^2 (the entries are
    complex; the defining relation is ||w||^2 = ||v^a||^2 - sum |h|^2).
  * The sums over the recycle vectors run over j = 0..k-1 (all k columns of C).
  * v^a_0 = A v_0, as the algorithm's second line computes it.
  * On t < 0 the cycle ends with the steps completed before it (their least-squares update is
    applied) and the next cycle restarts from the true residual; t = 0 is an invariant
    subspace: the step's column is kept with h_{i,i-1} = 0 and the cycle ends.  A |t| within
    the rounding error of the difference, 8 (i + k + 1) u ||v^a||^2 (u the unit roundoff, i + k + 1
    terms), counts as t = 0.
  * The first GCRO-DR cycle (no recycle space yet) is the classical GMRES cycle of the
    original algorithm, which the paper's pipelined listing takes over unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .krylov import Counter, Recycle, SolveInfo, _first_cycle_pk, _gcrodr_G, _gcrodr_pk, _ls, arnoldi


@dataclass
class P1Cycle:
    V: np.ndarray          # N x (j+1) orthonormal basis
    H: np.ndarray          # (j+1) x j Hessenberg
    B: np.ndarray          # k x j, C^H A V (empty without recycling)
    beta: float            # ||r|| of the start vector
    status: str            # "ok", "invariant" (t = 0) or "breakdown" (t < 0)


def p1_arnoldi(A, r: np.ndarray, steps: int, C: np.ndarray | None = None, VC: np.ndarray | None = None,
               stop=None) -> P1Cycle:
    """Latency-1 pipelined Arnoldi (the inner loop of both pipelined algorithms, sigma = 0).

    C (N x k, orthonormal) and VC = A C make it the process on (I - C C^H) A; ``stop(H, B,
    beta)`` may end it after a step (True ends).  Matrix-vector products: steps + 1.
    """
    k = 0 if C is None else C.shape[1]
    beta = float(np.linalg.norm(r))
    V = [r / beta]
    Va = [A(V[0])]                                   # v^a_0 = A v_0
    H = np.zeros((steps + 1, steps), dtype=complex)
    B = np.zeros((k, steps), dtype=complex)
    status = "ok"
    j = 0
    for i in range(1, steps + 1):
        va = Va[i - 1]
        w = A(va)                                    # the product of step i
        b = C.conj().T @ va if k else np.zeros(0, dtype=complex)
        h = np.array([np.vdot(V[jj], va) for jj in range(i)])
        nva = float(np.vdot(va, va).real)
        t = nva - float(np.sum(np.abs(h) ** 2)) - float(np.sum(np.abs(b) ** 2))
        # |t| within the rounding of the difference counts as t = 0
        t_round = 8.0 * (i + k + 1) * np.finfo(float).eps * nva
        if t < -t_round:
            status = "breakdown"     # the column of step i is unreliable: dropped
            break
        H[:i, i - 1] = h
        B[:, i - 1] = b
        if t <= t_round:
            status = "invariant"     # h_{i,i-1} = 0: the Krylov space is invariant
            V.append(np.zeros_like(va))
            j = i
            break
        hs = np.sqrt(t)
        H[i, i - 1] = hs
        vn = va - sum(V[jj] * h[jj] for jj in range(i))
        van = w - sum(Va[jj] * h[jj] for jj in range(i))
        if k:
            vn = vn - C @ b
            van = van - VC @ b
        V.append(vn / hs)
        Va.append(van / hs)
        j = i
        if stop is not None and stop(H[: i + 1, :i], B[:, :i], beta):
            break
    return P1Cycle(np.array(V).T, H[: j + 1, :j], B[:, :j], beta, status)


def p1_gmres(apply, b, m: int, tol: float, max_restarts: int = 10000, x0=None, precond=None):
    """Restarted latency-1 pipelined GMRES(m) (Alg. "pipe1fgmres"), right preconditioner M.

    Each cycle: the pipelined Arnoldi from r / ||r||, y = argmin ||H y - ||r|| e1||,
    x += M V y; the true residual is recomputed after every cycle, and a cycle ends early once
    its least-squares residual reaches tol.  Returns (x, SolveInfo, breakdowns).
    """
    D = Counter(apply)
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: D(M(v))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = float(np.linalg.norm(b))
    r = b - D(x) if x0 is not None else b.copy()
    info = SolveInfo()
    info.history.append(float(np.linalg.norm(r)) / bnorm)
    breakdowns = 0
    while info.history[-1] > tol and info.cycles < max_restarts:
        stop = lambda H, B, beta: _ls(H, beta * np.eye(H.shape[0], 1)[:, 0])[1] <= tol * bnorm
        cyc = p1_arnoldi(A, r, m, stop=stop)
        breakdowns += cyc.status == "breakdown"
        j = cyc.H.shape[1]
        info.iterations += j
        if j > 0:
            z, _ = _ls(cyc.H, cyc.beta * np.eye(j + 1, 1)[:, 0])
            x = x + M(cyc.V[:, :j] @ z)
        r = b - D(x)
        info.cycles += 1
        info.history.append(float(np.linalg.norm(r)) / bnorm)
        if j == 0 and cyc.status == "breakdown":
            break
    info.matvecs = D.count
    info.rel_residual = info.history[-1]
    info.converged = info.rel_residual <= tol
    return x, info, breakdowns


def p1_gcrodr(apply, b, m: int, k: int, tol: float, max_cycles: int = 10000, x0=None, precond=None,
              recycle: Recycle | None = None, u_limit: int = 10**9):
    """Latency-1 pipelined GCRO-DR(m, k) (Alg. "pipe1gcrodr"), right preconditioner M.

    As krylov.gcrodr, with the m - k Arnoldi steps of a recycling cycle taken by the pipelined
    process on (I - C C^H) A: per cycle v^c_j = A c_j (k products), then the pipelined inner loop
    records H and B = C^H A V; D_k, Vhat = [U D_k, V], What = [C, V_{m-k+1}] and G as in the
    classical algorithm; y = argmin ||What^H r - G y||, x += M Vhat y, r -= What G y; the recycle
    space is updated from G while fewer than u_limit updates were made.  The first cycle without
    a recycle space is the classical GMRES cycle.  Returns (x, SolveInfo, Recycle, breakdowns).
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
    breakdowns = 0
    while float(np.linalg.norm(r)) / bnorm > tol and info.cycles < max_cycles:
        if rec.U is not None:
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
            VC = np.array([A(C[:, jj]) for jj in range(kk)]).T      # v^c_j = A c_j
            rc = C.conj().T @ r

            def stop(H, B, beta):
                G = _gcrodr_G(dk, B, H)
                rhs = np.concatenate([rc, beta * np.eye(H.shape[0], 1)[:, 0]])
                return _ls(G, rhs)[1] <= tol * bnorm

            cyc = p1_arnoldi(A, r, m - kk, C, VC, stop)
            breakdowns += cyc.status == "breakdown"
            j = cyc.H.shape[1]
            info.iterations += j
            if j > 0:
                G = _gcrodr_G(dk, cyc.B, cyc.H)
                Vhat = np.concatenate([Ut, cyc.V[:, :j]], axis=1)
                What = np.concatenate([C, cyc.V], axis=1)
                y, _ = _ls(G, What.conj().T @ r)
                x = x + M(Vhat @ y)
                r = r - What @ (G @ y)
                if rec.updates < u_limit:
                    Pk = _gcrodr_pk(G, What.conj().T @ Vhat, kk)
                    Q, R = np.linalg.qr(G @ Pk)
                    rec.C = What @ Q
                    rec.U = Vhat @ Pk @ np.linalg.inv(R)
                    rec.updates += 1
            elif cyc.status == "breakdown":
                info.cycles += 1
                break
        info.cycles += 1
        r = b - D(x)
        info.history.append(float(np.linalg.norm(r)) / bnorm)
    info.matvecs = D.count
    info.rel_residual = float(np.linalg.norm(b - apply(x))) / bnorm
    info.converged = info.rel_residual <= tol
    return x, info, rec, breakdowns
