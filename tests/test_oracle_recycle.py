"""Pins of the oracle's GCRO-DR recycle-vector selection (Sec. 3.4).

GCRO-DR deflates the k harmonic Ritz vectors whose harmonic Ritz values are
smallest in modulus.  The invariants of the recycle space (A U = C, C^H C = I,
the augmented Arnoldi relation) hold for ANY choice of k columns, so they do
not check this choice.  These tests do:

  * on a normal matrix with known, well-separated eigenvalues and a start
    vector inside an invariant subspace, the harmonic Ritz vectors are exact
    eigenvectors, so range(U) must be the span of the eigenvectors of the k
    smallest |lambda| in that subspace (principal angles <= 1e-10);
  * on the coarse operator, every kept pair (theta, z) must satisfy the
    harmonic Petrov-Galerkin condition (A Vhat z - theta Vhat z) _|_ A Vhat,
    and the kept theta must be the k smallest in modulus among all harmonic
    Ritz values, computed independently from A Vhat itself
    (theta = 1 / eig(Q_W^H Vhat R_W^{-1}) with A Vhat = Q_W R_W).

A selection that keeps the largest |theta| instead, or plain Ritz vectors of
H_m (both planted below, on the CPU), fails these checks.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import coarse, krylov


def _normal_matrix(seed, lam):
    rng = np.random.default_rng(seed)
    n = len(lam)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return Q @ np.diag(lam) @ Q.conj().T, Q


# eigenvalues with well-separated moduli 0.3 .. 5.5, complex phases
LAM = np.array([0.3 * np.exp(0.4j), 0.6 * np.exp(-1.1j), 1.0 * np.exp(2.0j), 1.6 * np.exp(0.9j),
                2.3 * np.exp(-2.5j), 3.1 * np.exp(0.2j), 4.0 * np.exp(-0.7j), 5.5 * np.exp(1.7j),
                0.45 * np.exp(3.0j), 2.7 * np.exp(-1.9j)])
# the invariant subspace the start vector lies in, and the k smallest |lambda| inside it
SUB = [0, 2, 3, 5, 7, 8]
K = 3


def _smallest_in(sub, k):
    return sorted(sub, key=lambda i: abs(LAM[i]))[:k]


def _largest_pk_first(H, k):
    """Planted mistake: the first-cycle selection keeping the LARGEST |theta|."""
    m = H.shape[1]
    Hm = H[:m, :m]
    e = np.zeros(m, dtype=complex)
    e[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, e)
    theta, Z = np.linalg.eig(Hm + abs(H[m, m - 1]) ** 2 * np.outer(f, e))
    return Z[:, np.argsort(-np.abs(theta), kind="stable")[:k]]


def _largest_pk_gcrodr(G, WhV, k):
    """Planted mistake: the GCRO-DR update keeping the LARGEST finite |theta|."""
    theta, Z = sla.eig(G.conj().T @ G, G.conj().T @ WhV)
    mag = np.where(np.isfinite(theta), np.abs(theta), -np.inf)
    return Z[:, np.argsort(-mag, kind="stable")[:k]]


def _ritz_pk_first(H, k):
    """Planted mistake: plain Ritz vectors (eig(H_m)) instead of harmonic Ritz vectors."""
    m = H.shape[1]
    theta, Z = np.linalg.eig(H[:m, :m])
    return Z[:, np.argsort(np.abs(theta), kind="stable")[:k]]


def _max_angle_sin(A, B):
    """sin of the largest principal angle between range(A) and range(B) (equal dimensions)."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(Qa.conj().T @ Qb, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))


def _first_cycle_space_error(select):
    """range(V_m P_k) against the eigenvectors of the k smallest |lambda| of the invariant subspace."""
    M, Q = _normal_matrix(11, LAM)
    rng = np.random.default_rng(12)
    r0 = Q[:, SUB] @ (rng.standard_normal(len(SUB)) + 1j * rng.standard_normal(len(SUB)))
    V, H, _ = krylov.arnoldi(lambda v: M @ v, r0, len(SUB))
    assert abs(H[-1, -1]) < 1e-12 * np.abs(H).max()   # the Krylov space is invariant after |SUB| steps
    P = select(H, K)
    m = H.shape[1]
    U = V[:, :m] @ P
    return _max_angle_sin(U, Q[:, _smallest_in(SUB, K)])


def _gcrodr_space_error(select):
    """GCRO-DR update on an invariant augmented space given in a non-orthonormal basis."""
    M, Q = _normal_matrix(13, LAM)
    rng = np.random.default_rng(14)
    p = len(SUB)
    # Vhat: a skewed, non-orthonormal basis of the invariant subspace (as [U D_k, V] is in a cycle)
    T = rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p)) + 3 * np.eye(p)
    Vhat = Q[:, SUB] @ T
    AV = M @ Vhat
    # What: orthonormal basis of range(A Vhat) plus one unit vector orthogonal to it (its row of G is 0)
    Wq, _ = np.linalg.qr(AV)
    extra = Q[:, [i for i in range(len(LAM)) if i not in SUB][0]]
    What = np.concatenate([Wq, extra[:, None]], axis=1)
    G = What.conj().T @ AV
    assert np.linalg.norm(What @ G - AV) < 1e-12 * np.linalg.norm(AV)
    P = select(G, What.conj().T @ Vhat, K)
    return _max_angle_sin(Vhat @ P, Q[:, _smallest_in(SUB, K)])


def test_first_cycle_keeps_smallest_harmonic_ritz_vectors():
    assert _first_cycle_space_error(krylov._first_cycle_pk) < 1e-10


def test_gcrodr_update_keeps_smallest_harmonic_ritz_vectors():
    assert _gcrodr_space_error(krylov._gcrodr_pk) < 1e-10


def test_flipped_selection_fails_the_invariant_space_pins():
    assert _first_cycle_space_error(_largest_pk_first) > 0.5
    assert _gcrodr_space_error(_largest_pk_gcrodr) > 0.5


def _pg_check(A, Vhat, Z, k):
    """For the kept columns Z of the harmonic Ritz problem on range(Vhat):
    returns (max PG defect, max |theta_kept - theta_expected| / |theta_expected|), where the
    expected values are the k smallest |theta| of an independent computation from A Vhat."""
    W = np.array([A(v) for v in Vhat.T]).T
    Qw, Rw = np.linalg.qr(W)
    nu = np.linalg.eigvals(Qw.conj().T @ Vhat @ np.linalg.inv(Rw))
    nu = nu[np.abs(nu) > 1e-14 * np.abs(nu).max()]
    theta_all = 1.0 / nu
    expected = theta_all[np.argsort(np.abs(theta_all))][:k]
    kept, defect = [], 0.0
    for c in range(Z.shape[1]):
        y = Vhat @ Z[:, c]
        Ay = W @ Z[:, c]
        th = np.vdot(Ay, Ay) / np.vdot(Ay, y)            # from (A y)^H (A y - theta y) = 0
        res = W.conj().T @ (Ay - th * y)                  # (A y - theta y) _|_ range(A Vhat)
        defect = max(defect, np.linalg.norm(res) / (np.linalg.norm(W) * np.linalg.norm(Ay)))
        kept.append(th)
    kept = np.array(kept)
    # match each expected value to the nearest kept one
    mism = max(np.abs(kept - t).min() / abs(t) for t in expected)
    return defect, mism


def _coarse_A(st):
    return lambda v: coarse.apply(st["self"], st["hop"], st["cdims"], v)


def _rhs(st, idx):
    from synthetic import draws
    N = st["self"].shape[0] * st["self"].shape[1]
    return draws.rhs((*st["key"], 78), 1, N, idx)[0]


@pytest.mark.parametrize("select,pg_ok,smallest_ok", [(krylov._first_cycle_pk, True, True),
                                                       (_largest_pk_first, True, False),
                                                       (_ritz_pk_first, False, False)])
def test_first_cycle_harmonic_petrov_galerkin(ragged_setup, select, pg_ok, smallest_ok):
    st = ragged_setup
    A = _coarse_A(st)
    b = _rhs(st, 0)
    m, k = 12, 4
    V, H, _ = krylov.arnoldi(A, b, m)
    Z = select(H, k)
    defect, mism = _pg_check(A, V[:, :m], Z, k)
    assert (defect < 1e-10) == pg_ok         # eigenpairs of the harmonic problem satisfy PG, Ritz pairs do not
    assert (mism < 1e-8) == smallest_ok      # only the smallest-|theta| harmonic choice matches


def test_gcrodr_update_harmonic_petrov_galerkin(ragged_setup):
    st = ragged_setup
    A = _coarse_A(st)
    diag = []
    krylov.gcrodr(A, _rhs(st, 1), m=10, k=4, tol=1e-11, diagnostics=diag)
    assert diag
    for dgn in diag[:3]:
        Vhat, What, G = dgn["Vhat"], dgn["What"], dgn["G"]
        WhV = What.conj().T @ Vhat
        for select, ok in ((krylov._gcrodr_pk, True), (_largest_pk_gcrodr, False)):
            Z = select(G, WhV, 4)
            defect, mism = _pg_check(dgn["A"], Vhat, Z, 4)
            assert defect < 1e-9
            assert (mism < 1e-7) == ok
