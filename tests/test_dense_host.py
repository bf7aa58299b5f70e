"""Host build of the library's small dense FP64 routines, checked against LAPACK and the oracle.

The same source (csrc/dense.cuh) runs on the GPU as a warp team; here it is
compiled for the host with a single-lane team.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import krylov

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("dense") / "libdense_host.so"
    cuda_inc = os.environ.get("CUDA_HOME", "/usr/local/cuda") + "/include"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", cuda_inc,
                           os.path.join(HERE, "dense_host_harness.cpp"), "-o", str(out)])
    L = ctypes.CDLL(str(out))
    dp = ctypes.POINTER(ctypes.c_double)
    L.host_eig.argtypes = [ctypes.c_int, dp, dp, dp]
    L.host_hessenberg.argtypes = [ctypes.c_int, dp, dp, dp]
    L.host_leja.argtypes = [ctypes.c_int, dp]
    L.host_givens.argtypes = [dp, dp, dp]
    L.host_harmonic_nu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_givens(lib):
    rng = np.random.default_rng(0)
    for x, y in [(1 + 2j, 3 - 1j), (0j, 2 + 1j), (1 - 1j, 0j), (1e-200 + 0j, 1e-200j)]:
        out = np.zeros(5)
        lib.host_givens(_p(np.array([x.real, x.imag])), _p(np.array([y.real, y.imag])), _p(out))
        c, s, r = out[0], out[1] + 1j * out[2], out[3] + 1j * out[4]
        G = np.array([[c, s], [-np.conj(s), c]])
        v = G @ np.array([x, y])
        assert abs(v[1]) <= 1e-15 * max(abs(x), abs(y), 1e-300) * 4
        assert abs(v[0] - r) <= 1e-15 * abs(r) * 4
        assert np.allclose(G.conj().T @ G, np.eye(2), atol=1e-15)


@pytest.mark.parametrize("m", [1, 2, 5, 17, 40, 64])
def test_hessenberg_similarity(lib, m):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    H = np.zeros((m, m), complex)
    Z = np.zeros((m, m), complex)
    lib.host_hessenberg(m, _p(A.copy()), _p(H), _p(Z))
    assert np.abs(np.tril(H, -2)).max(initial=0) == 0
    assert np.abs(Z.conj().T @ Z - np.eye(m)).max() < 1e-13
    assert np.abs(Z @ H @ Z.conj().T - A).max() < 1e-12 * np.abs(A).max() * m


@pytest.mark.parametrize("m", [1, 2, 3, 8, 33, 50, 64])
def test_eig_matches_lapack(lib, m):
    rng = np.random.default_rng(100 + m)
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    lam = np.zeros(m, complex)
    X = np.zeros((m, m), complex)
    assert lib.host_eig(m, _p(A.copy()), _p(lam), _p(X)) == 0
    ref = np.linalg.eigvals(A)
    # match eigenvalues one to one
    for l in lam:
        assert np.abs(ref - l).min() < 1e-10 * max(1, abs(l))
    assert np.abs(np.sort_complex(np.round(lam, 8)) - np.sort_complex(np.round(ref, 8))).max() < 1e-7
    # eigenvector residuals
    for q in range(m):
        x = X[:, q]
        assert np.linalg.norm(A @ x - lam[q] * x) <= 1e-10 * np.linalg.norm(x) * np.abs(A).max() * m


def test_eig_hessenberg_input_and_repeated_values(lib):
    # already-triangular and diagonal inputs, repeated eigenvalues
    m = 6
    A = np.diag([1 + 1j, 1 + 1j, 2.0, 2.0, -3j, 0.5]).astype(complex)
    A[0, 3] = 0.3
    lam = np.zeros(m, complex)
    X = np.zeros((m, m), complex)
    assert lib.host_eig(m, _p(A.copy()), _p(lam), _p(X)) == 0
    assert np.abs(np.sort_complex(lam) - np.sort_complex(np.diag(A))).max() < 1e-14


def test_harmonic_ritz_via_eig(lib):
    """1/eig(Hbar^+ [I;0]) equals the oracle's harmonic Ritz values (H + |h|^2 f e^T)."""
    rng = np.random.default_rng(7)
    d = 8
    H = np.triu(rng.standard_normal((d + 1, d)) + 1j * rng.standard_normal((d + 1, d)), -1)
    H[np.arange(1, d + 1), np.arange(d)] = np.abs(H[np.arange(1, d + 1), np.arange(d)])
    M = np.linalg.pinv(H) @ np.vstack([np.eye(d), np.zeros((1, d))])
    lam = np.zeros(d, complex)
    X = np.zeros((d, d), complex)
    assert lib.host_eig(d, _p(M.astype(complex).copy()), _p(lam), _p(X)) == 0
    ref = krylov.harmonic_ritz(H)
    got = 1.0 / lam
    for g in got:
        assert np.abs(ref - g).min() < 1e-9 * abs(g)


def test_leja_matches_oracle_and_golden(lib):
    rng = np.random.default_rng(11)
    for d in (1, 2, 4, 8, 20):
        th = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        buf = np.ascontiguousarray(th.copy())
        lib.host_leja(d, _p(buf.view(np.float64)))
        assert np.array_equal(buf, krylov.leja_order(th))
    th = np.array([1, -2, 3j, 0.5, 2 + 2j], dtype=complex)
    lib.host_leja(5, _p(th.view(np.float64)))
    assert np.array_equal(th, np.array([3j, -2, 2 + 2j, 1, 0.5]))


@pytest.mark.parametrize("k,j,ld_b", [(4, 8, 32), (3, 10, 32), (32, 18, 32), (1, 5, 7)])
def test_harmonic_matrix_of_augmented_cycle(lib, k, j, ld_b):
    """Eigenvalues of the solver's harmonic Ritz matrix of a GCRO-DR cycle (Sec. 3.4) are 1/theta
    for the generalized problem G^H G z = theta G^H S z (SciPy QZ), with B stored at the solver's
    leading dimension (ld_b != k checks that the matrix is read with it)."""
    import scipy.linalg as sla
    rng = np.random.default_rng(100 * k + j)
    cplx = lambda *sh: rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    Hb = np.triu(cplx(j + 1, j), -1)
    Hb[np.arange(1, j + 1), np.arange(j)] = np.abs(Hb[np.arange(1, j + 1), np.arange(j)]) + 0.5
    B = cplx(k, j)
    Stop = np.eye(k) + 0.3 * cplx(k, k)
    Sbot = 0.3 * cplx(j + 1, k)
    G = np.zeros((k + j + 1, k + j), complex)
    G[:k, :k] = np.eye(k)
    G[:k, k:] = B
    G[k:, k:] = Hb
    S = np.zeros((k + j + 1, k + j), complex)
    S[:k, :k] = Stop
    S[k:, :k] = Sbot
    S[k:, k:] = np.eye(j + 1, j)
    nu = np.zeros(2 * (k + j))
    rc = lib.host_harmonic_nu(k, j, ld_b, _p(np.ascontiguousarray(Hb)), _p(np.ascontiguousarray(B)),
                              _p(np.ascontiguousarray(Stop)), _p(np.ascontiguousarray(Sbot)), _p(nu))
    assert rc == 0
    theta = 1.0 / (nu[0::2] + 1j * nu[1::2])
    ref = sla.eig(G.conj().T @ G, G.conj().T @ S, right=False)
    ref = ref[np.isfinite(ref)]
    for t in ref:
        assert np.abs(theta - t).min() <= 1e-9 * max(1.0, abs(t)), (t, theta)
