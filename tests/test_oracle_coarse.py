"""Pins of the oracle's aggregation / Galerkin construction and coarse stencil (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import coarse, fine, multigrid
from oracle.lattice import gamma5, volume


def test_test_vectors_reduce_residual(small_setup):
    from synthetic import draws
    D = small_setup["D"]
    starts = draws.test_vector_starts(small_setup["key"], 256, small_setup["nv"])
    for s, t in zip(starts, small_setup["tv"]):
        assert np.linalg.norm(D @ t) < np.linalg.norm(D @ s.reshape(-1))


def test_prolongator_orthonormal_and_chiral(small_setup):
    P = small_setup["P"]
    nv = small_setup["nv"]
    PhP = (P.conj().T @ P).toarray()
    assert np.abs(PhP - np.eye(P.shape[1])).max() < 1e-14
    G5 = fine.Gamma5(small_setup["dims"])
    s3 = np.tile(coarse.sigma3(nv), P.shape[1] // (2 * nv))
    assert np.abs((P.conj().T @ G5 @ P).toarray() - np.diag(s3)).max() < 1e-14


@pytest.mark.parametrize("which", ["small_setup", "ragged_setup"])
def test_galerkin_identity(which, request):
    st = request.getfixturevalue(which)
    D, P = st["D"], st["P"]
    rng = np.random.default_rng(1)
    v = rng.standard_normal(P.shape[1]) + 1j * rng.standard_normal(P.shape[1])
    ref = P.conj().T @ (D @ (P @ v))
    got = coarse.apply(st["self"], st["hop"], st["cdims"], v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("which", ["small_setup", "ragged_setup"])
def test_coarse_gamma5_relation(which, request):
    st = request.getfixturevalue(which)
    assert coarse.gamma5_defect(st["self"], st["hop"], st["cdims"]) < 1e-13


def test_coarse_apply_matches_assembly_and_adjoint(ragged_setup):
    st = ragged_setup
    A = coarse.assemble(st["self"], st["hop"], st["cdims"], mu=0.01)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    y = coarse.apply(st["self"], st["hop"], st["cdims"], v, mu=0.01)
    assert np.linalg.norm(y - A @ v) / np.linalg.norm(y) < 1e-14
    yh = coarse.apply_adjoint(st["self"], st["hop"], st["cdims"], v, mu=0.01)
    assert np.linalg.norm(yh - A.conj().T @ v) / np.linalg.norm(yh) < 1e-14
    # sigma3 D_c(mu) sigma3 = D_c(-mu)^H  (Gamma5-hermiticity on the coarse level)
    s3 = sp.diags(np.tile(coarse.sigma3(st["nv"]), volume(st["cdims"])))
    Am = coarse.assemble(st["self"], st["hop"], st["cdims"], mu=-0.01)
    assert abs(s3 @ A @ s3 - Am.conj().T).max() < 1e-13


def test_twisted_mass_galerkin(small_setup):
    """P^H (D + i mu Gamma5) P = D_c + i mu sigma3."""
    st = small_setup
    mu = 3e-3
    Dtm = fine.wilson_clover(st["U"], st["dims"], st["m0"], st["csw"], mu_tm=mu)
    P = st["P"]
    ref = (P.conj().T @ Dtm @ P).toarray()
    got = coarse.assemble(st["self"], st["hop"], st["cdims"], mu=mu).toarray()
    assert np.abs(got - ref).max() < 1e-13


def test_coarse_twisted_mass_singular_values(small_setup):
    st = small_setup
    mu = 1e-2
    A = coarse.assemble(st["self"], st["hop"], st["cdims"]).toarray()
    Atm = coarse.assemble(st["self"], st["hop"], st["cdims"], mu=mu).toarray()
    s3 = np.diag(np.tile(coarse.sigma3(st["nv"]), volume(st["cdims"])))
    lam = np.linalg.eigvalsh(s3 @ A)
    sv = np.linalg.svd(Atm, compute_uv=False)
    assert np.abs(np.sort(sv) - np.sort(np.sqrt(lam ** 2 + mu ** 2))).max() < 1e-12


def test_coarse_free_field_closed_form():
    """U = I, test vectors = the constant spin-colour basis of each chirality half:
    D_c = 1/2 D_W(2 m0) on the coarse lattice, so
    lambda_c = 1/2 [2 m0 + sum(1 - cos p) +- i sqrt(sum sin^2 p)] (multiplicity 6 each)."""
    fdims = (4, 6, 4, 4)
    cd = multigrid.coarse_dims(fdims)
    Vf = volume(fdims)
    U = np.tile(np.eye(3, dtype=complex), (4, Vf, 1, 1))
    m0 = -0.3
    nv = 6
    tv = np.zeros((nv, Vf, 4, 3), dtype=complex)
    for k in range(nv):
        tv[k, :, k // 3, k % 3] = 1.0          # chirality + half
        tv[k, :, 2 + k // 3, k % 3] = 1.0      # chirality - half
    P = multigrid.prolongator(tv.reshape(nv, -1), fdims)
    s, h = multigrid.galerkin_blocks(U, fdims, P, m0, 1.0, nv)
    ev = np.linalg.eigvals(coarse.assemble(s, h, cd).toarray())
    ref = []
    for n0 in range(cd[0]):
        for n1 in range(cd[1]):
            for n2 in range(cd[2]):
                for n3 in range(cd[3]):
                    p = 2 * np.pi * np.array([n0, n1, n2, n3]) / np.array(cd)
                    re = 0.5 * (2 * m0 + np.sum(1 - np.cos(p)))
                    im = 0.5 * np.sqrt(np.sum(np.sin(p) ** 2))
                    ref += [re + 1j * im] * 6 + [re - 1j * im] * 6
    a = np.sort_complex(np.round(ev, 9))
    b = np.sort_complex(np.round(np.array(ref), 9))
    assert np.abs(a - b).max() < 1e-8


@pytest.mark.parametrize("which", ["small_setup", "ragged_setup"])
def test_generator_matches_oracle(which, request):
    """The vectorised workload generator reproduces the oracle's Galerkin blocks."""
    from synthetic.coarse_op import build_coarse_operator
    st = request.getfixturevalue(which)
    op = build_coarse_operator(st["key"], st["dims"], st["nv"], st["m0"], st["csw"])
    scale = np.abs(st["hop"]).max()
    assert np.abs(op.self_blocks.numpy() - st["self"]).max() / scale < 1e-12
    assert np.abs(op.hop_blocks.numpy() - st["hop"]).max() / scale < 1e-12
    assert op.dims == st["cdims"]


def test_apply_at_equals_whole_lattice_apply(ragged_setup):
    """The per-site evaluation (used on sampled sites of lattices too large for the host) is the
    same stencil as the whole-lattice apply, which the assembled matrix pins."""
    st = ragged_setup
    s, h, dims = st["self"], st["hop"], st["cdims"]
    from synthetic import draws
    N = s.shape[0] * s.shape[1]
    v = draws.rhs((*st["key"], 90), 1, N)[0]
    sites = np.arange(s.shape[0])
    for mu in (0.0, 0.05):
        full = coarse.apply(s, h, dims, v, mu).reshape(s.shape[0], -1)
        at = coarse.apply_at(lambda x: (s[x], h[x]), dims, v, sites, mu)
        assert np.abs(at - full).max() <= 1e-13 * np.abs(full).max()
