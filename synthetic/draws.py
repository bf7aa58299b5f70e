"""Seeded random draws shared by the oracle, the tests and the benchmark.

Every random number that enters a coarse solve is drawn here, on the host,
with NumPy's PCG64 seeded by ``SeedSequence([config_id, instance, stream])``.
PCG64 is platform independent, so the same key gives bit-identical draws on
x86 and Arm hosts.  Nothing in this module performs any step of the solver.

Streams:
    0  gauge links (site-major, direction-minor)
    1  test-vector starting vectors
    2  right-hand sides
    3  polynomial start vector
    4  loss vector ``c`` and finite-difference entry picks
    5  recipe of a batch of uneven operators
"""
from __future__ import annotations

import numpy as np

STREAM_GAUGE = 0
STREAM_TESTVEC = 1
STREAM_RHS = 2
STREAM_POLY = 3
STREAM_GRAD = 4
STREAM_BATCH = 5


def rng(key, stream: int) -> np.random.Generator:
    """Generator for ``key`` (tuple of ints, e.g. (config_id, instance)) and ``stream``."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([*map(int, key), int(stream)])))


def complex_gaussian(gen: np.random.Generator, shape) -> np.ndarray:
    """Complex128 array whose real and imaginary parts are iid N(0, 1)."""
    shape = tuple(shape)
    z = gen.standard_normal(shape + (2,))
    return z[..., 0] + 1j * z[..., 1]


def gauge_algebra(key, volume: int) -> np.ndarray:
    """Raw 3x3 complex Gaussian matrices for every (site, direction), shape (V, 4, 3, 3)."""
    return complex_gaussian(rng(key, STREAM_GAUGE), (volume, 4, 3, 3))


def test_vector_starts(key, volume: int, nv: int) -> np.ndarray:
    """Starting vectors of the ``nv`` test vectors, shape (nv, V, 4, 3)."""
    gen = rng(key, STREAM_TESTVEC)
    return np.stack([complex_gaussian(gen, (volume, 4, 3)) for _ in range(nv)])


def rhs(key, count: int, n_unknowns: int, index0: int = 0) -> np.ndarray:
    """``count`` complex Gaussian right-hand sides of length ``n_unknowns``.

    Right-hand side ``index0 + i`` is always the same vector whatever ``count`` is,
    so a sample of a longer sequence can be regenerated cheaply.
    """
    out = np.empty((count, n_unknowns), dtype=np.complex128)
    for i in range(count):
        gen = rng((*key, index0 + i), STREAM_RHS)
        out[i] = complex_gaussian(gen, (n_unknowns,))
    return out


def poly_start(key, n_unknowns: int) -> np.ndarray:
    """Random start vector of the polynomial's Arnoldi process (unnormalised)."""
    return complex_gaussian(rng(key, STREAM_POLY), (n_unknowns,))


def grad_draws(key, n_unknowns: int, volume: int, n: int, picks: int):
    """Loss vector ``c``, source ``b`` and ``picks`` random block entries for the FD check.

    Entries are (site, block, row, col) with block 0 = self and 1..8 = hop direction 0..7.
    """
    gen = rng(key, STREAM_GRAD)
    c = complex_gaussian(gen, (n_unknowns,))
    b = complex_gaussian(gen, (n_unknowns,))
    ent = np.stack([gen.integers(0, volume, picks), gen.integers(0, 9, picks),
                    gen.integers(0, n, picks), gen.integers(0, n, picks)], axis=1)
    return c, b, ent


def batch_recipe(key, count: int, extents=(4, 6, 8), nvs=(8, 16, 24), m0_range=(-0.44, -0.38), max_rhs=12):
    """Uneven batch: per operator (coarse extent L, nv, m0, number of right-hand sides)."""
    gen = rng(key, STREAM_BATCH)
    L = gen.choice(extents, size=count)
    nv = gen.choice(nvs, size=count)
    m0 = gen.uniform(m0_range[0], m0_range[1], size=count)
    nr = gen.integers(1, max_rhs + 1, size=count)
    return [(int(L[i]), int(nv[i]), float(m0[i]), int(nr[i])) for i in range(count)]
