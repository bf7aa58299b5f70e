"""FP64 CPU oracle for the coarsest-level solver (TEST INFRASTRUCTURE ONLY).

Plain, slow, obviously-correct NumPy/SciPy restatement of what the paper
computes, used only by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The library in
``paper_2205_09104_gb300`` never imports it, and it imports nothing from the
library: the two share only the seeded draws of ``synthetic.draws`` and
``synthetic.gauge`` (random numbers and the synthetic gauge field).

Modules and the passages they follow:
    lattice    gamma matrices (Sec. 2.1, Clifford relation), periodic neighbours
    fine       Wilson-clover / twisted-mass operator (Sec. 2.1, the Wilson-Dirac,
               clover and twisted-mass equations)
    multigrid  test vectors, aggregation prolongator, Galerkin blocks (Sec. 2.2)
    coarse     coarse stencil apply, sparse assembly, gamma5 relation (Sec. 2.2)
    krylov     Arnoldi (Alg. 1), GMRES(m) (Sec. 3.1), harmonic Ritz values and
               the GMRES polynomial (Sec. 3.3), Leja ordering (Alg. 2),
               polynomially preconditioned GMRES (Alg. 3), GCRO-DR (Sec. 3.4)
    gradient   adjoint solve and block gradients (Sec. 4.2: Q = Gamma5 D is Hermitian)
    oddeven    odd-even reduced system with block-Jacobi preconditioning (Sec. 2, 3.2)
    pipelined  latency-1 pipelined GMRES and GCRO-DR (Sec. 3.5, Alg. "pipe1fgmres",
               "pipe1gcrodr")

Every function is pinned by the ``-m "not gpu"`` tests to something other than
itself: closed forms, exact identities, brute force, or dense LU.  Functions
without such a pin say "parity unpinned" in their docstring; there are none.
"""
