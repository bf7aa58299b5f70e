"""coarse_residual_noalloc against coarse_residual, through the C ABI.

The no-allocation variant serves callers that cannot allocate device memory
during the call (an outside memory arena, a code path where allocation is not
allowed); its scratch is one static device array shared by all calls.  It must
give the same residual and norms as the ordinary entry point, also on a second
call in a row (the shared array keeps the previous call's contents).
Tolerance: the FP64 apply bar of the other tests, 1e-12 relative.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _residuals(dev, b, x):
    from paper_2205_09104_gb300 import _abi
    L = _abi.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    r1 = torch.empty_like(b)
    r2 = torch.full_like(b, float("nan"))
    n1 = (ctypes.c_double * 2)()
    n2 = (ctypes.c_double * 2)()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    _abi.check(L.coarse_residual(dev.handle, P(b), P(x), P(r1), n1, s))
    _abi.check(L.coarse_residual_noalloc(dev.handle, P(b), P(x), P(r2), n2, s))
    return r1.cpu().numpy(), r2.cpu().numpy(), np.array(n1[:]), np.array(n2[:])


def test_noalloc_residual_matches_twice():
    from gpu_helpers import make_op, rhs, to_cuda
    op = make_op((1, 0), (8, 8, 8, 8), 8, m0=-0.4)       # 4^4 coarse, n = 16: 4096 unknowns
    dev = to_cuda(op, mu=0.01, precisions=())
    N = op.volume * op.n
    for call in range(2):
        v = rhs((1, 70 + call), 2, N)
        b = torch.from_numpy(v[0]).cuda()
        x = torch.from_numpy(v[1]).cuda()
        r1, r2, n1, n2 = _residuals(dev, b, x)
        assert np.linalg.norm(r2 - r1) <= 1e-12 * np.linalg.norm(r1), call
        assert np.all(np.abs(n2 - n1) <= 1e-12 * n1), call
    dev.close()


def test_noalloc_ragged_lattice_after_larger_one():
    """A smaller, ragged operator right after: stale counters of the previous call must not leak."""
    from gpu_helpers import make_op, rhs, to_cuda
    op = make_op((600, 0), (6, 4, 4, 6), 8, m0=-0.4)     # 3x2x2x3 coarse sites
    dev = to_cuda(op, precisions=())
    N = op.volume * op.n
    v = rhs((600, 71), 2, N)
    r1, r2, n1, n2 = _residuals(dev, torch.from_numpy(v[0]).cuda(), torch.from_numpy(v[1]).cuda())
    assert np.linalg.norm(r2 - r1) <= 1e-12 * np.linalg.norm(r1)
    dev.close()


def test_noalloc_rejects_too_large():
    from paper_2205_09104_gb300 import CoarseOp, _abi
    V, nv = 8 * 8 * 8 * 8, 24                            # 4096 sites x 48 = 196608 unknowns > 131072
    g = torch.Generator(device="cpu").manual_seed(1)
    s = torch.randn(V, 48, 48, dtype=torch.complex128, generator=g).cuda()
    h = torch.randn(V, 4, 48, 48, dtype=torch.complex128, generator=g).cuda()
    dev = CoarseOp(s, h, (8, 8, 8, 8), nv, precisions=(), assume_gamma5=True)
    N = V * 48
    b = torch.zeros(N, dtype=torch.complex128, device="cuda")
    r = torch.empty_like(b)
    n = (ctypes.c_double * 2)()
    L = _abi.lib()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = L.coarse_residual_noalloc(dev.handle, P(b), P(b.clone()), P(r), n,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"exceed" in L.coarse_last_error()
    dev.close()
