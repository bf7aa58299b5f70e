"""Subprocess body of test_gpu_eo_configs: with COARSE_AUTOTUNE_CACHE fixing the layout of the
odd-even half apply, apply S in FP64 / FP32 / BF16 and check it against the oracle, then solve
through the reduced system (right-hand side pass with z, polynomial chain with acc, solution
retrieval with base) in FP32, FP32 with the BF16 chain, and BF16, each to the oracle's 1e-10."""
import sys

import numpy as np
import torch

sys.path.insert(0, __file__.rsplit("/", 1)[0])
from gpu_helpers import check_schur_entrywise, make_op, rel, rhs  # noqa: E402
from oracle import coarse as ocoarse  # noqa: E402
from oracle import oddeven as ooe  # noqa: E402

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-2}


def main(nv, fdims, mu):
    from paper_2205_09104_gb300 import CoarseOp, autotune_report
    big = 1
    for d in fdims:
        big *= d
    # large lattices: the synthetic operator is built on the GPU (the same arrays feed the oracle)
    op = make_op((540, nv), fdims, nv, device="cuda" if big >= 16 ** 4 else "cpu")
    op.self_blocks, op.hop_blocks = op.self_blocks.cpu(), op.hop_blocks.cpu()
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(1, 2))
    N2 = op.volume * op.n // 2
    x = rhs((541, nv), 1, N2)[0]
    ref = ooe.schur_apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    for prec in (0, 1, 2):
        dt = torch.complex128 if prec == 0 else torch.complex64
        y = dev.schur(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy()
        assert rel(y, ref) <= TOL[prec], (prec, rel(y, ref))
        check_schur_entrywise(y, torch.from_numpy(x).to(dt).numpy(), op.self_blocks.numpy(), op.hop_blocks.numpy(),
                              op.dims, prec, mu, f"layout worker {fdims}")
    from paper_2205_09104_gb300 import COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_ZERO_GUESS, solve_params
    sb, hb = op.self_blocks.numpy(), op.hop_blocks.numpy()
    b = rhs((542, nv), 1, 2 * N2)[0]
    for prec, extra in ((1, 0), (1, COARSE_POLY_BF16), (2, 0)):
        p = solve_params(m=30, tol=1e-10, precision=prec, poly_degree=4, defl_k=8, recycle_updates=5,
                         inner_tol=2e-6 if prec == 1 else 1e-2, max_ir=40,
                         flags=COARSE_ZERO_GUESS | COARSE_ODD_EVEN | extra)
        xs, info = dev.solve(torch.from_numpy(b).cuda(), params=p)
        res = np.linalg.norm(b - ocoarse.apply(sb, hb, op.dims, xs.cpu().numpy(), mu)) / np.linalg.norm(b)
        assert info[0]["status"] == 0 and res <= 1e-10, (prec, extra, info[0], res)
    dev.close()
    print(autotune_report())
    print("ok")


if __name__ == "__main__":
    main(int(sys.argv[1]), tuple(int(v) for v in sys.argv[2].split("x")), float(sys.argv[3]))
