"""Subprocess body of test_gpu_eo_configs: with COARSE_AUTOTUNE_CACHE fixing the layout of the
odd-even half apply, apply S in FP64 / FP32 / BF16 and check it against the oracle."""
import sys

import torch

sys.path.insert(0, __file__.rsplit("/", 1)[0])
from gpu_helpers import make_op, rel, rhs  # noqa: E402
from oracle import oddeven as ooe  # noqa: E402

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-2}


def main(nv, fdims, mu):
    from paper_2205_09104_gb300 import CoarseOp, autotune_report
    op = make_op((540, nv), fdims, nv)
    dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=mu, precisions=(1, 2))
    N2 = op.volume * op.n // 2
    x = rhs((541, nv), 1, N2)[0]
    ref = ooe.schur_apply(op.self_blocks.numpy(), op.hop_blocks.numpy(), op.dims, x, mu)
    for prec in (0, 1, 2):
        dt = torch.complex128 if prec == 0 else torch.complex64
        y = dev.schur(torch.from_numpy(x).to("cuda", dt), precision=prec).cpu().numpy()
        assert rel(y, ref) <= TOL[prec], (prec, rel(y, ref))
    dev.close()
    print(autotune_report())
    print("ok")


if __name__ == "__main__":
    main(int(sys.argv[1]), tuple(int(v) for v in sys.argv[2].split("x")), float(sys.argv[3]))
