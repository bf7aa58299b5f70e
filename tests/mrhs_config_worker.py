"""Subprocess body of test_gpu_mrhs_configs: with COARSE_AUTOTUNE_CACHE pointing at a file that
fixes the multi-RHS launch configuration per lattice-size bucket, apply Y = D_c X for several
operators and check every column against the oracle on the BF16-rounded operands (2e-5)."""
import sys

import numpy as np
import torch

sys.path.insert(0, __file__.rsplit("/", 1)[0])
from gpu_helpers import abs_apply, assert_entrywise, make_op, rel, rhs, stencil_factor  # noqa: E402
from oracle import coarse as ocoarse  # noqa: E402
from oracle.lattice import neighbours  # noqa: E402


def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return torch.complex(re, im).numpy()


def main(nv, fine_dims_list, nrhs_list):
    from paper_2205_09104_gb300 import CoarseOp, autotune_report
    for i, fdims in enumerate(fine_dims_list):
        op = make_op((520, nv, i), fdims, nv)
        s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
        s3 = ocoarse.sigma3(op.n // 2)
        nb = neighbours(op.dims)
        sr, hr = bf16(s), bf16(h)
        for mu in range(4):
            back = hr[nb[:, 4 + mu], mu]
            hr[:, 4 + mu] = s3[None, :, None] * np.conj(np.transpose(back, (0, 2, 1))) * s3[None, None, :]
        dev = CoarseOp(op.self_blocks.cuda(), op.hop_blocks.cuda(), op.dims, op.nv, mu=0.02, precisions=(2,),
                       max_nrhs=12)
        N = op.volume * op.n
        for nrhs in nrhs_list:
            X = torch.from_numpy(rhs((520, nv, i, nrhs), nrhs, N)).to("cuda", torch.complex64)
            Y = dev.apply(X, precision=2).cpu().numpy().astype(np.complex128)
            X32 = X.cpu().numpy().astype(np.complex128)
            Xr = bf16(X32)
            s3v = np.tile(s3, op.volume)
            for c in range(nrhs):
                ref = ocoarse.apply(sr, hr, op.dims, Xr[c], 0.0) + 1j * 0.02 * s3v * X32[c]
                err = rel(Y[c], ref)
                assert err <= 2e-5, (fdims, nrhs, c, err)
                mag = abs_apply(sr, hr, op.dims, Xr[c]) + 0.02 * np.abs(X32[c])
                assert_entrywise(Y[c], ref, stencil_factor(2, op.n, rounded_operands=True) * mag,
                                 f"{fdims} nrhs={nrhs} column {c}")
        dev.close()
    print(autotune_report())
    print("ok")


if __name__ == "__main__":
    nv = int(sys.argv[1])
    dims = [tuple(int(v) for v in d.split("x")) for d in sys.argv[2].split(",")]
    counts = [int(v) for v in sys.argv[3].split(",")]
    main(nv, dims, counts)
