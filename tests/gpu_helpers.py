"""Shared fixtures of the GPU parity tests: seeded synthetic operators and the oracle side."""
import numpy as np
import torch

from synthetic import draws
from synthetic.coarse_op import build_coarse_operator


def make_op(key, fine_dims, nv, m0=-0.4, csw=1.0, device="cpu"):
    return build_coarse_operator(key, fine_dims, nv, m0, csw, device=device)


def to_cuda(op, mu=0.0, precisions=(1, 2), max_nrhs=1):
    from paper_2205_09104_gb300 import CoarseOp
    s = op.self_blocks.to("cuda").contiguous()
    h = op.hop_blocks.to("cuda").contiguous()
    return CoarseOp(s, h, op.dims, op.nv, mu=mu, precisions=precisions, max_nrhs=max_nrhs)


def rhs(key, count, N, index0=0):
    return draws.rhs(key, count, N, index0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
