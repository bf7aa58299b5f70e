"""Every layout the autotuner may pick for the odd-even half apply (one CTA of 4 warps per site,
one warp per site, one CTA of 2 warps per site with rolled or unrolled directions, the last two
also with the inverse block and epilogue vectors prefetched into shared memory, and the streamed
persistent layout) gives the oracle's S = 1 - D_ee^-1 D_eo D_oo^-1 D_oe, and solves through it
reach the oracle's 1e-10: the layout is fixed through the autotuner's cache file in a
subprocess.  The small lattices give the streamed layout one site per CTA; the coarse 8^4
lattice (2048 sites per parity on 152 SMs) makes its CTAs walk 13-14 sites, so that every stage
(3 in FP32, 5 in BF16) is refilled several times, its mbarrier phases flip, and the producer
reads its neighbour records in two batches of 8 sites."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = [(8, "8x8x8x8", 0.0), (16, "8x4x4x8", 0.03), (24, "4x8x4x4", 0.0)]  # coarse 4^4, 4x2x2x4, 2x4x2x2


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("nv,fdims,mu", CASES)
def test_eo_layout(tmp_path, variant, nv, fdims, mu):
    _run(tmp_path, variant, nv, fdims, mu)


def test_eo_streamed_many_sites_per_cta(tmp_path):
    _run(tmp_path, 6, 16, "16x16x16x16", 0.03)


def _run(tmp_path, variant, nv, fdims, mu):
    n = 2 * nv
    V = 1
    for d in fdims.split("x"):
        V *= int(d) // 2
    b = V.bit_length() - 1
    cache = tmp_path / "tune.txt"
    with open(cache, "w") as f:
        for p in (0, 1, 2):
            f.write(f"eo/p{p}/n{n}/v{b} {variant} 0 0 0\n")
    env = dict(os.environ, COARSE_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(HERE)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, os.path.join(HERE, "eo_config_worker.py"), str(nv), fdims, str(mu)],
                         env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert out.stdout.strip().endswith("ok")
    for p in (0, 1, 2):  # (FP64 blocks run the streamed choice as the prefetching layout 4)
        assert f"eo/p{p}/n{n}/v{b} -> {variant} 0 0" in out.stdout
