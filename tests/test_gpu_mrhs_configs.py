"""Every launch configuration the autotuner may pick for the multi-RHS apply (sites per stage P,
pipeline stages S) gives the oracle's result: the configurations are fixed through the
autotuner's cache file (COARSE_AUTOTUNE_CACHE) in a subprocess, one per lattice-size bucket and
column-tile count, and each is checked against the oracle on BF16-rounded operands."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# coarse lattices of 16, 36 and 81 sites (buckets 4, 5, 6) from fine lattices of twice the extent
FINE = ["4x4x4x4", "6x4x4x6", "6x6x6x6"]
BUCKETS = [4, 5, 6]
LAYOUTS = {  # nv: (P, S) per bucket
    8: [(2, 3), (4, 5), (8, 8)],
    16: [(1, 3), (2, 5), (4, 8)],
    24: [(1, 8), (2, 3), (1, 5)],
}


@pytest.mark.parametrize("nv", [8, 16, 24])
def test_mrhs_every_config(tmp_path, nv):
    n = 2 * nv
    cache = tmp_path / "tune.txt"
    with open(cache, "w") as f:
        for b, (P, S) in zip(BUCKETS, LAYOUTS[nv]):
            for t in (1, 2, 3):
                f.write(f"mrhs/n{n}/t{t}/v{b} {P} {S} 0 0\n")
    env = dict(os.environ, COARSE_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(HERE)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, os.path.join(HERE, "mrhs_config_worker.py"), str(nv), ",".join(FINE),
                          "2,7,12"], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert out.stdout.strip().endswith("ok")
    for b, (P, S) in zip(BUCKETS, LAYOUTS[nv]):
        assert f"mrhs/n{n}/t3/v{b} -> {P} {S} 0" in out.stdout
