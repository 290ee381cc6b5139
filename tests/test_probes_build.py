"""The measurement programs under ``paper_2401_02852_gb300/probes/`` (cluster
exchange, L2-resident phases, tile movers) are not part of the library, but
the design notes quote their numbers: each must still compile for sm_103a."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROBES = os.path.join(ROOT, "paper_2401_02852_gb300", "probes")


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(PROBES) if f.endswith(".cu")))
def test_probe_compiles(name, tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = tmp_path / (name[:-3] + ".o")
    res = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-c",
                          os.path.join(PROBES, name), "-o", str(out)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-3000:]
