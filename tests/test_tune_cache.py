"""Host logic of the autotuner's cache (no GPU): the key, the last matching
line winning, malformed and out-of-range lines ignored, a miss and a missing
file reported as no entry."""
import os
import shutil

import pytest


@pytest.fixture(scope="module")
def lookup():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_00281_gb300.build import build_library
    build_library()
    from paper_2005_00281_gb300 import bh
    return bh.tune_lookup


def test_cache_lookup(lookup, tmp_path):
    p = tmp_path / "cache.txt"
    p.write_text("# comment line\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 32 0 0 1 0 12.5 ms/32-step-pair\n"
                 "NVIDIA_GB300|nr240|P1600|shots1 1 2 1 0 1 3.1 ms/32-step-pair\n"
                 "garbage line\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 99 0 0 0 0 bad group\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 2 5 0 0 bad tile code\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 2 1 3 0 bad split\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 2 1 1 2 bad order\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 2 1 1 11.0 missing order\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 2 1 11.0 missing split\n"
                 "NVIDIA_GB300|nr240|P2016|shots64 16 0 1 1 1 11.0 ms/32-step-pair\n"
                 "NVIDIA_GB300|nr240|P2048|shots16 16 0 1 2 0 5.0 ms/32-step-pair\n")
    # blanks in the GPU name become underscores; the last valid line wins
    assert lookup(str(p), "NVIDIA GB300", 240, 2016, 64) == (16, 0, 1, 1, 1)
    assert lookup(str(p), "NVIDIA GB300", 240, 1600, 1) == (1, 2, 1, 0, 1)
    assert lookup(str(p), "NVIDIA GB300", 240, 2048, 16) == (16, 0, 1, 2, 0)
    # other shapes, other GPUs, a missing file: no entry
    assert lookup(str(p), "NVIDIA GB300", 240, 2016, 63) is None
    assert lookup(str(p), "NVIDIA B200", 240, 2016, 64) is None
    assert lookup(str(tmp_path / "none.txt"), "NVIDIA GB300", 240, 2016, 64) is None


def test_committed_cache_is_well_formed(lookup):
    """Every line of the committed cache parses and names a valid choice."""
    from paper_2005_00281_gb300.bh import TUNE_CACHE
    if not os.path.exists(TUNE_CACHE):
        pytest.skip("no committed cache")
    for line in open(TUNE_CACHE):
        if not line.strip() or line.startswith("#"):
            continue
        key, g, f, v, sp, od = line.split()[:6]
        gpu, nr, P, shots = key.split("|")
        assert 1 <= int(g) <= 32 and int(f) in (0, 1, 2) and int(v) in (0, 1)
        assert int(sp) in (0, 1, 2, 3, 4) and int(od) in (0, 1)
        assert lookup(TUNE_CACHE, gpu, int(nr[2:]), int(P[1:]), int(shots[5:])) is not None
