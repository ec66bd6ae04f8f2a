"""Consistency of the committed ncu summaries the bench reads its DRAM traffic
from: each GEMM summary names its tile, the kernel source it was captured on
and the bytes per launch; the figures are plausible for an 8192^3 BF16 GEMM
and at least one summary matches the current kernel source."""
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _profiles():
    return sorted(glob.glob(os.path.join(ROOT, "profiles", "gemm_kernel_bf16_8192_*.md")))


def _kv(path):
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith(("#", "|", " ")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    return kv


@pytest.mark.parametrize("path", _profiles(), ids=os.path.basename)
def test_gemm_profile_records(path):
    kv = _kv(path)
    tile = tuple(int(x) for x in kv["tile"].split(","))
    assert len(tile) == 5
    bm, bn, bk, s, g = tile
    assert os.path.basename(path) == "gemm_kernel_bf16_8192_%dx%dx%d_s%d_g%d.md" % tile
    algorithmic = 2 * (8192 * 8192 * 2) + 8192 * 8192 * 4       # BF16 A and B once, FP32 C once
    traffic = float(kv["traffic_bytes"])
    assert algorithmic * 0.9 < traffic < algorithmic * 4
    assert len(kv["source_sha"]) == 16
    with open(path) as f:
        text = f.read()
    assert "--clock-control none" in text and "ncu" in text       # the command that made it


def test_a_profile_matches_the_current_kernel_source():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    shas = {_kv(p)["source_sha"] for p in _profiles()}
    assert bench._kernel_source_sha() in shas
