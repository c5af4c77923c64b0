"""The symmetric product's tile order (csrc/tile_walk.cuh), checked on the host.

The header is plain integer code shared by the kernel and this check: tests/native/tile_walk_check.cpp
includes it, walks every CTA's range and verifies that the CTAs together visit each tile of the upper
triangle exactly once, that segment starts (where the kernel loads a row's operands and, at the
previous tile, adds out_I onto out) fall exactly on a CTA's first tile, a band change or a row change,
that the per-CTA counts the kernel sizes its loops by match the walk, that every band is split evenly,
and that with a single band the order is the row-by-row numbering of the triangle cut into contiguous
ranges.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_17898_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "tile_walk_check.cpp")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("tile_walk") / "tile_walk_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, SRC, "-o", exe], check=True)
    return exe


def _band_width(t):
    """The host's band width (csrc/mv_tc.cu, tcs_band_tiles): 48 MiB of column-side operands per band."""
    return max(1, (48 << 20) // (128 * (8 * t + 64)))


@pytest.mark.parametrize("nb,W,ncta", [
    (8, 8, 36),                       # N = 1024: more CTAs than tiles per row, one band
    (782, _band_width(32), 152),      # N = 100000, t = 32: one band (the LML bench)
    (3907, _band_width(32), 152),     # N = 500000, t = 32: four bands
    (3907, _band_width(16), 152),     # N = 500000, t = 16
    (1229, 1228, 152),                # one column more than a band: a one-column last band
    (100, 7, 13), (5, 2, 3), (10, 3, 152), (1, 1, 1), (2, 1, 3), (300, 1, 152),
])
def test_every_tile_once_and_segments_consistent(checker, nb, W, ncta):
    out = subprocess.run([checker, str(nb), str(W), str(ncta)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    ok, tiles, bands = out.stdout.split()
    assert ok == "ok" and int(tiles) == nb * (nb + 1) // 2
    assert int(bands) == -(-nb // max(1, min(W, nb)))


def test_band_width_keeps_the_bench_shape_in_one_band():
    """At N = 100000 the column-side operands fit L2 whole, so the order is the plain row-by-row one."""
    assert _band_width(32) >= 782 and _band_width(16) >= 782
