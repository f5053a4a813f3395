"""Host-side arithmetic of the benchmark's roofline objects, on CPU.

The algorithmic flop counts are checked against brute-force loops over the
tiled schedule written out step by step (every product column of every tile
update; every row of every diagonal tile and column), and the
traffic lookup against a committed-summary stand-in: the figure is reported
only while the kernel source matches the hash the capture was taken on.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Inst:
    def __init__(self, n, m_real, m_cplx):
        self.n, self.m_real, self.m_cplx = n, m_real, m_cplx
        self.ncol = m_real + 2 * m_cplx


def _tiles(n, br):
    """(first row, height) of every diagonal tile, bottom tile last: the top
    tile takes the remainder."""
    N = -(-n // br)
    b0 = n - (N - 1) * br
    out, p = [(0, b0)], b0
    while p < n:
        out.append((p, br))
        p += br
    return out


@pytest.mark.parametrize("n,br,ncol", [(4096, 64, 1024), (1000, 64, 37), (130, 32, 5), (64, 64, 3)])
def test_update_flops_brute_force(n, br, ncol):
    total, launches = bench.update_flops(n, ncol, br)
    tiles = _tiles(n, br)
    brute, count = 0, 0
    for (p0, bt) in tiles[1:]:  # every tile but the top one updates the rows above it
        count += 1
        for _col in range(2 * ncol):  # [Z'|W]: two product columns per solution column
            brute += 2 * p0 * bt  # one multiply-add per (row above, tile row)
    assert launches == count == len(tiles) - 1
    assert total == brute


@pytest.mark.parametrize("n,br,mr,mc", [(4096, 64, 512, 256), (200, 64, 3, 2), (64, 64, 1, 0),
                                         (130, 32, 4, 3)])
def test_diag_flops_brute_force(n, br, mr, mc):
    # the per-column count of the diagonal-tile work (Table "flops-vector"):
    # 5 b_r flops per row of every diagonal tile and solution column (a
    # complex shift owns two columns)
    total, launches = bench.diag_flops(_Inst(n, mr, mc), br)
    brute = 0
    for (_p0, bt) in _tiles(n, br):
        for _col in range(mr + 2 * mc):
            for _row in range(bt):
                brute += 5 * br
    assert launches == len(_tiles(n, br))
    assert total == brute


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "kern.cu"
    src.write_text("__global__ void k() {}\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.source_hash("kern.cu")
    (prof / "k.txt").write_text("notes: x\nsource_sha256: %s\n"
                                "dram_bytes_per_launch_full_size: 12345\n" % h)
    assert bench.profiled_traffic("kern.cu", "k.txt") == 12345.0
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.profiled_traffic("kern.cu", "k.txt") is None
    assert bench.profiled_traffic("kern.cu", "missing.txt") is None

