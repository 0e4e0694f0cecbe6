"""The tile order of the triangular (symmetric rank-k) residue product, host side: for
every n up to 1500 and both triangles and tile widths, the tiles momms_tri_tile
enumerates are exactly the 128 x tile_n tiles of the n x n C that hold an element of the
triangle, each once, tile row by tile row -- checked against brute force over the tile
grid (the kernel maps its units with the same function)."""
import ctypes

import pytest

from paper_1904_05717_gb300 import iomodel
from paper_1904_05717_gb300 import momms as M


def brute(uplo, tile_n, n):
    out = []
    for r in range((n + 127) // 128):
        r0, r1 = 128 * r, min(n, 128 * r + 128) - 1
        for c in range((n + tile_n - 1) // tile_n):
            c0, c1 = tile_n * c, min(n, tile_n * c + tile_n) - 1
            if (r1 >= c0) if uplo == M.LOWER else (r0 <= c1):
                out.append((r, c))
    return out


@pytest.mark.parametrize("uplo", [M.LOWER, M.UPPER])
@pytest.mark.parametrize("tile_n", [96, 192])
def test_tri_tile_order_is_the_triangle_row_by_row(uplo, tile_n):
    sizes = list(range(1, 400)) + list(range(400, 1500, 37)) + [8192]
    for n in sizes:
        got = iomodel.tri_tiles(uplo, tile_n, n)
        assert got == brute(uplo, tile_n, n), n


def test_tri_tile_counts_and_errors():
    tm, tn, cnt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    lib = M.lib()
    # n = 8192 lower, 192-wide tiles: 64 tile rows, row r holds floor((128 r + 127) / 192) + 1 tiles
    assert lib.momms_tri_tile(M.LOWER, 192, 8192, 0, ctypes.byref(tm), ctypes.byref(tn), ctypes.byref(cnt)) == 1
    assert cnt.value == sum(min(43, (128 * r + 127) // 192 + 1) for r in range(64))
    assert lib.momms_tri_tile(M.UPPER, 96, 0, 0, ctypes.byref(tm), ctypes.byref(tn), ctypes.byref(cnt)) == 0
    assert cnt.value == 0
    assert lib.momms_tri_tile(5, 96, 10, 0, ctypes.byref(tm), ctypes.byref(tn), None) == -1
    assert lib.momms_tri_tile(M.LOWER, 128, 10, 0, ctypes.byref(tm), ctypes.byref(tn), None) == -2
    assert lib.momms_tri_tile(M.LOWER, 96, -1, 0, ctypes.byref(tm), ctypes.byref(tn), None) == -3
    assert lib.momms_tri_tile(M.LOWER, 96, 10, -1, ctypes.byref(tm), ctypes.byref(tn), None) == -4
    assert lib.momms_tri_tile(M.LOWER, 96, 10, 0, None, ctypes.byref(tn), None) == -5
    assert lib.momms_tri_tile(M.LOWER, 96, 10, 0, ctypes.byref(tm), None, None) == -6


def test_triangle_io_model_pins():
    # one tile (n <= 128): the round reads the n plane rows once per modulus and writes the
    # n^2 residues of each modulus
    for n, k, N in [(1, 1, 7), (100, 70, 12), (128, 8192, 13)]:
        b = iomodel.triangle_dram_bytes(M.LOWER, n, k, N)
        k_pad = -(-k // 64) * 64
        assert b["tiles"] == 1 and b["rounds"] == 1
        assert b["planes"] == N * n * k_pad * 2 and b["residues"] == N * n * n
    # the full 8192 problem: about half the full product's tiles, and each round of 152 tiles reads
    # no more plane rows than the whole plane
    b = iomodel.triangle_dram_bytes(M.LOWER, 8192, 8192, 12)
    full_tiles = 64 * 43
    assert full_tiles / 2 < b["tiles"] < full_tiles / 2 + 64
    assert b["planes"] <= 12 * b["rounds"] * 8192 * 8192 * 2
    assert b["residues"] == 12 * sum((min(8192, 128 * r + 128) - 128 * r) * (min(8192, 192 * c + 192) - 192 * c)
                                     for r, c in iomodel.tri_tiles(M.LOWER, 192, 8192))
    # the upper triangle visits about as many tiles as the lower one (the tiles are 128 x 192,
    # so the two sets differ along the diagonal by at most one tile per tile row)
    u = iomodel.triangle_dram_bytes(M.UPPER, 8192, 8192, 12)
    assert abs(u["tiles"] - b["tiles"]) <= 64
