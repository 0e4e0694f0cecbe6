"""I/O model of the MOMMS family on the GPU's memory levels.

The paper counts the words a resident algorithm moves between a slow and a fast
memory (Sec. 2.2): Resident C with an m_c x n_c block of C reads A ceil(n/n_c)
times and B ceil(m/m_c) times; Resident A (B) keeps an m_c x k_c (k_c x n_c) block
and re-reads and re-writes C once per k_c block.  This module states those closed
forms and applies them to the GPU level structure:

* HBM -> L2: the resident block is the set of C tiles the ~one wave of persistent
  CTAs works on at a time; its tile rows and columns are read from HBM once per
  wave (and, in the emulated kernel, once per digit pair, because the
  diagonal-major loop streams every pair's panels again).  Which tiles share a
  wave is the member's tile order, taken from the library itself
  (``momms_member_tile``), so the model and the kernels cannot drift apart.
* L2 -> SM: each CTA streams its own A and B panels for every tile.

The closed forms are pinned to the CPU oracle's counting simulation in the tests.
"""
from __future__ import annotations

import ctypes
import math

from . import momms as M

MEMBERS = {"C2": M.MEMBER_C2, "A2": M.MEMBER_A2, "B2": M.MEMBER_B2, "A1": M.MEMBER_A1}


def cdiv(a: int, b: int) -> int:
    return -(-a // b)


# ----------------------------------------------------------------------------- closed forms (Sec. 2.2)
def resident_c_words(m, n, k, mc, nc, c_read=True):
    """Sec. 2.2.1: C block m_c x n_c resident; A, B streamed."""
    return {"a_reads": m * k * cdiv(n, nc), "b_reads": k * n * cdiv(m, mc),
            "c_reads": m * n if c_read else 0, "c_writes": m * n}


def resident_a_words(m, n, k, mc, kc, c_read=True):
    """Sec. 2.2.2: A block m_c x k_c resident; B and C streamed, C once per k_c block."""
    nk = cdiv(k, kc)
    return {"a_reads": m * k, "b_reads": k * n * cdiv(m, mc),
            "c_reads": m * n * (nk - 1 + int(c_read)), "c_writes": m * n * nk}


def resident_b_words(m, n, k, kc, nc, c_read=True):
    """Mirror of Resident A (Sec. 2.2.2)."""
    nk = cdiv(k, kc)
    return {"a_reads": m * k * cdiv(n, nc), "b_reads": k * n,
            "c_reads": m * n * (nk - 1 + int(c_read)), "c_writes": m * n * nk}


def goto_words(m, n, k, nc, kc, c_read=True):
    """Goto's A2C0 at the main-memory level (Sec. 4.3, Sec. 5.2): A per n_c panel, B once,
    C read and written once per k_c block."""
    nk = cdiv(k, kc)
    return {"a_reads": m * k * cdiv(n, nc), "b_reads": k * n,
            "c_reads": m * n * (nk - 1 + int(c_read)), "c_writes": m * n * nk}


def intensity_flops_per_word(m, n, k, words):
    return 2.0 * m * n * k / sum(words.values())


# ----------------------------------------------------------------------------- member tile orders
def member_tile(member: int, group: int, cta: int, ctas: int, i: int, tiles_m: int, tiles_n: int):
    """The i-th tile of CTA `cta` under `member` (None when the CTA has no i-th tile)."""
    tm = ctypes.c_int(0)
    tn = ctypes.c_int(0)
    ok = M.lib().momms_member_tile(member, group, cta, ctas, i, tiles_m, tiles_n, ctypes.byref(tm),
                                   ctypes.byref(tn))
    return (tm.value, tn.value) if ok == 1 else None


def tri_tiles(uplo: int, tile_n: int, n: int):
    """The tiles a triangular product (the modular symmetric rank-k update of an n x n C)
    visits, in the kernel's order (``momms_tri_tile``)."""
    tm = ctypes.c_int(0)
    tn = ctypes.c_int(0)
    cnt = ctypes.c_int64(0)
    out = []
    t = 0
    while True:
        ok = M.lib().momms_tri_tile(uplo, tile_n, n, t, ctypes.byref(tm), ctypes.byref(tn), ctypes.byref(cnt))
        if ok < 0:
            raise ValueError(f"momms_tri_tile: bad argument {-ok}")
        if ok == 0:
            break
        out.append((tm.value, tn.value))
        t += 1
    if len(out) != cnt.value:
        raise RuntimeError("momms_tri_tile: count and enumeration disagree")
    return out


def waves(member: int, tiles_m: int, tiles_n: int, ctas: int, group: int = 0):
    """For every round i of the persistent loop, the distinct tile rows and columns in flight."""
    out = []
    i = 0
    while True:
        rows, cols = set(), set()
        for b in range(ctas):
            t = member_tile(member, group, b, ctas, i, tiles_m, tiles_n)
            if t is not None:
                rows.add(t[0])
                cols.add(t[1])
        if not rows:
            return out
        out.append((len(rows), len(cols)))
        i += 1


# ----------------------------------------------------------------------------- GPU predictions
def emulated_dram_bytes(member: int, m: int, n: int, k: int, S: int, ctas: int = 152, bm: int = 128,
                        bn: int = 192, group: int = 0, beta_nonzero: bool = True):
    """HBM bytes of one slice-product launch: per round of persistent CTAs and per digit pair, the
    tile rows of A's slice and tile columns of B's slice in flight are read once (Resident C at the
    L2 level, the round's tiles being the resident block); plus C read (beta != 0) and written."""
    tiles_m, tiles_n = cdiv(m, bm), cdiv(n, bn)
    k_pad = cdiv(k, 64) * 64
    pairs = S * (S + 1) // 2
    w = waves(member, tiles_m, tiles_n, min(ctas, tiles_m * tiles_n), group)
    a_rows = sum(min(r * bm, m) for r, _ in w)
    b_cols = sum(min(c * bn, n) for _, c in w)
    digits = pairs * (a_rows + b_cols) * k_pad * 2
    c_bytes = 8 * m * n * (2 if beta_nonzero else 1)
    return {"digits": digits, "c": c_bytes, "total": digits + c_bytes, "rounds": len(w),
            "mean_rows_per_round": a_rows / max(len(w), 1) / bm,
            "mean_cols_per_round": b_cols / max(len(w), 1) / bn}


def modular_dram_bytes(member: int, m: int, n: int, k: int, N: int, ctas: int = 152, bm: int = 128,
                       bn: int = 192, group: int = 0):
    """HBM bytes of one residue-product launch of the modular encoding: the units run modulus by
    modulus through the member's tile order, so per modulus and round the tile rows of A's residue
    plane and tile columns of B's plane in flight are read once (as a digit pair of the slice
    kernel); the launch writes the N residue bytes of every element of C and does not touch C."""
    tiles_m, tiles_n = cdiv(m, bm), cdiv(n, bn)
    k_pad = cdiv(k, 64) * 64
    w = waves(member, tiles_m, tiles_n, min(ctas, tiles_m * tiles_n), group)
    a_rows = sum(min(r * bm, m) for r, _ in w)
    b_cols = sum(min(c * bn, n) for _, c in w)
    planes = N * (a_rows + b_cols) * k_pad * 2
    residues = N * m * n
    return {"planes": planes, "residues": residues, "total": planes + residues, "rounds": len(w)}


def triangle_dram_bytes(uplo: int, n: int, k: int, N: int, ctas: int = 152, bn: int = 192, bm: int = 128):
    """HBM bytes of the residue-product launch of a symmetric rank-k update (C n x n, one
    triangle): per modulus the units run through the tiles that meet the triangle in the kernel's
    order (``tri_tiles``), a round being ``ctas`` consecutive tiles.  Both operands are the same
    residue plane (op(A) and its transpose), so a round reads the union of the plane rows its tile
    rows (bm each) and tile columns (bn each) need, once per modulus.  The launch writes the N
    residue bytes of every element of the visited tiles (the whole diagonal tiles)."""
    order = tri_tiles(uplo, bn, n)
    k_pad = cdiv(k, 64) * 64
    rows_read = 0
    for r0 in range(0, len(order), ctas):
        need = set()
        for tm, tn in order[r0:r0 + ctas]:
            need.update(range(tm * bm, min(n, tm * bm + bm)))
            need.update(range(tn * bn, min(n, tn * bn + bn)))
        rows_read += len(need)
    planes = N * rows_read * k_pad * 2
    elems = sum((min(n, tm * bm + bm) - tm * bm) * (min(n, tn * bn + bn) - tn * bn) for tm, tn in order)
    residues = N * elems
    return {"planes": planes, "residues": residues, "total": planes + residues,
            "rounds": cdiv(len(order), ctas), "tiles": len(order)}


def emulated_l2_to_sm_bytes(m: int, n: int, k: int, S: int, bm: int = 128, bn: int = 192):
    """L2 -> SM bytes: every tile streams its A (bm rows) and B (bn rows) digit panels per pair."""
    tiles_m, tiles_n = cdiv(m, bm), cdiv(n, bn)
    k_pad = cdiv(k, 64) * 64
    pairs = S * (S + 1) // 2
    return pairs * tiles_m * tiles_n * (bm + bn) * k_pad * 2


def kept_a_l2_to_sm_bytes(m: int, n: int, k: int, N: int, ctas: int = 152, bm: int = 128, bn: int = 192):
    """L2 -> SM bytes of the short-k residue product (k <= 256) with the A tile kept in shared
    memory: CTA b takes the tiles [floor(b T / C), floor((b + 1) T / C)) row-major, modulus after
    modulus; it loads an A tile (bm rows of the modulus's plane) when its unit's (modulus, tile
    row) differs from the last one's, and every unit's B tile (bn rows).  The units are walked in
    the kernel's order (`ring` = the same units with A and B per unit, the ring kernel's bytes)."""
    tiles_m, tiles_n = cdiv(m, bm), cdiv(n, bn)
    T = tiles_m * tiles_n
    k_pad = cdiv(k, 64) * 64
    a_loads = units = 0
    for b in range(ctas):
        start, end = (b * T) // ctas, ((b + 1) * T) // ctas
        last = None
        for l in range(N):
            for t in range(start, end):
                key = (l, t // tiles_n)
                if key != last:
                    a_loads += 1
                    last = key
                units += 1
    a = a_loads * bm * k_pad * 2
    bb = units * bn * k_pad * 2
    return {"a": a, "b": bb, "total": a + bb, "a_loads": a_loads, "units": units,
            "ring": units * (bm + bn) * k_pad * 2}


def paper_member_intensity(name: str, M_words: int | None = None):
    """Flops per byte of the paper's CPU members at their published blocksizes (large m=n=k)."""
    L = 10 ** 7
    if name == "goto":
        w = goto_words(L, L, L, 3000, 192)
    elif name == "b3a2c0":
        w = resident_b_words(L, L, L, 768, 768)
    elif name == "a3b2c0":
        w = resident_a_words(L, L, L, 768, 768)
    elif name == "c3a2c0":
        w = resident_c_words(L, L, L, 624, 624)
    else:
        raise ValueError(name)
    return intensity_flops_per_word(L, L, L, w) / 8.0


def lower_bound_reads(m, n, k, M_words):
    """Sec. 2.1: at least 2mnk/sqrt(M) - 2M words read into a fast memory of M words."""
    return 2.0 * m * n * k / math.sqrt(M_words) - 2.0 * M_words
