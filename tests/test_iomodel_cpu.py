"""The I/O model's closed forms against the oracle's counting simulation, and the
member tile orders (queried from the library, no GPU needed) against their
definition: every tile exactly once, in the stated order."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import iomodel as I
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn


@pytest.mark.parametrize("member,fn,b1,b2,b3", [("resident_c", I.resident_c_words, 8, 6, 0),
                                                ("resident_a", I.resident_a_words, 8, 5, 0),
                                                ("resident_b", I.resident_b_words, 5, 6, 0),
                                                ("goto", I.goto_words, 6, 5, 4)])
@pytest.mark.parametrize("c_read", [True, False])
def test_model_equals_counting_oracle(member, fn, b1, b2, b3, c_read):
    m, n, k = 37, 29, 41
    A = syn.matrix("int", m, k, 11)
    B = syn.matrix("int", k, n, 12)
    C = syn.matrix("int", m, n, 13)
    cnt = oracle.count_member(member, A, B, C.copy(order="F"), b1, b2, b3, c_read=c_read)
    want = fn(m, n, k, b1, b2, c_read)
    for key, v in want.items():
        assert cnt[key] == v


def test_paper_intensities_from_model():
    assert round(I.paper_member_intensity("goto"), 2) == 23.26
    assert round(I.paper_member_intensity("b3a2c0"), 2) == 64.0


@pytest.mark.parametrize("member", [M.MEMBER_C2, M.MEMBER_A2, M.MEMBER_B2, M.MEMBER_A1])
@pytest.mark.parametrize("tiles_m,tiles_n,ctas", [(7, 5, 4), (64, 43, 152), (3, 1, 8), (1, 9, 2)])
def test_member_orders_cover_every_tile_once(member, tiles_m, tiles_n, ctas):
    seen = np.zeros((tiles_m, tiles_n), dtype=int)
    for b in range(ctas):
        i = 0
        while True:
            t = I.member_tile(member, 8, b, ctas, i, tiles_m, tiles_n)
            if t is None:
                break
            seen[t] += 1
            i += 1
    assert np.all(seen == 1)


def test_member_orders_match_their_definitions():
    tm_, tn_, ctas = 20, 30, 7
    for b in range(ctas):
        for i in range(3):
            t = b + i * ctas
            assert I.member_tile(M.MEMBER_A2, 8, b, ctas, i, tm_, tn_) == (t // tn_, t % tn_)   # row-major
            assert I.member_tile(M.MEMBER_B2, 8, b, ctas, i, tm_, tn_) == (t % tm_, t // tm_)   # column-major
    # C2: groups of 8 tile rows walked column by column
    assert I.member_tile(M.MEMBER_C2, 8, 0, 1, 0, tm_, tn_) == (0, 0)
    assert I.member_tile(M.MEMBER_C2, 8, 0, 1, 7, tm_, tn_) == (7, 0)
    assert I.member_tile(M.MEMBER_C2, 8, 0, 1, 8, tm_, tn_) == (0, 1)
    # A1: contiguous runs per CTA
    per = -(-tm_ * tn_ // ctas)
    assert I.member_tile(M.MEMBER_A1, 8, 2, ctas, 0, tm_, tn_) == ((2 * per) // tn_, (2 * per) % tn_)


def test_wave_model_orders_members_as_the_paper_predicts():
    # one resident block per round of persistent CTAs: the grouped raster (C2) has the most
    # square round footprint and so the fewest HBM bytes; the blocked order (A1) the most
    sizes = {name: I.emulated_dram_bytes(mem, 8192, 8192, 8192, 6)["total"] for name, mem in I.MEMBERS.items()}
    assert sizes["C2"] < sizes["A2"] < sizes["A1"]
    assert sizes["C2"] < sizes["B2"] < sizes["A1"]


def test_modular_model_is_the_slice_model_with_moduli_for_pairs():
    # the residue product streams one plane pair per modulus as the slice kernel streams one per
    # digit pair: with N = S(S+1)/2 the operand bytes agree; it writes N bytes per element of C
    m, n, k = 4096, 4096, 4096
    for member in (1, 2, 3, 4):
        s = I.emulated_dram_bytes(member, m, n, k, S=4)
        r = I.modular_dram_bytes(member, m, n, k, N=10)
        assert r["planes"] == s["digits"] and r["residues"] == 10 * m * n


@pytest.mark.parametrize("m,n,N,ctas", [(16384, 16384, 15, 152), (300, 500, 11, 5), (2084, 1700, 12, 152),
                                        (128, 192, 3, 1)])
def test_kept_a_bytes_against_the_strips(m, n, N, ctas):
    # every unit's B tile once; an A tile per modulus and distinct tile row of each CTA's strip
    # (a strip of consecutive row-major tiles spans last_row - first_row + 1 tile rows)
    k = 256
    r = I.kept_a_l2_to_sm_bytes(m, n, k, N, ctas)
    tiles_m, tiles_n = -(-m // 128), -(-n // 192)
    T = tiles_m * tiles_n
    rows = 0
    for b in range(ctas):
        s, e = b * T // ctas, (b + 1) * T // ctas
        if e > s:
            rows += (e - 1) // tiles_n - s // tiles_n + 1
    assert r["units"] == N * T
    assert r["a_loads"] == N * rows
    assert r["b"] == N * T * 192 * k * 2 and r["a"] == N * rows * 128 * k * 2
    assert r["total"] <= r["ring"]  # equal when every strip holds one tile per modulus
    if (m, n) == (16384, 16384):
        # the rank-k launch: 96 KB of B per unit, A about once per modulus and CTA strip row
        assert r["b"] == 15 * 11008 * 96 * 1024
        assert r["a"] / r["ring"] < 0.02
