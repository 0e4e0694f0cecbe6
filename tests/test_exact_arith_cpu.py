"""The exact integer arithmetic the residue kernels do in FP32 and with multiply-high quotients,
replayed in numpy with the same operations and roundings, against the definitions: the residue
split's FP32 scheme (four 14-bit pieces, a quotient rounded from 1/p, one centring step), the
kept-A drain's conversion of an FP32 accumulator sum by the 1.5 2^23 magic add, and its exact-floor
residue of sums below 2^22.  The GPU tests compare the kernels' outputs with the oracle; these pin
the bounds the kernels' comments rely on, over every modulus and the ends of each range."""
import numpy as np

MODULI = [255, 254, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]
MAGIC = np.float64(12582912.0)  # 1.5 2^23


def centred(x, p):
    r = np.mod(x, p)
    return np.where(r > (p - 1) // 2, r - p, r)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_product(t, inv32):
    """fmaf(t, inv32, 1.5 2^23) - 1.5 2^23 for integer-valued t, |t| < 2^24: the exact product
    t inv32 rounded once to the nearest integer, ties to even (1.5 2^23 + t inv32 lies in
    [2^23, 2^24), where FP32 steps by 1).  inv32 = M 2^-E with M an integer, so the product is the
    integer t M over 2^E, rounded here in integer arithmetic."""
    mant, exp = np.frexp(np.float64(inv32))
    M, E = int(mant * 2 ** 24), 24 - int(exp)
    num = t.astype(np.int64) * M                     # |num| < 2^48: exact
    q = num >> E                                     # floor
    rem = num - (q << E)
    half = 1 << (E - 1)
    q = q + ((rem > half) | ((rem == half) & ((q & 1) == 1))).astype(np.int64)
    return q.astype(np.float64)


def test_residue_split_fp32_scheme():
    rng = np.random.default_rng(20)
    for bits in (20, 37, 53, 56):
        A = rng.integers(0, 1 << bits, 200_000, dtype=np.uint64)
        A = np.concatenate([A, np.array([0, 1, (1 << bits) - 1, (1 << bits) - 2, 1 << (bits - 1)], dtype=np.uint64)])
        for neg in (False, True):
            pieces = [((A >> np.uint64(14 * j)) & np.uint64(0x3FFF)).astype(np.float64) for j in range(4)]
            if neg:
                pieces = [-a for a in pieces]
            x = -A.astype(np.int64) if neg else A.astype(np.int64)
            for p in MODULI:
                k = [float((1 << (14 * (j + 1))) % p) for j in range(3)]
                # fmaf chain: every partial sum an integer below 2^24 in magnitude, so exact
                t = pieces[0] + pieces[1] * k[0] + pieces[2] * k[1] + pieces[3] * k[2]
                assert np.abs(t).max() < 2 ** 24
                q = round_product(t, np.float32(1.0) / np.float32(p))
                r = t - q * p                        # exact
                assert np.abs(r).max() < p / 2 + 2
                lo, hi = -(p // 2), (p - 1) // 2
                r = np.where(r > hi, r - p, np.where(r < lo, r + p, r))
                assert np.array_equal(r, centred(x, p)), (bits, neg, p)
                # the fp16 code of 1536 + r is the low half of the FP32 bits of 0xC06600 + r
                code = f32(r + 12609024.0).astype(np.float32).view(np.uint32) & 0xFFFF
                assert np.array_equal(code.astype(np.int64), 0x6600 + r.astype(np.int64))


def test_magic_add_conversion_below_2_22():
    x = np.arange(-(1 << 22) + 1, 1 << 22, dtype=np.int64)
    bits = (x.astype(np.float32) + np.float32(12582912.0)).view(np.int32).astype(np.int64)
    assert np.array_equal(bits - 0x4B400000, x)


def test_exact_floor_residue_below_2_22():
    rng = np.random.default_rng(21)
    x = np.concatenate([np.arange(-(1 << 22) + 1, -(1 << 22) + 20_000), np.arange((1 << 22) - 20_000, 1 << 22),
                        np.arange(-20_000, 20_000), rng.integers(-(1 << 22) + 1, 1 << 22, 1_000_000)]).astype(np.int64)
    for p in MODULI:
        magic_up = -(-(1 << 32) // p)          # ceil(2^32 / p)
        off22 = p * (-(-(1 << 22) // p))       # p ceil(2^22 / p)
        assert magic_up < (1 << 32)
        u = (x + off22).astype(np.uint64)
        assert int(u.max()) < (1 << 24) and int(u.min()) >= 0
        q = (u * np.uint64(magic_up)) >> np.uint64(32)   # the multiply-high, no correction
        r = u.astype(np.int64) - (q * np.uint64(p)).astype(np.int64)
        assert np.array_equal(r, np.mod(x, p)), p
