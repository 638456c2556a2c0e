"""Pins of the oracle's codec: the dither generator, the fixed-point quantizer (Sec. 3.1
Eq. 3), the dithered store (Sec. 5 Eq. 11) and the bit pack / bit struct placement
(Sec. 7).  CPU only."""
import math

import numpy as np
import pytest

from conftest import read_golden


def test_philox_known_answers(oracle):
    import ctypes as ct
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        assert oracle.philox(vals[0:4], vals[4:6]) == vals[6:10]
        # the generator with a round count (the dither draws take 7) is the same function
        c = (ct.c_uint32 * 4)(*vals[0:4])
        k = (ct.c_uint32 * 2)(*vals[4:6])
        o = (ct.c_uint32 * 4)()
        oracle.lib().or_philox4x32(c, k, 10, o)
        assert list(o) == vals[6:10]


def test_dither_rounds_differ_from_ten(oracle):
    # the dither generator stops after DITHER_ROUNDS = 7 rounds: its blocks differ from the
    # ten-round ones, and consecutive counters give unrelated blocks
    key = [0x01234567, 0x89ABCDEF]
    b7 = [oracle.philox([i, 3, 0, 0], key, rounds=oracle.DITHER_ROUNDS) for i in range(64)]
    b10 = [oracle.philox([i, 3, 0, 0], key) for i in range(64)]
    assert oracle.DITHER_ROUNDS == 7 and all(a != b for a, b in zip(b7, b10))
    bits = np.array([[(w >> k) & 1 for w in blk for k in range(32)] for blk in b7])
    assert abs(bits.mean() - 0.5) < 4 * 0.5 / np.sqrt(bits.size)


def test_dither_draw_counter(oracle):
    # the draw of component c is the 16-bit half c % 2 of word (c // 2) % 4 of the Philox
    # block (slot, step, c // 8, 0) of DITHER_ROUNDS rounds, placed mid-bucket among the
    # 32-bit fractions
    seed = 0x0123456789ABCDEF
    for slot, step, comp in [(0, 0, 0), (5, 7, 3), (123456, 99, 13), (2**31, 2**20, 23), (9, 9, 8)]:
        block = oracle.philox([slot, step, comp // 8, 0], [seed & 0xFFFFFFFF, seed >> 32],
                              rounds=oracle.DITHER_ROUNDS)
        w = block[(comp // 2) % 4]
        q = (w >> 16) if comp % 2 else (w & 0xFFFF)
        assert oracle.dither_draw(seed, slot, step, comp) == (q << 16) | 0x8000


def test_dither_round_up_probability_is_the_fraction(oracle):
    # the probability of rounding up, counted exactly over all 2^16 draws q, equals the
    # fraction rounded to 16 bits (so within 2^-17 of it), Sec. 5 Eq. 11
    for f in [0, 1, 0x7FFF, 0x8000, 0x8001, 0x12345678, 0x80000000, 0xFFFF7FFF, 0xFFFF8000, 0xFFFFFFFF]:
        ups = sum(1 for q in range(1 << 16) if f > ((q << 16) | 0x8000))
        assert abs(ups / 65536.0 - f / 2.0 ** 32) <= 2.0 ** -17 + 1e-15


@pytest.mark.parametrize("bits,frac,lo", [(16, 16, 0.0), (16, 13, -4.0), (12, 9, -4.0),
                                          (21, 21, 0.0), (8, 3, -16.0)])
def test_round_to_nearest_error_bound(oracle, bits, frac, lo):
    # |v - phi^-1(phi(v))| <= Delta / 2 inside the window (Sec. 3.2: the integral limits)
    delta = 2.0 ** -frac
    offset = int(math.floor(lo / delta))
    gen = np.random.default_rng(7)
    top = (offset + 2 ** bits - 1) * delta
    for v in gen.uniform(offset * delta, top, 2000):
        u, fl = oracle.encode(v, bits, frac, offset, dither=False)
        assert fl & 1 == 0
        assert abs(oracle.decode(u, frac, offset) - v) <= 0.5 * delta * (1 + 1e-12)


def test_dithered_error_bound(oracle):
    bits, frac, offset = 16, 13, -4 * 2 ** 13
    delta = 2.0 ** -frac
    gen = np.random.default_rng(8)
    for i, v in enumerate(gen.uniform(-3.9, 3.9, 2000)):
        r = oracle.dither_draw(11, i, 1, 0)
        u, fl = oracle.encode(v, bits, frac, offset, dither=True, r=r)
        assert abs(oracle.decode(u, frac, offset) - v) < delta


def test_decode_is_lossless(oracle):
    # phi^-1(u) = (u + offset) * Delta, exact in FP64 (Sec. 3.1); re-encoding it is exact
    for frac, offset in [(16, 0), (13, -32768), (9, -32768), (21, 0), (-2, 5)]:
        for u in [0, 1, 12345, 65535]:
            v = oracle.decode(u, frac, offset)
            assert v == (u + offset) * 2.0 ** -frac
            assert oracle.encode(v, 16, frac, offset, dither=False)[0] == u
            assert oracle.encode(v, 16, frac, offset, dither=True, r=12345)[0] == u


def test_fig4_correlated_error(oracle):
    # Sec. 5 Fig. 4: +1.4 Delta per frame, round to nearest: -0.4 Delta every frame
    bits, frac, offset = 2, 0, 0
    delta = 1.0
    y = 0.0
    for frame, level, err in read_golden("fig4_correlated_error.txt"):
        u, fl = oracle.encode(y + 1.4 * delta, bits, frac, offset, dither=False)
        assert u == int(level)
        y_new = oracle.decode(u, frac, offset)
        assert abs((y_new - (y + 1.4 * delta)) / delta - float(err)) < 1e-12
        assert fl == 4  # rounded down
        y = y_new
    # the next frame overflows the four levels and saturates
    u, fl = oracle.encode(y + 1.4 * delta, bits, frac, offset, dither=False)
    assert u == 3 and fl & 1


def _single_codec(oracle, bits, frac, offset, seed):
    cd = oracle.Codec()
    cd.n_comp = 1
    cd.n_words = 1
    cd.bits[0] = bits
    cd.frac[0] = frac
    cd.offset[0] = offset
    cd.bitpos[0] = 0
    cd.field[0] = 1
    cd.seed = seed
    cd.dither = 1
    return cd


@pytest.mark.parametrize("Y", [0.3, 0.05, 0.77])
def test_dither_rounds_up_with_probability_Y(oracle, Y):
    # Sec. 5: P(Y + xi > 1/2) = Y, so the dithered store is unbiased; 1e6 draws
    n = 1_000_000
    frac, offset, bits = 10, -512, 12
    v = (37 + Y) * 2.0 ** -frac
    cd = _single_codec(oracle, bits, frac, offset, seed=2024)
    stats = np.zeros(oracle.N_STATS, dtype=np.int64)
    s = np.full((n, 1), v)
    w = oracle.encode_state(cd, s, 3, stats)
    ups = int(stats[4 + 1])
    downs = int(stats[8 + 1])
    assert ups + downs == n
    sigma = math.sqrt(Y * (1 - Y) / n)
    assert abs(ups / n - Y) < 4 * sigma
    err = oracle.decode_state(cd, w)[:, 0] - v
    # mean error is zero within 4 standard errors (the error variance is Y(1-Y) Delta^2)
    assert abs(err.mean()) < 4 * math.sqrt(Y * (1 - Y)) * 2.0 ** -frac / math.sqrt(n)


def test_dither_unbiased_on_uniform_signal(oracle):
    # round-ups / round-downs ~ 1 for dithered stores of a spread signal (Sec. 8.1,
    # Table 4 reports 0.999976); 1e6 draws
    n = 1_000_000
    gen = np.random.default_rng(5)
    s = gen.uniform(-0.4, 0.4, (n, 1))
    cd = _single_codec(oracle, 12, 10, -512, seed=77)
    stats = np.zeros(oracle.N_STATS, dtype=np.int64)
    w = oracle.encode_state(cd, s, 1, stats)
    ups, downs = int(stats[5]), int(stats[9])
    assert abs(ups / downs - 1.0) < 4 * 2 / math.sqrt(n)
    err = oracle.decode_state(cd, w)[:, 0] - s[:, 0]
    assert abs(err.mean()) < 4 * 2.0 ** -10 / math.sqrt(6 * n)


def test_saturation_and_nan(oracle):
    bits, frac, offset = 8, 4, -128  # window [-8, 8)
    assert oracle.encode(100.0, bits, frac, offset)[0] == 255
    assert oracle.encode(100.0, bits, frac, offset)[1] & 1
    assert oracle.encode(-100.0, bits, frac, offset)[0] == 0
    assert oracle.encode(float("nan"), bits, frac, offset) == (0, 1)
    assert oracle.encode(float("inf"), bits, frac, offset)[0] == 255
    # the top level rounds up out of the window -> saturates at the top
    v = (offset + 255 + 0.75) * 2.0 ** -frac
    assert oracle.encode(v, bits, frac, offset) == (255, 1)


def test_fig6_bit_pack_vs_bit_struct(oracle):
    # Sec. 7 Fig. 6: three 17-bit values: 3 words as 32-bit bit structs, 2 as a bit pack.
    for layout, cont, nval, b, words in read_golden("fig6_bitpack.txt"):
        cont, nval, b, words = int(cont), int(nval), int(b), int(words)
        # x is the three-component field (3D); v follows in its own 32-bit container so
        # its first bit marks where x's storage ends
        bits = [b] * 3 + [8] * 3 + [8] * 9 + [8]
        pos, nw = oracle.layout(3, "fluid", bits, (cont, 32, 32, 32))
        assert pos[3] // 32 == words


def test_layout_rules(oracle):
    # x 3 x 21 bits in one 64-bit container
    bits = [21] * 3 + [16] * 3 + [12] * 9 + [16] * 9
    pos, nw = oracle.layout(3, "corotated", bits, (64, 0, 0, 0))
    assert pos[:3] == [0, 21, 42]
    assert pos[3] == 64  # v starts after the 64-bit container
    total = 64 + 3 * 16 + 9 * 12 + 9 * 16
    assert nw == (total + 31) // 32
    # all bit pack: contiguous
    pos, nw = oracle.layout(2, "neohookean", [16] * 12, (0, 0, 0, 0))
    assert pos == [16 * c for c in range(12)] and nw == 6
    # bit struct: a component that does not fit opens the next container
    pos, nw = oracle.layout(2, "fluid", [20, 20, 20, 20, 10, 10, 10, 10, 7], (32, 64, 32, 0))
    assert pos[:2] == [0, 32]
    assert pos[2:4] == [64, 84]
    assert pos[4:8] == [128, 138, 148, 160]
    assert pos[8] == 192 and nw == 7


def test_pack_matches_big_integer(oracle):
    # the record is one little-endian bit string: bit b of the record is bit (b % 32) of
    # word b // 32 (Fig. 7: a value spanning two words is rebuilt from both)
    gen = np.random.default_rng(3)
    for trial in range(200):
        dim = int(gen.choice([2, 3]))
        mat = str(gen.choice(["neohookean", "fluid"]))
        nc = oracle.n_comp(dim, mat)
        bits = [int(b) for b in gen.integers(1, 33, nc)]
        cont = [int(c) for c in gen.choice([0, 32, 64], 4)]
        pos, nw = oracle.layout(dim, mat, bits, cont)
        u = [int(gen.integers(0, 2 ** b)) for b in bits]
        big = 0
        for c in range(nc):
            big |= u[c] << pos[c]
        expect = [(big >> (32 * i)) & 0xFFFFFFFF for i in range(nw)]
        assert oracle.pack(bits, pos, nw, u) == expect
        assert oracle.unpack(bits, pos, expect) == u
        # no two components overlap
        spans = sorted((pos[c], pos[c] + bits[c]) for c in range(nc))
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
