"""Pins of the oracle's data-translation step (codes -> levels) against
exhaustive hand-written code tables and hand-packed words."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

# level of every code, written out (reading: b < 8 -> 2c - (2^b - 1); b = 8 -> int8)
TABLE = {
    1: [-1, 1],
    2: [-3, -1, 1, 3],
    4: [-15, -13, -11, -9, -7, -5, -3, -1, 1, 3, 5, 7, 9, 11, 13, 15],
    8: list(range(0, 128)) + list(range(-128, 0)),
}


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_every_code(orc, bits):
    codes = np.arange(1 << bits)
    reps = max(1, (32 // bits) // len(codes))
    codes = np.tile(codes, reps)
    n = len(codes) - len(codes) % (32 // bits)
    words = synth.pack(codes[:n], bits)
    got = orc.decode(bits, words, n)
    want = np.array(TABLE[bits] * reps, dtype=np.float64)[:n]
    assert np.array_equal(got, want)


def test_int8_matches_twos_complement_view(orc):
    b = np.arange(256, dtype=np.uint8)
    words = b.view(np.uint32)  # little-endian bytes, sample j in bits [8j, 8j+8)
    assert np.array_equal(orc.decode(8, words, 256), b.view(np.int8).astype(np.float64))


def test_bit_order_hand_packed(orc):
    # 2-bit: 0xE4 = 11 10 01 00b -> samples 0..3 are codes 0,1,2,3 (LSB first)
    assert list(orc.decode(2, np.array([0x000000E4], np.uint32), 16)[:5]) == [-3, -1, 1, 3, -3]
    # 8-bit: bytes LSB first 0x7F, 0x01, 0xFF, 0x80
    assert list(orc.decode(8, np.array([0x80FF017F], np.uint32), 4)) == [127, 1, -1, -128]
    # 4-bit: nibbles LSB first F, 0, 1, F, 0...
    assert list(orc.decode(4, np.array([0x0000F10F], np.uint32), 5)) == [15, -15, -13, 15, -15]
    # 1-bit: 0b0101 -> +1, -1, +1, -1
    assert list(orc.decode(1, np.array([0x5], np.uint32), 5)) == [1, -1, 1, -1, -1]


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_random_codes_roundtrip(orc, bits):
    rng = np.random.default_rng(bits)
    n = 4096
    codes = synth.random_codes(rng, n, bits)
    got = orc.decode(bits, synth.pack(codes, bits), n)
    assert np.array_equal(got, np.array(TABLE[bits], dtype=np.float64)[codes.astype(np.int64)])
