"""Pins of the oracle's nibble codec (paper Sec. II-B, Tables 1 and 2)."""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append([c.strip() for c in line.split("|")])
    return out


def test_table1_worked_examples(orc):
    rows = _rows("table1_codec.txt")
    assert len(rows) == 3
    for diffs, printed_mask, info, data in rows:
        d = [int(v) for v in diffs.split(",")]
        mask, inf, dat = orc.encode_block(d)
        # the table prints element 0 leftmost: bit k of the integer mask is
        # character k of the printed string
        assert "".join("1" if (mask >> k) & 1 else "0" for k in range(6)) == printed_mask
        want_info = [] if info == "-" else [int(c, 16) for c in info]
        want_data = [] if data == "-" else [int(c, 16) for c in data]
        assert list(inf) == want_info
        assert list(dat) == want_data


def _bits_one_value(orc, v):
    # one value in a block of w=32 costs one mask bit plus 4 bits per nibble
    mask, inf, dat = orc.encode_block([v])
    return 1 + 4 * (len(inf) + len(dat))


def test_table2_required_bits(orc):
    for lo, hi, bits in _rows("table2_bits.txt"):
        lo, hi, bits = int(lo), int(hi), int(bits)
        for v in {lo, hi, (lo + hi) // 2}:
            assert _bits_one_value(orc, v) == bits, (v, bits)


def test_stream_size_closed_form(orc):
    """Encoded stream length equals the Table-2 sum plus 32-bit masks."""
    rng = np.random.default_rng(7)
    table = [(int(a), int(b), int(c)) for a, b, c in _rows("table2_bits.txt")]

    def bits(v):
        for lo, hi, b in table:
            if lo <= v <= hi:
                return b
        raise AssertionError(v)

    for trial in range(50):
        cnt = int(rng.integers(1, 200))
        gaps = np.where(rng.random(cnt) < 0.6, 1,
                        rng.integers(2, 1 << int(rng.integers(2, 28)), cnt))
        J = np.cumsum(gaps) - 1
        J = J.astype(np.int64)
        if J[-1] >= 2 ** 31:
            continue
        d = np.diff(np.concatenate([[-1], J]))
        nblocks = (cnt + 31) // 32
        want_bits = sum(bits(int(v)) for v in d) - cnt + 32 * nblocks
        assert want_bits % 4 == 0
        assert orc.stream_nibbles(J.astype(np.int32)) == want_bits // 4


def test_record_round_trip_and_layout(orc):
    rng = np.random.default_rng(3)
    for compress in (True, False):
        for cnt in [0, 1, 5, 31, 32, 33, 64, 100, 257]:
            gaps = np.where(rng.random(cnt) < 0.5, 1, rng.integers(1, 70000, cnt))
            J = (np.cumsum(gaps) - 1).astype(np.int32)
            m = rng.integers(1, 256, cnt).astype(np.uint8)
            rec = orc.encode_record(J, m, 32, compress)
            assert len(rec) % 4 == 0
            assert int(rec[:4].view(np.uint32)[0]) == cnt
            assert np.array_equal(rec[4:4 + cnt], m)
            assert not rec[4 + cnt:4 + ((cnt + 3) & ~3)].any()
            J2, m2 = orc.decode_record(rec, 32, compress)
            assert np.array_equal(J2, J) and np.array_equal(m2, m)
            if not compress:
                body = rec[4 + ((cnt + 3) & ~3):].view(np.uint32)
                assert np.array_equal(body[:cnt], J.astype(np.uint32))


def test_first_block_hand_encoded(orc):
    """A w=32 record checked nibble by nibble against a hand derivation."""
    J = np.array([0, 1, 2, 5, 20, 21, 300], np.int32)   # diffs 1,1,1,3,15,1,279
    m = np.full(7, 0xFF, np.uint8)
    rec = orc.encode_record(J, m, 32, True)
    body = rec[12:]
    nib = []
    for b in body:
        nib += [int(b) & 0xF, int(b) >> 4]
    mask = 0b1011000  # lanes 3, 4, 6 are non-ones
    want = [(mask >> (4 * t)) & 0xF for t in range(8)]
    want += [3 + 6, 0, 2]          # info: 3 -> 9; 15 -> one nibble; 279 -> three
    want += [0xF, 0x1, 0x1, 0x7]   # data: F then 117 (MSB first)
    assert nib[:len(want)] == want
    assert all(v == 0 for v in nib[len(want):])


def test_uncompressed_is_larger_at_typical_gaps(orc):
    rng = np.random.default_rng(11)
    gaps = np.where(rng.random(150) < 0.6, 1, rng.integers(2, 40, 150))
    J = (np.cumsum(gaps) - 1).astype(np.int32)
    assert orc.record_bytes(J, 32, True) < orc.record_bytes(J, 32, False) / 2
