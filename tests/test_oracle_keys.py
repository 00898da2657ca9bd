"""Pins of the oracle's SFC keys, sort and octree (paper Sec. II-A)."""
import itertools

import numpy as np
import pytest

from paper_2602_19873_gb300 import workloads as wl


def test_quantize_special_values(orc):
    assert orc.quantize(0.0, 0.0, 1.0) == 0
    assert orc.quantize(1.0, 0.0, 1.0) == 2 ** 21 - 1          # upper face clamps
    for k in [1, 2, 3, 1000, 2 ** 20, 2 ** 21 - 2]:
        x = k / 2.0 ** 21                                        # exactly representable
        assert orc.quantize(x, 0.0, 1.0) == k
        assert orc.quantize(np.nextafter(np.float32(x), np.float32(0)), 0.0, 1.0) == k - 1
    # shifted box: lo = -1, hi = 1 -> cell width 2^-20
    assert orc.quantize(-1.0, -1.0, 1.0) == 0
    assert orc.quantize(0.0, -1.0, 1.0) == 2 ** 20


def test_morton_closed_form(orc):
    assert orc.morton3(1, 0, 0) == 4
    assert orc.morton3(0, 1, 0) == 2
    assert orc.morton3(0, 0, 1) == 1
    assert orc.morton3(2, 0, 0) == 32
    full = 2 ** 21 - 1
    assert orc.morton3(full, full, full) == 2 ** 63 - 1
    assert orc.morton3(full, 0, 0) == int("100" * 21, 2)
    rng = np.random.default_rng(0)
    for _ in range(200):
        q = [int(v) for v in rng.integers(0, 2 ** 21, 3)]
        k = orc.morton3(*q)
        for a in range(3):
            got = sum(((k >> (3 * b + 2 - a)) & 1) << b for b in range(21))
            assert got == q[a]


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_bijection_and_adjacency(orc, bits):
    side = 1 << bits
    seen = {}
    for q in itertools.product(range(side), repeat=3):
        k = orc.hilbert3(*q, bits=bits)
        assert 0 <= k < side ** 3
        seen[k] = q
    assert len(seen) == side ** 3
    assert seen[0] == (0, 0, 0)                     # the curve starts at the origin
    for k in range(side ** 3 - 1):
        a, b = np.array(seen[k]), np.array(seen[k + 1])
        assert np.abs(a - b).sum() == 1, (k, seen[k], seen[k + 1])


def test_hilbert_21bit_sub_curve_and_roundtrip(orc):
    # the 21-bit curve restricted to [0, 2^k)^3 is a curve over [0, 8^k)
    for q in itertools.product(range(4), repeat=3):
        assert orc.hilbert3(*q, bits=21) < 64
    rng = np.random.default_rng(1)
    for _ in range(300):
        q = tuple(int(v) for v in rng.integers(0, 2 ** 21, 3))
        k = orc.hilbert3(*q, bits=21)
        assert k < 2 ** 63
        assert orc.hilbert3_inverse(k, 21) == q
        # neighbours along the curve are face neighbours on the 21-bit grid
        if k + 1 < 2 ** 63:
            a = np.array(orc.hilbert3_inverse(k + 1, 21), dtype=np.int64)
            assert np.abs(a - np.array(q, dtype=np.int64)).sum() == 1


def test_keys_match_scalar_definitions(orc):
    d = wl.uniform(2000, seed=5)
    for kind in (0, 1):
        k = orc.keys(d["x"], d["y"], d["z"], d["box"], kind)
        for i in range(0, 2000, 97):
            q = [orc.quantize(d[a][i], 0.0, 1.0) for a in "xyz"]
            want = orc.morton3(*q) if kind == 0 else orc.hilbert3(*q)
            assert int(k[i]) == want


def test_sort_is_stable_by_original_index(orc):
    rng = np.random.default_rng(2)
    k = rng.integers(0, 50, 5000).astype(np.uint64)     # many equal keys
    perm = orc.sort(k)
    assert np.array_equal(perm, np.argsort(k, kind="stable"))


def test_hilbert_locality_on_points(orc):
    """Consecutive SFC particles are close on average (Sec. II-A premise)."""
    d = wl.uniform(20000, seed=9)
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], 1)
    p = orc.sort(k)
    xyz = np.stack([d["x"][p], d["y"][p], d["z"][p]], 1).astype(np.float64)
    step = np.linalg.norm(np.diff(xyz, axis=0), axis=1)
    spacing = (1.0 / 20000) ** (1 / 3)
    assert np.median(step) < 2.0 * spacing
    rnd = np.linalg.norm(xyz[1:] - xyz[np.random.default_rng(0).permutation(20000)[1:]], axis=1)
    assert np.mean(step) < 0.1 * np.mean(rnd)


def _octree_python(keys, bucket):
    out = []

    def rec(level, a, b):
        leaf = (b - a <= bucket) or level == 21
        out.append((level, a, b, leaf))
        if leaf:
            return
        shift = 63 - 3 * (level + 1)
        s = a
        while s < b:
            c = int(keys[s]) >> shift
            e = s
            while e < b and (int(keys[e]) >> shift) == c:
                e += 1
            rec(level + 1, s, e)
            s = e
    if len(keys):
        rec(0, 0, len(keys))
    return out


@pytest.mark.parametrize("n,bucket", [(1, 4), (7, 8), (500, 8), (3000, 16), (3000, 64)])
def test_octree_definition(orc, n, bucket):
    d = wl.plummer(n, n_spheres=1, seed=n)
    k = np.sort(orc.keys(d["x"], d["y"], d["z"], d["box"], 1))
    t = orc.octree(k, bucket)
    ref = _octree_python(k, bucket)
    got = list(zip(t["level"].tolist(), t["first"].tolist(), t["end"].tolist(), t["leaf"].tolist()))
    assert got == ref
    leaves = [(l, a, b) for l, a, b, f in got if f]
    # leaves tile [0, n) in order; every non-level-21 leaf holds <= bucket
    assert leaves[0][1] == 0 and leaves[-1][2] == n
    for (l0, a0, b0), (l1, a1, b1) in zip(leaves, leaves[1:]):
        assert b0 == a1
    for l, a, b in leaves:
        assert b - a <= bucket or l == 21
        pref = int(k[a]) >> (63 - 3 * l) if l else 0
        assert all((int(v) >> (63 - 3 * l) if l else 0) == pref for v in k[a:b])


def test_octree_duplicate_keys_cap_at_level_21(orc):
    k = np.array([5] * 40 + [6] * 3, np.uint64)
    t = orc.octree(k, 8)
    leaves = [(int(l), int(a), int(b)) for l, a, b, f in
              zip(t["level"], t["first"], t["end"], t["leaf"]) if f]
    assert leaves == [(21, 0, 40), (21, 40, 43)]

