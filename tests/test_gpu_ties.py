"""Pairs exactly on the radius decide like the canonical FP32 predicate.

Isolated particle pairs, far apart from each other, get radii picked in
float32 so that the pair's canonical squared distance, ((dx^2 + dy^2) + dz^2)
with every operation rounded to nearest, equals r^2 exactly (not a neighbor:
the predicate is d2 < r^2) or so that r is one float above such a tie (a
neighbor).  A kernel that rounds any step of the distance differently, for
example by contracting a product and a sum into a fused multiply-add,
decides a share of these pairs the other way, and the tile of such a pair is
then listed (or dropped) although no other pair of that tile is in range.
Records (full and half lists, compressed and raw) must equal the oracle's
byte for byte, and the neighbor counts must equal the oracle's."""
import numpy as np
import pytest

from nlcheck import compare_records, full_reference, gpu_build, gpu_counts, oracle_sorted

F = np.float32


def _canonical_d2(xi, yi, zi, xj, yj, zj):
    dx, dy, dz = F(xj - xi), F(yj - yi), F(zj - zi)
    return F(F(F(dx * dx) + F(dy * dy)) + F(dz * dz))


def tie_pairs(n_pairs=3000, grid=15, seed=7):
    """Particle pairs in separate unit cells of a grid^3 box; returns the
    system (support 2, so r = 2h exactly) and which pairs are ties."""
    rng = np.random.default_rng(seed)
    cells = rng.choice(grid ** 3, size=n_pairs, replace=False)
    c = np.stack([cells % grid, (cells // grid) % grid, cells // (grid * grid)], 1).astype(np.float64)
    xi = (c + 0.3 + 0.4 * rng.random((n_pairs, 3))).astype(F)
    u = rng.normal(size=(n_pairs, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    xj = (xi.astype(np.float64) + u * (0.05 + 0.05 * rng.random((n_pairs, 1)))).astype(F)
    r = np.zeros(n_pairs, F)
    tie = np.zeros(n_pairs, bool)
    for p in range(n_pairs):
        d2 = _canonical_d2(*xi[p], *xj[p])
        r0 = F(np.sqrt(np.float64(d2)))
        cand = [r0]
        for _ in range(4):
            cand.append(np.nextafter(cand[-1], F(np.inf)))
            cand.insert(0, np.nextafter(cand[0], F(0)))
        exact = [v for v in cand if F(v * v) == d2]
        if exact:
            t = exact[0]
            if p % 2 == 0:
                r[p], tie[p] = t, True                       # d2 == r^2: not a neighbor
            else:
                r[p] = np.nextafter(t, F(np.inf))            # one float above the tie
        else:
            r[p] = min(v for v in cand if F(v * v) > d2)     # smallest radius in range
    x = np.empty(2 * n_pairs, F); y = np.empty_like(x); z = np.empty_like(x); h = np.empty_like(x)
    x[0::2], y[0::2], z[0::2] = xi[:, 0], xi[:, 1], xi[:, 2]
    x[1::2], y[1::2], z[1::2] = xj[:, 0], xj[:, 1], xj[:, 2]
    h[0::2] = h[1::2] = F(0.5) * r
    box = {"lo": np.zeros(3, F), "hi": np.full(3, grid, F), "periodic": np.zeros(3, np.int32)}
    d = {"x": x, "y": y, "z": z, "h": h, "m": np.ones(2 * n_pairs, F), "box": box,
         "kind": 1, "support": 2.0}
    return d, tie


def test_tie_construction_is_exact():
    d, tie = tie_pairs(n_pairs=400)
    assert tie.sum() > 50
    for p in np.nonzero(tie)[0][:50]:
        d2 = _canonical_d2(d["x"][2 * p], d["y"][2 * p], d["z"][2 * p],
                           d["x"][2 * p + 1], d["y"][2 * p + 1], d["z"][2 * p + 1])
        r = F(F(2.0) * d["h"][2 * p])
        assert F(r * r) == d2


def test_oracle_decides_the_constructed_ties():
    d, tie = tie_pairs(n_pairs=400)
    o = oracle_sorted(d)
    g_off = full_reference(o, d)[0]
    cc = np.empty(len(o["xs"]), np.int64)
    cc[o["perm"]] = np.diff(g_off)
    assert (cc[0::2][tie] == 0).all() and (cc[1::2][tie] == 0).all()
    assert (cc[0::2][~tie] == 1).all() and (cc[1::2][~tie] == 1).all()


@pytest.mark.gpu
@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("compress", [1, 0])
def test_records_and_counts_on_exact_ties(half, compress):
    d, tie = tie_pairs()
    o = oracle_sorted(d)
    g_off, g_idx, p_off, p_idx = full_reference(o, d)
    n = len(o["xs"])
    cnt_want = np.diff(g_off)
    L, t = gpu_build(d, cluster=8, compress=compress, half_list=half)
    nsc = L.sizes()["n_superclusters"]
    compare_records(L, o, d, 8, compress, np.arange(nsc), np.arange(n), p_off, p_idx,
                    jcluster=8, half=bool(half))
    cnt = gpu_counts(L, n)[o["perm"]]
    assert np.array_equal(cnt, cnt_want)
    L.free()
