"""Pins of the oracle's neighbor sets and canonical cluster lists."""
import math

import numpy as np
import pytest

from paper_2602_19873_gb300 import workloads as wl


def _small(name, n):
    if name == "uniform":
        return wl.uniform(n, seed=11)
    if name == "evrard":
        return wl.evrard(n, seed=12, n_target=40)
    if name == "lj_fluid":
        d = wl.lj_fluid(n, seed=13)
        return d
    if name == "plummer":
        return wl.plummer(n, n_spheres=4, seed=14, n_target=40)
    if name == "batched_cube":
        d = wl.batched(4, seed=15, log_n=(3.0, 3.3))[0]
        return d
    if name == "batched_plummer":
        return wl.batched(4, seed=15, log_n=(3.0, 3.3))[1]
    raise KeyError(name)


def _sorted(orc, d):
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    p = orc.sort(k)
    return [np.asarray(d[a])[p] for a in ("x", "y", "z", "h", "m")]


def _brute_numpy(xs, ys, zs, hs, box, support, mode):
    """Independent O(n^2) restatement with numpy float32 vector arithmetic."""
    n = len(xs)
    L = (box["hi"] - box["lo"]).astype(np.float32)
    out = []
    r = (np.float32(support) * hs).astype(np.float32)
    for i in range(n):
        d = []
        for a, arr in enumerate((xs, ys, zs)):
            dd = (arr - arr[i]).astype(np.float32)
            if box["periodic"][a]:
                half = np.float32(0.5) * L[a]
                dd = np.where(dd > half, (dd - L[a]).astype(np.float32),
                              np.where(dd < -half, (dd + L[a]).astype(np.float32), dd))
            d.append(dd.astype(np.float32))
        d2 = ((d[0] * d[0]).astype(np.float32) + (d[1] * d[1]).astype(np.float32)).astype(np.float32)
        d2 = (d2 + (d[2] * d[2]).astype(np.float32)).astype(np.float32)
        rr = r if mode == 1 else np.full(n, r[i], np.float32)
        rij = np.maximum(rr, r[i]).astype(np.float32)
        ok = d2 < (rij * rij).astype(np.float32)
        ok[i] = False
        out.append(np.nonzero(ok)[0])
    return out


@pytest.mark.parametrize("name,n", [("uniform", 1500), ("evrard", 1500), ("lj_fluid", 1200),
                                    ("plummer", 2000), ("batched_cube", 1100),
                                    ("batched_plummer", 1100)])
def test_cell_list_matches_brute_force(orc, name, n):
    d = _small(name, n)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    box, sup = d["box"], d["support"]
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, box, sup)
    ref = _brute_numpy(xs, ys, zs, hs, box, sup, 0)
    for i in range(len(xs)):
        assert np.array_equal(g_idx[g_off[i]:g_off[i + 1]], ref[i]), i
    # symmetric sets: union with the transpose == direct max-radius predicate
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    refs = _brute_numpy(xs, ys, zs, hs, box, sup, 1)
    b_off, b_idx = orc.brute_neighbors(xs, ys, zs, hs, box, sup, 1, np.arange(len(xs)))
    for i in range(len(xs)):
        row = p_idx[p_off[i]:p_off[i + 1]]
        assert np.array_equal(row, refs[i]), i
        assert np.array_equal(row, b_idx[b_off[i]:b_off[i + 1]]), i


def test_predicate_bitwise_symmetric(orc):
    d = _small("lj_fluid", 800)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    hs = hs * np.float32(0.3) + np.random.default_rng(0).random(len(hs)).astype(np.float32)
    rng = np.random.default_rng(1)
    for _ in range(3000):
        i, j = (int(v) for v in rng.integers(0, len(xs), 2))
        assert orc.dist2(xs, ys, zs, i, j, d["box"]) == orc.dist2(xs, ys, zs, j, i, d["box"])
        assert orc.pred(xs, ys, zs, hs, 1.0, i, j, d["box"], 1) == \
            orc.pred(xs, ys, zs, hs, 1.0, j, i, d["box"], 1)


def test_mean_count_closed_form(orc):
    """Uniform periodic cube: E[#neighbors] = n * (4/3) pi (2h)^3."""
    d = wl.uniform(20000, seed=21, n_target=60.0)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, _ = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    cnt = np.diff(g_off)
    expect = (len(xs) - 1) * 4.0 / 3.0 * math.pi * (2.0 * float(hs[0])) ** 3
    assert abs(cnt.mean() - expect) < 4.0 * math.sqrt(expect / len(xs)) + 0.05
    # LJ fluid: 100 / nm^3 with rc = 0.9 nm
    f = wl.lj_fluid(27000, seed=22)
    xs, ys, zs, hs, ms = _sorted(orc, f)
    g_off, _ = orc.gather_all(xs, ys, zs, hs, f["box"], 1.0)
    want = 100.0 * 4.0 / 3.0 * math.pi * 0.9 ** 3
    assert abs(np.diff(g_off).mean() - want) / want < 0.02


def _cluster_lists_python(n, M, rows_sym):
    nsc = (n + 8 * M - 1) // (8 * M)
    out = []
    for s in range(nsc):
        m = {}
        for i in range(s * 8 * M, min(n, (s + 1) * 8 * M)):
            k = (i - s * 8 * M) // M
            for j in rows_sym[i]:
                m[j // M] = m.get(j // M, 0) | (1 << k)
        Js = sorted(m)
        out.append((np.array(Js, np.int32), np.array([m[J] for J in Js], np.uint8)))
    return out


@pytest.mark.parametrize("M", [4, 8, 16])
def test_cluster_lists_definition(orc, M):
    d = _small("plummer", 1700)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    refs = _brute_numpy(xs, ys, zs, hs, d["box"], 2.0, 1)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    n = len(xs)
    nsc = (n + 8 * M - 1) // (8 * M)
    o, J, m = orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), np.arange(nsc))
    want = _cluster_lists_python(n, M, refs)
    for s in range(nsc):
        assert np.array_equal(J[o[s]:o[s + 1]], want[s][0])
        assert np.array_equal(m[o[s]:o[s + 1]], want[s][1])
    # sampled super-clusters from sampled rows give the same records
    pick = np.array([0, nsc // 2, nsc - 1])
    rows = np.concatenate([np.arange(s * 8 * M, min(n, (s + 1) * 8 * M)) for s in pick])
    b_off, b_idx = orc.brute_neighbors(xs, ys, zs, hs, d["box"], 2.0, 1, rows)
    o2, J2, m2 = orc.cluster_lists(n, M, b_off, b_idx, rows, pick)
    for t, s in enumerate(pick):
        assert np.array_equal(J2[o2[t]:o2[t + 1]], want[s][0])
        assert np.array_equal(m2[o2[t]:o2[t + 1]], want[s][1])


def test_self_tile_and_isolated_particle(orc):
    """The own cluster appears iff a pair inside it passes; an isolated
    particle has no neighbors (i = j is never a pair)."""
    x = np.array([0.1, 0.1001, 0.9, 0.5], np.float32)
    y = np.array([0.1, 0.1, 0.9, 0.5], np.float32)
    z = np.array([0.1, 0.1, 0.9, 0.5], np.float32)
    h = np.array([0.01, 0.01, 0.01, 0.01], np.float32)
    box = {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32), "periodic": np.zeros(3, np.int32)}
    g_off, g_idx = orc.gather_all(x, y, z, h, box, 2.0)
    assert g_idx.tolist() == [1, 0]
    o, J, m = orc.cluster_lists(4, 4, g_off, g_idx, np.arange(4), np.arange(1))
    assert J.tolist() == [0] and m.tolist() == [1]


@pytest.mark.parametrize("M,MJ", [(8, 4), (16, 8)])
def test_cluster_lists_with_half_j_clusters(orc, M, MJ):
    """j-clusters of half the i-cluster size: J counts j-clusters, masks
    still mark the 8 i-clusters of the super-cluster."""
    d = _small("evrard", 1500)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    refs = _brute_numpy(xs, ys, zs, hs, d["box"], 2.0, 1)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    n = len(xs)
    nsc = (n + 8 * M - 1) // (8 * M)
    o, J, m = orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), np.arange(nsc), jcluster=MJ)
    for s in range(nsc):
        want = {}
        for i in range(s * 8 * M, min(n, (s + 1) * 8 * M)):
            for j in refs[i]:
                want[j // MJ] = want.get(j // MJ, 0) | (1 << ((i - s * 8 * M) // M))
        Js = sorted(want)
        assert J[o[s]:o[s + 1]].tolist() == Js
        assert m[o[s]:o[s + 1]].tolist() == [want[x] for x in Js]


def _tiles(o, J, m, sc_ids):
    out = set()
    for t, s in enumerate(sc_ids):
        for J_, mk in zip(J[o[t]:o[t + 1]], m[o[t]:o[t + 1]]):
            for k in range(8):
                if (int(mk) >> k) & 1:
                    out.add((8 * int(s) + k, int(J_)))
    return out


@pytest.mark.parametrize("M", [4, 8])
@pytest.mark.parametrize("name", ["plummer", "uniform"])
def test_half_lists_store_every_cluster_pair_once(orc, name, M):
    """The half list with its transposes is the full list; a pair of clusters
    of different super-clusters is stored exactly once, by the lower one; the
    super-cluster's own clusters keep both orders."""
    d = _small(name, 1900)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    n = len(xs)
    nsc = (n + 8 * M - 1) // (8 * M)
    sc = np.arange(nsc)
    full = _tiles(*orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), sc), sc)
    o, J, m = orc.half_lists(*orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), sc), sc)
    half = _tiles(o, J, m, sc)
    assert half | {(b, a) for a, b in half} == full
    for (a, b) in full:
        if a // 8 != b // 8:
            assert ((a, b) in half) != ((b, a) in half)
            assert ((a, b) in half) == (b // 8 > a // 8)
        else:
            assert (a, b) in half
    # records stay ascending and carry no empty masks
    for s in sc:
        Js = J[o[s]:o[s + 1]]
        assert np.all(np.diff(Js) > 0) and np.all(Js >= 8 * s)
        assert np.all(m[o[s]:o[s + 1]] != 0)
    assert len(J) < len(orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), sc)[1])


@pytest.mark.parametrize("name", ["uniform", "plummer"])
def test_nearest_distance_against_kd_tree(orc, name):
    """The nearest member of each gather set against scipy's k-d tree (its
    periodic box for the cube): the nearest other particle, if it lies inside
    the radius, else +inf (radius ties within 1e-6 skipped)."""
    from scipy.spatial import cKDTree
    d = _small(name, 3000)
    xs, ys, zs, hs0, ms = _sorted(orc, d)
    # every third particle with a radius too small to hold a neighbor
    hs = np.where(np.arange(len(xs)) % 3 == 0, hs0 * np.float32(0.02), hs0).astype(np.float32)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    got = orc.nearest(xs, ys, zs, d["box"], g_off, g_idx)
    P = np.stack([xs, ys, zs], 1).astype(np.float64)
    if np.any(d["box"]["periodic"]):
        L = float(np.float32(d["box"]["hi"][0]) - np.float32(d["box"]["lo"][0]))
        tree = cKDTree(P - np.asarray(d["box"]["lo"], np.float64), boxsize=L)
        dist, _ = tree.query(P - np.asarray(d["box"]["lo"], np.float64), k=2)
    else:
        tree = cKDTree(P)
        dist, _ = tree.query(P, k=2)
    d1 = dist[:, 1]
    r = 2.0 * hs.astype(np.float64)
    clear = np.abs(d1 - r) > 1e-6 * r
    inside = clear & (d1 < r)
    assert np.allclose(got[inside], d1[inside], rtol=1e-12, atol=0)
    assert np.all(np.isinf(got[clear & (d1 >= r)]))
    assert inside.sum() > 0.5 * len(xs) and (clear & (d1 >= r)).sum() > 0.2 * len(xs)
