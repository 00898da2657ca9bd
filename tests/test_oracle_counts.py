"""Pins of two oracle quantities built on the neighbor sets.

* ``h_at_count``: smoothing lengths with exactly k gather neighbors (the
  centre of the h iteration's window): every particle's brute-force count is
  k, and scipy's k-d tree puts the k-th neighbor inside and the (k+1)-th
  outside the radius.
* ``computed_pairs`` / ``cluster_overhead`` (Sec. III-A): closed forms for
  1x1 clusters (the list is the pair list itself), for particles all within
  range of each other (every tile fully listed) and for isolated clusters
  (only the own tiles)."""
import numpy as np
import pytest

from paper_2602_19873_gb300 import workloads as wl


def _sorted(orc, d):
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    p = orc.sort(k)
    return k[p], [np.ascontiguousarray(np.asarray(d[a], np.float32)[p]) for a in "xyzhm"]


@pytest.mark.parametrize("name,k", [("uniform", 40), ("plummer", 60), ("evrard", 30)])
def test_h_at_count_has_exactly_k_neighbors(orc, name, k):
    d = {"uniform": lambda: wl.uniform(4000, seed=31),
         "plummer": lambda: wl.plummer(5000, n_spheres=3, seed=32),
         "evrard": lambda: wl.evrard(3000, seed=33)}[name]()
    keys, (xs, ys, zs, hs, ms) = _sorted(orc, d)
    h = orc.h_at_count(xs, ys, zs, keys, d["box"], 2.0, k)
    cnt = orc.gather_counts_brute(xs, ys, zs, h, d["box"], 2.0, np.arange(len(xs)))
    assert np.all(cnt == k), np.unique(cnt)
    # scipy's k-d tree (periodic boxes through boxsize) brackets the radius
    spatial = pytest.importorskip("scipy.spatial")
    pts = np.stack([xs, ys, zs], 1).astype(np.float64)
    per = bool(np.any(d["box"]["periodic"]))
    if per:
        lo = np.asarray(d["box"]["lo"], np.float64)
        pts = pts - lo
        tree = spatial.cKDTree(pts, boxsize=np.asarray(d["box"]["hi"], np.float64) - lo)
    else:
        tree = spatial.cKDTree(pts)
    dist, _ = tree.query(pts, k + 2)        # column 0 is the particle itself
    r = 2.0 * h.astype(np.float64)
    assert np.all(dist[:, k] < r * (1 + 1e-5)) and np.all(dist[:, k + 1] > r * (1 - 1e-5))


def test_computed_pairs_of_one_particle_clusters_is_the_pair_count(orc):
    d = wl.plummer(2500, n_spheres=2, seed=34, n_target=30)
    keys, (xs, ys, zs, hs, ms) = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    n = len(xs)
    nsc = (n + 7) // 8
    o, J, m = orc.cluster_lists(n, 1, p_off, p_idx, np.arange(n), np.arange(nsc))
    assert orc.computed_pairs(m, 1) == int(p_off[-1])


@pytest.mark.parametrize("M,MJ", [(8, 8), (8, 4), (4, 4)])
def test_computed_pairs_all_in_range_and_isolated(orc, M, MJ):
    rng = np.random.default_rng(35)
    box = {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
           "periodic": np.zeros(3, np.int32)}
    # all within range of each other: n a multiple of 8M, every tile listed
    n = 8 * M * 3
    x, y, z = (rng.uniform(0.4, 0.41, n).astype(np.float32) for _ in range(3))
    h = np.full(n, 0.5, np.float32)
    g_off, g_idx = orc.gather_all(x, y, z, h, box, 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    assert p_off[-1] == n * (n - 1)
    o, J, m = orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), np.arange(n // (8 * M)),
                                jcluster=MJ)
    assert orc.computed_pairs(m, M, MJ) == n * n
    assert orc.cluster_overhead(m, M, int(p_off[-1]), n, MJ) == 1.0
    # isolated i-clusters (each a tight group far from the others): own tiles only
    ncl = 8 * 2
    centres = rng.permutation(ncl) * (1.0 / ncl) + 0.5 / ncl
    x = np.repeat(centres, M).astype(np.float32)
    x += np.tile(np.arange(M, dtype=np.float32) * 1e-4, ncl)
    y = np.full(len(x), 0.5, np.float32)
    z = np.full(len(x), 0.5, np.float32)
    h = np.full(len(x), 0.01, np.float32)
    n = len(x)
    g_off, g_idx = orc.gather_all(x, y, z, h, box, 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    assert p_off[-1] == ncl * M * (M - 1)
    o, J, m = orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), np.arange(n // (8 * M)),
                                jcluster=MJ)
    assert orc.computed_pairs(m, M, MJ) == ncl * M * M
    assert abs(orc.cluster_overhead(m, M, int(p_off[-1]), n, MJ) - 1.0) < 1e-15
