"""Pins of the oracle's learned-start inputs (per-cluster features and
training targets; the learned start is not in the paper, its features are
this project's definition): a hand-built two-super-cluster system whose
values follow from its geometry, invariance under exact scaling, and the
axis features following an exchange of axes."""
import math

import numpy as np

FL = 1e-7 * 8.0   # floor of every length: 1e-7 of the largest box side (8)


def _hand_system():
    """Clusters of M = 4, so a super-cluster holds 32 particles; 39 particles
    give super-cluster 0 (clusters 0..7, full) and super-cluster 1 (cluster 8
    full, cluster 9 with 3 particles, clusters 10..15 empty)."""
    pts = []
    # cluster 0: sides 1, 2, 4
    pts += [(0, 0, 0), (1, 0, 0), (0, 2, 0), (0, 0, 4)]
    # clusters 1..7: a segment of length 0.25 along x starting at 0.5 c
    for c in range(1, 8):
        pts += [(0.5 * c, 0, 0), (0.5 * c + 0.25, 0, 0), (0.5 * c, 0, 0), (0.5 * c, 0, 0)]
    # cluster 8: sides 0.5, 1, 0
    pts += [(6, 6, 6), (6.5, 6, 6), (6, 7, 6), (6, 6, 6)]
    # cluster 9: three coincident particles
    pts += [(7, 7, 7)] * 3
    p = np.array(pts, np.float32)
    box = {"lo": np.zeros(3, np.float32), "hi": np.full(3, 8.0, np.float32),
           "periodic": np.zeros(3, np.int32)}
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), box


def test_features_of_hand_built_system(orc):
    xs, ys, zs, box = _hand_system()
    X, e64 = orc.mlp_features(xs, ys, zs, box, 4)
    assert X.shape == (16, 8) and e64.shape == (2,)
    # super-cluster boxes: [0,3.75]x[0,2]x[0,4] and [6,7]^3; both together [0,7]^3
    assert np.allclose(e64, [4.0, 1.0], rtol=0, atol=1e-12)
    d0 = math.log(4.0 / 8.0) + math.log(39.0) / 3.0
    d1 = math.log(1.0 / 8.0) + math.log(39.0) / 3.0
    want = {
        0: [0.0, math.log(7 / 4), math.log(7 / 4), math.log(1 / 4), math.log(2 / 4), 0.0, 0.0, d0],
        3: [math.log(0.25 / 4), math.log(7 / 4), math.log(7 / 4), 0.0, math.log(FL / 0.25),
            math.log(FL / 0.25), 0.0, d0],
        8: [0.0, math.log(7.0), math.log(7.0), math.log(0.5), 0.0, math.log(FL), 0.0, d1],
        9: [math.log(FL), math.log(7.0), math.log(7.0), 0.0, 0.0, 0.0, math.log(3 / 4), d1],
    }
    for c, row in want.items():
        assert np.allclose(X[c], row, rtol=0, atol=1e-12), (c, X[c], row)
    assert np.all(X[10:] == 0.0)
    # clusters 1..7 are alike
    for c in range(1, 8):
        assert np.allclose(X[c], X[3], rtol=0, atol=1e-12)


def test_targets_of_hand_built_system(orc):
    xs, ys, zs, box = _hand_system()
    X, e64 = orc.mlp_features(xs, ys, zs, box, 4)
    hs = np.ones(39, np.float32)
    hs[0:4] = [1, 2, 3, 4]          # cluster 0: mean 2.5, e64 = 4
    hs[36:39] = [0.5, 1.0, 1.5]     # cluster 9: mean 1.0, e64 = 1
    y, w = orc.mlp_targets(hs, 4, e64)
    assert math.isclose(y[0], math.log(2.5 / 4.0), abs_tol=1e-12)
    assert math.isclose(y[9], 0.0, abs_tol=1e-12)
    assert math.isclose(y[8], math.log(1.0), abs_tol=1e-12)
    assert math.isclose(y[5], math.log(1.0 / 4.0), abs_tol=1e-12)
    assert np.all(w[:10] == 1.0) and np.all(w[10:] == 0.0) and np.all(y[10:] == 0.0)


def _sorted_plummer(orc, n=3000):
    from paper_2602_19873_gb300 import workloads as wl
    d = wl.plummer(n, n_spheres=3, seed=21)
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    p = orc.sort(k)
    return [np.ascontiguousarray(np.asarray(d[a], np.float32)[p]) for a in "xyz"], d["box"]


def test_features_invariant_under_exact_scaling(orc):
    (xs, ys, zs), box = _sorted_plummer(orc)
    X, e64 = orc.mlp_features(xs, ys, zs, box, 8)
    s = np.float32(0.125)   # a power of two: every coordinate scales exactly
    box2 = {"lo": box["lo"] * s, "hi": box["hi"] * s, "periodic": box["periodic"]}
    X2, e2 = orc.mlp_features(xs * s, ys * s, zs * s, box2, 8)
    assert np.allclose(e2, e64 * 0.125, rtol=1e-12, atol=0)
    assert np.allclose(X2, X, rtol=0, atol=1e-9)


def test_axis_features_follow_an_exchange_of_axes(orc):
    (xs, ys, zs), box = _sorted_plummer(orc)
    X, _ = orc.mlp_features(xs, ys, zs, box, 8)
    box2 = {"lo": box["lo"][[1, 0, 2]], "hi": box["hi"][[1, 0, 2]],
            "periodic": box["periodic"][[1, 0, 2]]}
    Y, _ = orc.mlp_features(ys, xs, zs, box2, 8)
    assert np.array_equal(Y[:, [0, 1, 2, 5, 6, 7]], X[:, [0, 1, 2, 5, 6, 7]])
    assert np.array_equal(Y[:, 3], X[:, 4]) and np.array_equal(Y[:, 4], X[:, 3])
    # a partly filled last cluster counts its real particles only
    n = len(xs)
    last = (n - 1) // 8
    assert math.isclose(X[last, 6], math.log((n - 8 * last) / 8.0), abs_tol=1e-12)


def test_region_features_of_a_line_of_super_clusters(orc):
    """Twelve super-clusters of M = 4 (32 particles each) on a line: super-
    cluster s spans x in [s, s + 0.25] at y = z = 0.5.  Its own box is 0.25
    wide; the 8 super-clusters around it are s-3 .. s+4 clipped to 0 .. 11,
    the 64 around it all twelve, so the region features are known by hand."""
    nsc = 12
    j = np.arange(32, dtype=np.float64)
    x = np.concatenate([s + 0.25 * j / 31.0 for s in range(nsc)]).astype(np.float32)
    y = np.full(len(x), 0.5, np.float32)
    box = {"lo": np.zeros(3, np.float32), "hi": np.full(3, 16.0, np.float32),
           "periodic": np.zeros(3, np.int32)}
    X, e64 = orc.mlp_features(x, y, y.copy(), box, 4)
    assert np.allclose(e64, 0.25, rtol=0, atol=1e-12)
    # s: (first, last) super-cluster of the 8 around it
    spans = {0: (0, 4), 1: (0, 5), 3: (0, 7), 4: (1, 8), 6: (3, 10), 8: (5, 11), 10: (7, 11),
             11: (8, 11)}
    for s, (a, b) in spans.items():
        for c in range(8 * s, 8 * s + 8):
            assert abs(X[c, 1] - math.log((b - a + 0.25) / 0.25)) < 1e-12, (s, c)
            assert abs(X[c, 2] - math.log(11.25 / 0.25)) < 1e-12, (s, c)
