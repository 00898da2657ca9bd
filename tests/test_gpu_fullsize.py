"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (8x8 clusters, compressed list, leaf bucket 256).

The oracle sorts all particles itself and computes, by O(n) brute force per
particle, the symmetric neighbor sets of a sample of whole super-clusters:
their records must match the GPU's byte for byte, and the density / forces /
counts of their particles must match within the tolerances of the small-size
tests.  Smoothing lengths are either the generators' or, for the converged
configurations (200 neighbors on the Plummer mixture and the Evrard sphere,
100 on the batched systems), the oracle's own: halfway between each
particle's 200th and 201st (100th and 101st) neighbor, so every particle has
exactly that many gather neighbors.  The GPU's own h iteration is checked by
the window property on sampled particles."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import DENSITY_RTOL, compare_records, gpu_build, gpu_counts, gpu_density, oracle_sorted

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5


def _sample_sc(nsc, seed, k=6):
    rng = np.random.default_rng(seed)
    pick = {0, nsc - 1, nsc // 2}
    pick |= set(int(v) for v in rng.integers(0, nsc, k - len(pick)))
    return np.array(sorted(pick), np.int64)


def _rows(sc, n, M=8):
    return np.concatenate([np.arange(s * 8 * M, min(n, (s + 1) * 8 * M)) for s in sc])


def _check_sampled(d, name, with_density=True, o=None):
    o = oracle_sorted(d) if o is None else o
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=8, compress=1, bucket=256)
    nsc = L.sizes()["n_superclusters"]
    sc = _sample_sc(nsc, seed=n % 1000)
    rows = _rows(sc, n)
    p_off, p_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"],
                                       d["support"], 1, rows)
    compare_records(L, o, d, 8, 1, sc, rows, p_off, p_idx)
    g_off, g_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"],
                                       d["support"], 0, rows)
    cnt = gpu_counts(L, n)[o["perm"]]
    assert np.array_equal(cnt[rows], np.diff(g_off)), name
    if with_density:
        rho = gpu_density(L, t, n)[o["perm"]]
        want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                           rows)
        rel = np.abs(rho[rows] - want) / want
        assert rel.max() <= DENSITY_RTOL, (name, rel.max())
    return L, t, o, rows, g_off, g_idx


def test_uniform_periodic_32k_full():
    """The small configuration: every record, count and density exact."""
    d = wl.config("uniform_periodic_32k")
    o = oracle_sorted(d)
    n = len(o["xs"])
    g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], d["support"])
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    L, t = gpu_build(d)
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, 8, 1, np.arange(nsc), np.arange(n), p_off, p_idx)
    assert L.sizes()["list_bytes"] == total
    # O(n^2) brute force agrees with the cell list on a sample
    b_off, b_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0, 0,
                                       np.arange(0, n, 97))
    for q, i in enumerate(range(0, n, 97)):
        assert np.array_equal(b_idx[b_off[q]:b_off[q + 1]], g_idx[g_off[i]:g_off[i + 1]])
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    assert (np.abs(rho - want) / want).max() <= DENSITY_RTOL
    assert np.array_equal(gpu_counts(L, n)[o["perm"]], np.diff(g_off))
    # the paper's mean count: n (4/3) pi (2h)^3 ~ 100
    assert abs(np.diff(g_off).mean() - 100.0) < 1.0
    L.free()


def test_evrard_2m_sampled():
    d = wl.cached(wl.evrard, "evrard_%d_2" % (1 << 21), 1 << 21, seed=2)
    L, t, o, rows, g_off, g_idx = _check_sampled(d, "evrard_2m")
    L.free()


def test_lj_fluid_4m_sampled_with_forces():
    import torch
    d = wl.cached(wl.lj_fluid, "lj_fluid_4000000_3", 4_000_000, seed=3)
    L, t, o, rows, g_off, g_idx = _check_sampled(d, "lj_fluid_4m", with_density=False)
    n = len(o["xs"])
    fx, fy, fz, fa = orc.lj_force(o["xs"], o["ys"], o["zs"], d["box"], 1.0, 0.3, g_off, g_idx,
                                  rows)
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_LJ, *out, eps=1.0, sigma=0.3)
    torch.cuda.synchronize()
    got = np.stack([a.cpu().numpy()[o["perm"]][rows] for a in out], 1)
    err = np.linalg.norm(got - np.stack([fx, fy, fz], 1), axis=1) / fa
    assert err.max() <= FORCE_RTOL, err.max()
    # about 305 neighbors at 100 / nm^3 within 0.9 nm
    assert abs(np.diff(g_off).mean() - 305.4) < 15.0
    L.free()


@pytest.fixture(scope="module")
def plummer16m():
    """The benchmark's 2^24-particle system and the oracle's sort of it."""
    d = wl.cached(wl.plummer, "plummer64_%d_4" % (1 << 24), 1 << 24, n_spheres=64, seed=4)
    return d, oracle_sorted(d)


def _at_count(d, o, k):
    """Copies of (d, o) with the oracle's smoothing lengths at exactly k
    gather neighbors (sorted and caller order)."""
    hs = orc.h_at_count(o["xs"], o["ys"], o["zs"], o["keys"], d["box"], d["support"], k)
    h = np.empty_like(hs)
    h[o["perm"]] = hs
    d2, o2 = dict(d), dict(o)
    d2["h"], o2["hs"] = h, hs
    return d2, o2


def _check_half_list(d, o, name, k):
    """Half list (the benchmark's storage): sampled records byte-exact
    against the oracle's half lists, counts exact (k for every particle of
    the sample, within the window for all), density within tolerance."""
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=8, compress=1, bucket=256, half_list=1)
    nsc = L.sizes()["n_superclusters"]
    sc = _sample_sc(nsc, seed=n % 997, k=8)
    rows = _rows(sc, n)
    p_off, p_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"],
                                       d["support"], 1, rows)
    compare_records(L, o, d, 8, 1, sc, rows, p_off, p_idx, half=True)
    g_off, g_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"],
                                       d["support"], 0, rows)
    assert np.abs(np.diff(g_off) - k).max() <= 2, name
    cnt = gpu_counts(L, n)[o["perm"]]
    assert np.array_equal(cnt[rows], np.diff(g_off)), name
    assert np.abs(cnt.astype(np.int64) - k).max() <= 2, name
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx, rows)
    rel = np.abs(rho[rows] - want) / want
    assert rel.max() <= DENSITY_RTOL, (name, rel.max())
    L.free()


def test_plummer64_16m_headline_half_list_at_200_neighbors(plummer16m):
    """The benchmark's headline form: 2^24 particles in 64 Plummer spheres, h
    at 200 neighbors, 8x8 clusters, leaf bucket 256, compressed half list."""
    d, o = _at_count(*plummer16m, 200)
    _check_half_list(d, o, "plummer64_16m half list", 200)


def test_evrard_2m_half_list_at_200_neighbors():
    d = wl.cached(wl.evrard, "evrard_%d_2" % (1 << 21), 1 << 21, seed=2)
    d, o = _at_count(d, oracle_sorted(d), 200)
    _check_half_list(d, o, "evrard_2m half list", 200)


def test_plummer64_16m_sampled_and_h_window(plummer16m):
    import torch
    d, o = plummer16m
    L, t, o, rows, g_off, g_idx = _check_sampled(d, "plummer64_16m", o=o)
    L.free()
    # GPU h iteration from the plain start: sampled particles are in the window
    h = t["h"].clone()
    H = nl.NeighborList()
    p = nl.make_params(key=d["kind"], cluster=8, support=2.0)
    info = H.iterate_h(t["x"], t["y"], t["z"], h, d["box"], p, 200.0, 2.0, max_iter=60,
                       start=nl.NL_HSTART_PLAIN)
    assert info["unconverged"] == 0
    hc = h.cpu().numpy()
    rng = np.random.default_rng(7)
    q = rng.integers(0, len(hc), 96)
    dd = dict(d)
    dd["h"] = hc
    cnt = orc.gather_counts_brute(d["x"], d["y"], d["z"], hc, d["box"], 2.0, q)
    assert np.abs(cnt - 200).max() <= 2
    H.free()


def test_batched_256_full_size_graph_largest_and_smallest():
    """The batched configuration at full size (256 systems, 36M particles, h
    at 100 neighbors from the oracle), through the autotuner and one replay
    of the captured half-list graph, as the benchmark runs it.  Checked
    against the oracle run on each system alone: the 3 largest, the 3
    smallest and the median system (records byte-exact, counts exact,
    density within tolerance), so the persistent queue and the staging
    growth of the largest systems are covered."""
    import torch
    systems = wl.cached(wl.batched, "batched256_5", 256, seed=5)
    sizes = np.array([len(d["x"]) for d in systems])
    order = np.argsort(sizes, kind="stable")
    check = sorted(set(order[:3].tolist() + order[-3:].tolist() + [int(order[len(order) // 2])]))
    sortd = {}
    hs = []
    for k, d in enumerate(systems):
        d = dict(d)
        d["support"] = 2.0
        o = oracle_sorted(d, kind=1)
        d, o = _at_count(d, o, 100)
        hs.append(d["h"])
        if k in check:
            sortd[k] = (d, o)
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    boxes = [d["box"] for d in systems]
    cat = {a: np.concatenate([d[a] for d in systems]).astype(np.float32) for a in "xyzm"}
    cat["h"] = np.concatenate(hs).astype(np.float32)
    dev = {a: torch.from_numpy(v).cuda() for a, v in cat.items()}
    n = int(offs[-1])
    stream = torch.cuda.Stream()
    base = nl.make_params(key=1, cluster=8, support=2.0, half_list=1)
    with torch.cuda.stream(stream):
        best, _ = nl.autotune_batch(dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], offs, boxes,
                                    base, reps=1, stream=stream)
        assert best.half_list == 1
        rho = torch.zeros(n, dtype=torch.float32, device="cuda")
        L = nl.NeighborList()
        G = nl.Graph(L, dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], rho, offs, boxes, best,
                     stream)
        G.launch(stream)
        G.check(stream)
        cnt = torch.empty(n, dtype=torch.int32, device="cuda")
        L.neighbor_counts(cnt, stream)
        stream.synchronize()
    rho, cnt = rho.cpu().numpy(), cnt.cpu().numpy()
    M, MJ = best.cluster, L.sizes()["j_cluster"]
    assert MJ == M
    rec_off, data = L.records()
    pad = [0]
    for s in sizes:
        pad.append(pad[-1] + (int(s) + 8 * M - 1) // (8 * M) * 8 * M)
    for k in check:
        d, o = sortd[k]
        ns = len(o["xs"])
        g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0)
        p_off, p_idx = orc.symmetrize(g_off, g_idx)
        nsc = (ns + 8 * M - 1) // (8 * M)
        so, J, m = orc.cluster_lists(ns, M, p_off, p_idx, np.arange(ns), np.arange(nsc))
        so, J, m = orc.half_lists(so, J, m, np.arange(nsc))
        sc0, cl0 = pad[k] // (8 * M), pad[k] // M
        for t in range(nsc):
            want = orc.encode_record(J[so[t]:so[t + 1]] + cl0, m[so[t]:so[t + 1]], 32, True)
            b = int(rec_off[sc0 + t])
            assert np.array_equal(data[b:b + len(want)], want), (k, ns, t)
        want_rho = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                               np.arange(ns))
        got_rho = rho[offs[k]:offs[k + 1]][o["perm"]]
        assert (np.abs(got_rho - want_rho) / want_rho).max() <= DENSITY_RTOL, (k, ns)
        assert np.array_equal(cnt[offs[k]:offs[k + 1]][o["perm"]], np.diff(g_off)), (k, ns)
    G.free()
    L.free()
