"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (8x8 clusters, compressed list, leaf bucket 256).

The oracle sorts all particles itself and computes, by O(n) brute force per
particle, the symmetric neighbor sets of a sample of whole super-clusters:
their records must match the GPU's byte for byte, and the density / forces /
counts of their particles must match within the tolerances of the small-size
tests.  Smoothing lengths are the generators' (inputs); the GPU's own h
iteration is checked by the window property on sampled particles."""
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


def _check_sampled(d, name, with_density=True):
    o = oracle_sorted(d)
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


def test_plummer64_16m_sampled_and_h_window():
    import torch
    d = wl.cached(wl.plummer, "plummer64_%d_4" % (1 << 24), 1 << 24, n_spheres=64, seed=4)
    L, t, o, rows, g_off, g_idx = _check_sampled(d, "plummer64_16m")
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
