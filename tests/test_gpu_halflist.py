"""Half lists (every pair of clusters of two super-clusters stored once, the
symmetric lists of Sec. II-D): records byte-exact against the oracle's half
lists, densities within 1e-5 and counts exact against the oracle, repeatable
bit for bit (the j shares are added as integers), in batches and CUDA graphs
too; SPH pressure, LJ and LJ + Coulomb forces on both particles of a pair
within 1e-5 (FP64 sums of the shares)."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import (DENSITY_RTOL, compare_records, full_reference, gpu_build, gpu_counts,
                     gpu_density, oracle_sorted)

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "uniform": lambda: wl.uniform(20037, seed=131, n_target=60.0),
        "evrard": lambda: wl.evrard(20011, seed=132, n_target=60.0),
        "plummer": lambda: wl.plummer(24001, n_spheres=3, seed=133, n_target=60.0),
        "lj_fluid": lambda: wl.lj_fluid(12000, seed=134),
    }


@pytest.fixture(scope="module")
def cases():
    out = {}
    for k, f in _cases().items():
        d = f()
        o = oracle_sorted(d)
        out[k] = (d, o, full_reference(o, d))
    return out


@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("name", ["uniform", "evrard", "plummer", "lj_fluid"])
def test_half_list_records_density_counts(cases, name, cluster):
    d, o, (g_off, g_idx, p_off, p_idx) = cases[name]
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=cluster, half_list=1)
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, cluster, 1, np.arange(nsc), np.arange(n), p_off,
                                      p_idx, half=True)
    assert L.sizes()["list_bytes"] == total
    assert L.sizes()["n_entries"] == len(J)
    rho = gpu_density(L, t, n)
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    rel = np.abs(rho[o["perm"]] - want) / want
    assert rel.max() <= DENSITY_RTOL, rel.max()
    assert np.array_equal(gpu_counts(L, n)[o["perm"]], np.diff(g_off))
    # the same bits on a second pass
    assert np.array_equal(gpu_density(L, t, n), rho)
    # about half of the full list's entries
    F, _ = gpu_build(d, cluster=cluster)
    assert L.sizes()["list_bytes"] < 0.75 * F.sizes()["list_bytes"]
    F.free()
    L.free()


def test_half_list_uncompressed(cases):
    d, o, (g_off, g_idx, p_off, p_idx) = cases["plummer"]
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=8, compress=0, half_list=1)
    nsc = L.sizes()["n_superclusters"]
    compare_records(L, o, d, 8, 0, np.arange(nsc), np.arange(n), p_off, p_idx, half=True)
    assert np.array_equal(gpu_counts(L, n)[o["perm"]], np.diff(g_off))
    L.free()


FORCE_RTOL = 1e-5   # |a_gpu - a_64| / sum_j |f_ij|_64, per particle


def _forces(out, o):
    return np.stack([a.cpu().numpy()[o["perm"]] for a in out], 1)


@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("name", ["evrard", "uniform"])
def test_half_list_sph_pressure_force(cases, name, cluster):
    """Both particles of a stored pair take the symmetric pressure force
    (a_j gets -m_i/m_j of a_i's pair term); inputs as in the full-list test."""
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases[name]
    n = len(o["xs"])
    rho64 = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                        np.arange(n))
    rho32 = rho64.astype(np.float32)
    pres32 = (np.float32(2.0 / 3.0) * rho32 * np.float32(0.05)).astype(np.float32)
    ax, ay, az, fa = orc.sph_force(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"],
                                   rho32.astype(np.float64), pres32.astype(np.float64), d["box"],
                                   p_off, p_idx, np.arange(n))
    L, t = gpu_build(d, cluster=cluster, half_list=1)
    inv = np.empty(n, np.int64)
    inv[o["perm"]] = np.arange(n)
    rho_c = torch.from_numpy(rho32[inv]).cuda()
    pres_c = torch.from_numpy(pres32[inv]).cuda()
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_SPH_PRESSURE, *out, m=t["m"], rho=rho_c, pres=pres_c)
    torch.cuda.synchronize()
    got = _forces(out, o)
    err = np.linalg.norm(got - np.stack([ax, ay, az], 1), axis=1) / np.maximum(fa, 1e-300)
    assert err.max() <= FORCE_RTOL, err.max()
    mom = (o["ms"][:, None].astype(np.float64) * got).sum(0)
    assert np.abs(mom).max() <= 1e-5 * (o["ms"][:, None] * fa[:, None]).sum()
    L.free()


@pytest.mark.parametrize("cluster", [4, 8, 16])
def test_half_list_lj_force(cases, cluster):
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases["lj_fluid"]
    n = len(o["xs"])
    fx, fy, fz, fa = orc.lj_force(o["xs"], o["ys"], o["zs"], d["box"], 1.0, 0.3, g_off, g_idx,
                                  np.arange(n))
    L, t = gpu_build(d, cluster=cluster, half_list=1)
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_LJ, *out, eps=1.0, sigma=0.3)
    torch.cuda.synchronize()
    got = _forces(out, o)
    err = np.linalg.norm(got - np.stack([fx, fy, fz], 1), axis=1) / fa
    assert err.max() <= FORCE_RTOL, err.max()
    assert np.abs(got.sum(0)).max() <= 1e-5 * fa.sum()
    # a second pass: the FP64 sums round to the same FP32 values (up to rare
    # ties of the rounding)
    L.force_pass(nl.NL_FORCE_LJ, *out, eps=1.0, sigma=0.3)
    torch.cuda.synchronize()
    again = _forces(out, o)
    assert np.mean(again != got) < 1e-3
    assert (np.abs(again - got).max(1) / fa).max() <= 1e-6
    L.free()


def test_half_list_lj_coulomb_force_and_refresh():
    """The Verlet-buffer workload on a half list: the pairs within rc before
    and after a refresh of the positions, against the oracle."""
    import torch
    d = wl.lj_coulomb(12000, seed=138)
    o = oracle_sorted(d)
    q = np.asarray(d["q"], np.float32)[o["perm"]]
    n = len(o["xs"])
    L, t = gpu_build(d, half_list=1)
    qd = torch.from_numpy(np.asarray(d["q"], np.float32)).cuda()
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    rng = np.random.default_rng(139)
    pos = [o["xs"], o["ys"], o["zs"]]
    for step in range(2):
        if step:
            v = rng.normal(size=(n, 3))
            v *= (0.45 * (d["r_list"] - d["rc"]) * rng.random(n) / np.linalg.norm(v, axis=1))[:, None]
            Lf = np.float32(d["L"])
            new = {}
            for a, k in enumerate("xyz"):
                p = (np.asarray(d[k], np.float64) + v[:, a]).astype(np.float32)
                p = np.where(p < 0, p + Lf, p)
                new[k] = np.where(p >= Lf, p - Lf, p).astype(np.float32)
            nd = {k: torch.from_numpy(new[k]).cuda() for k in "xyz"}
            L.refresh_positions(nd["x"], nd["y"], nd["z"])
            pos = [new[k][o["perm"]] for k in "xyz"]
        L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out, m=qd, eps=d["eps"], sigma=d["sigma"],
                     rc=d["rc"], kc=d["kc"])
        torch.cuda.synchronize()
        got = _forces(out, o)
        hr = np.full(n, np.float32(d["rc"]), np.float32)
        g_off, g_idx = orc.gather_all(*pos, hr, d["box"], 1.0)
        fx, fy, fz, fa = orc.ljc_force(*pos, d["box"], d["eps"], d["sigma"], q, d["kc"], g_off,
                                       g_idx, np.arange(n))
        err = np.linalg.norm(got - np.stack([fx, fy, fz], 1), axis=1) / fa
        assert err.max() <= FORCE_RTOL, (step, err.max())
    L.free()


def test_half_list_needs_whole_j_clusters(cases):
    d, o, _ = cases["lj_fluid"]
    with pytest.raises(nl.NLError):
        gpu_build(d, cluster=8, j_cluster=4, half_list=1)


def test_half_list_batch_of_open_and_periodic_systems():
    import torch
    systems = wl.batched(n_systems=10, seed=135, log_n=(2.7, 3.6))
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    dev = {k: torch.from_numpy(np.concatenate([d[k] for d in systems]).astype(np.float32)).cuda()
           for k in "xyzhm"}
    p = nl.make_params(key=1, cluster=8, support=2.0, half_list=1)
    L = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs,
                                      [d["box"] for d in systems], p)
    n = int(offs[-1])
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    L.density_pass(dev["m"], rho)
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    L.neighbor_counts(cnt)
    torch.cuda.synchronize()
    rho, cnt = rho.cpu().numpy(), cnt.cpu().numpy()
    for k, d in enumerate(systems):
        o = oracle_sorted(d, kind=1)
        g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0)
        want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                           np.arange(len(o["xs"])))
        got = rho[offs[k]:offs[k + 1]][o["perm"]]
        assert (np.abs(got - want) / want).max() <= DENSITY_RTOL, k
        assert np.array_equal(cnt[offs[k]:offs[k + 1]][o["perm"]], np.diff(g_off)), k
    L.free()


def test_half_list_graph_replay_matches_normal_build():
    import torch
    stream = torch.cuda.Stream()
    systems = wl.batched(n_systems=8, seed=136, log_n=(2.7, 3.5))
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    dev = {k: torch.from_numpy(np.concatenate([d[k] for d in systems]).astype(np.float32)).cuda()
           for k in "xyzhm"}
    boxes = [d["box"] for d in systems]
    p = nl.make_params(key=1, cluster=8, support=2.0, half_list=1)
    with torch.cuda.stream(stream):
        A = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs, boxes, p,
                                          stream)
        want = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
        A.density_pass(dev["m"], want, stream)
        stream.synchronize()
        rho = torch.zeros(int(offs[-1]), dtype=torch.float32, device="cuda")
        L = nl.NeighborList()
        G = nl.Graph(L, dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], rho, offs, boxes, p,
                     stream)
        rho.zero_()
        for _ in range(2):
            G.launch(stream)
        G.check(stream)
        stream.synchronize()
        assert np.array_equal(rho.cpu().numpy(), want.cpu().numpy())
        assert L.sizes()["list_bytes"] == A.sizes()["list_bytes"]
    A.free()
    G.free()
    L.free()


def test_half_list_evrard_2m_sampled():
    """Full size (2^21 particles, 8x8, compressed, leaf bucket 256): sampled
    super-clusters byte-exact against the oracle's half lists, their
    particles' densities within 1e-5."""
    d = wl.cached(wl.evrard, "evrard_%d_2" % (1 << 21), 1 << 21, seed=2)
    o = oracle_sorted(d)
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=8, compress=1, bucket=256, half_list=1)
    nsc = L.sizes()["n_superclusters"]
    rng = np.random.default_rng(137)
    sc = np.unique(np.concatenate([[0, nsc // 2, nsc - 1], rng.integers(0, nsc, 5)]))
    rows = np.concatenate([np.arange(s * 64, min(n, (s + 1) * 64)) for s in sc])
    p_off, p_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0, 1, rows)
    compare_records(L, o, d, 8, 1, sc, rows, p_off, p_idx, half=True)
    g_off, g_idx = orc.brute_neighbors(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0, 0, rows)
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx, rows)
    assert (np.abs(rho[rows] - want) / want).max() <= DENSITY_RTOL
    assert np.array_equal(gpu_counts(L, n)[o["perm"]][rows], np.diff(g_off))
    L.free()


def test_half_list_from_host_buffers_and_mass_scaling(cases):
    """The host-buffer entry point on half lists: the same bits as the device
    build and pass, and the oracle's density for masses scaled by 2^+-k and by
    3 (the fixed-point unit follows the largest mass)."""
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases["plummer"]
    n = len(o["xs"])
    L, t = gpu_build(d, half_list=1)
    want = gpu_density(L, t, n)
    L.free()
    p = nl.make_params(key=d["kind"], cluster=8, support=d["support"], half_list=1)
    E = nl.NeighborList()
    host = {k: np.ascontiguousarray(d[k], dtype=np.float32) for k in ("x", "y", "z", "h", "m")}
    rho = np.empty(n, np.float32)
    E.density_from_host(host["x"], host["y"], host["z"], host["h"], host["m"], d["box"], p, rho)
    assert np.array_equal(rho, want)
    for scale in (1024.0, 1.0 / 4096.0, 3.0, 1e-20, 1e20):
        m = host["m"] * np.float32(scale)
        E.density_from_host(host["x"], host["y"], host["z"], host["h"], m, d["box"], p, rho)
        ref = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"] * np.float32(scale),
                          d["box"], g_off, g_idx, np.arange(n))
        assert (np.abs(rho[o["perm"]] - ref) / ref).max() <= DENSITY_RTOL, scale
    E.free()


def test_h_iteration_with_half_list_params_builds_full_lists(cases):
    """The h iteration re-runs single super-clusters, so it works on full lists
    whatever half_list says: the same h as with full-list parameters."""
    import torch
    d, o, _ = cases["evrard"]
    t = {k: torch.from_numpy(np.ascontiguousarray(d[k], np.float32)).cuda() for k in "xyzh"}
    out = []
    for half in (0, 1):
        h = t["h"].clone()
        H = nl.NeighborList()
        p = nl.make_params(key=d["kind"], cluster=8, support=2.0, half_list=half)
        H.iterate_h(t["x"], t["y"], t["z"], h, d["box"], p, 60.0, 2.0, max_iter=60,
                    start=nl.NL_HSTART_PLAIN)
        assert H.sizes()["list_bytes"] > 0
        out.append((h.cpu().numpy(), H.sizes()["list_bytes"]))
        H.free()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]  # both left a full list
