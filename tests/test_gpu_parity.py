"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs (keys/sort/octree/records bit-exact, density within
1e-5 relative, counts exact)."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import (DENSITY_RTOL, TILES, compare_records, full_reference, gpu_build,
                     gpu_counts, gpu_density, oracle_sorted)

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "uniform": lambda: wl.uniform(20037, seed=101, n_target=60.0),
        "evrard": lambda: wl.evrard(20011, seed=102, n_target=60.0),
        "lj_fluid": lambda: wl.lj_fluid(12000, seed=103),
        "plummer": lambda: wl.plummer(24001, n_spheres=3, seed=104, n_target=60.0),
    }


@pytest.fixture(scope="module")
def cases():
    out = {}
    for k, f in _cases().items():
        d = f()
        o = oracle_sorted(d)
        out[k] = (d, o, full_reference(o, d))
    return out


@pytest.mark.parametrize("name", ["uniform", "evrard", "lj_fluid", "plummer"])
def test_keys_and_stable_sort_bit_exact(cases, name):
    d, o, _ = cases[name]
    L, t = gpu_build(d)
    keys, perm = L.sorted()
    assert np.array_equal(keys, o["keys"])
    assert np.array_equal(perm.astype(np.int64), o["perm"])
    L.free()


@pytest.mark.parametrize("name", ["uniform", "plummer"])
@pytest.mark.parametrize("bucket", [16, 64, 256])
def test_octree_bit_exact(cases, name, bucket):
    d, o, _ = cases[name]
    L, t = gpu_build(d, bucket=bucket)
    g = L.octree()
    ref = orc.octree(o["keys"], bucket)
    assert np.array_equal(g["level"], ref["level"])
    assert np.array_equal(g["first"], ref["first"])
    assert np.array_equal(g["end"], ref["end"])
    assert np.array_equal(g["leaf"].astype(bool), ref["leaf"])
    # skip = first node after the subtree: next node whose level <= own level
    lev = ref["level"]
    nn = len(lev)
    for v in range(0, nn, max(1, nn // 500)):
        w = v + 1
        while w < nn and lev[w] > lev[v]:
            w += 1
        assert g["skip"][v] == w
    L.free()


@pytest.mark.parametrize("name", ["uniform", "evrard", "lj_fluid", "plummer"])
@pytest.mark.parametrize("cluster,jcl", TILES)
@pytest.mark.parametrize("compress", [1, 0])
def test_records_byte_exact(cases, name, cluster, jcl, compress):
    d, o, (g_off, g_idx, p_off, p_idx) = cases[name]
    L, t = gpu_build(d, cluster=cluster, compress=compress, j_cluster=jcl)
    s = L.sizes()
    n = len(o["xs"])
    nsc = s["n_superclusters"]
    assert nsc == (n + 8 * cluster - 1) // (8 * cluster)
    total, so, J, m = compare_records(L, o, d, cluster, compress, np.arange(nsc), np.arange(n),
                                      p_off, p_idx, jcluster=jcl)
    assert s["j_cluster"] == jcl
    assert s["list_bytes"] == total
    assert s["n_entries"] == len(J)
    assert s["n_tiles"] == int(sum(bin(int(v)).count("1") for v in m))
    L.free()


@pytest.mark.parametrize("name", ["uniform", "evrard", "lj_fluid", "plummer"])
@pytest.mark.parametrize("cluster,jcl", TILES)
def test_density_and_counts(cases, name, cluster, jcl):
    d, o, (g_off, g_idx, p_off, p_idx) = cases[name]
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    n = len(o["xs"])
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    rel = np.abs(rho - want) / want
    assert rel.max() <= DENSITY_RTOL, rel.max()
    cnt = gpu_counts(L, n)[o["perm"]]
    assert np.array_equal(cnt, np.diff(g_off))
    L.free()


def test_uncompressed_pass_matches_compressed(cases):
    d, o, _ = cases["plummer"]
    La, ta = gpu_build(d, compress=1)
    Lb, tb = gpu_build(d, compress=0)
    n = len(o["xs"])
    assert np.array_equal(gpu_density(La, ta, n), gpu_density(Lb, tb, n))
    sa, sb = La.sizes(), Lb.sizes()
    assert sa["list_bytes"] < sb["list_bytes"]
    La.free()
    Lb.free()


def test_rebuild_reuses_handle(cases):
    d1, o1, (g1, _, p1o, p1i) = cases["uniform"]
    d2, o2, (g2, _, p2o, p2i) = cases["plummer"]
    L, t = gpu_build(d1)
    from nlcheck import to_dev
    t2 = to_dev(d2)
    p = nl.make_params(key=d2["kind"], cluster=8, support=d2["support"])
    L.build(t2["x"], t2["y"], t2["z"], t2["h"], d2["box"], p)
    n = len(o2["xs"])
    compare_records(L, o2, d2, 8, 1, np.arange(L.sizes()["n_superclusters"]), np.arange(n), p2o, p2i)
    L.free()


# ----------------------------------------------------------------------------- edge cases
def _tiny(n, seed, per=True, h=0.05):
    rng = np.random.default_rng(seed)
    p = rng.random((3, n)).astype(np.float32)
    return {"x": p[0], "y": p[1], "z": p[2], "h": np.full(n, h, np.float32),
            "m": np.full(n, 1.0 / max(n, 1), np.float32),
            "box": {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
                    "periodic": np.array([per] * 3, np.int32)}, "kind": 1, "support": 2.0}


@pytest.mark.parametrize("n", [1, 2, 5, 63, 64, 65, 130, 4097])
@pytest.mark.parametrize("cluster,jcl", TILES)
def test_small_and_ragged_sizes(n, cluster, jcl):
    d = _tiny(n, seed=n, h=0.2 if n < 100 else 0.05)
    o = oracle_sorted(d)
    g_off, g_idx, p_off, p_idx = full_reference(o, d)
    L, t = gpu_build(d, cluster=cluster, bucket=8, j_cluster=jcl)
    nsc = L.sizes()["n_superclusters"]
    compare_records(L, o, d, cluster, 1, np.arange(nsc), np.arange(n), p_off, p_idx, jcluster=jcl)
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    assert (np.abs(rho - want) / want).max() <= DENSITY_RTOL
    L.free()


def test_coincident_particles_and_box_faces():
    """Equal keys beyond the leaf bucket (level-21 leaves), particles on the
    box faces of a periodic box, and pairs across the periodic wrap."""
    n = 300
    d = _tiny(n, seed=5, h=0.03)
    d["x"][:100] = 0.5
    d["y"][:100] = 0.5
    d["z"][:100] = 0.5
    d["x"][100:110] = 0.0
    d["x"][110:120] = 1.0
    d["y"][120:130] = np.float32(0.999)
    d["y"][130:140] = np.float32(0.001)
    o = oracle_sorted(d)
    g_off, g_idx, p_off, p_idx = full_reference(o, d)
    L, t = gpu_build(d, bucket=8)
    tree = L.octree()
    ref = orc.octree(o["keys"], 8)
    assert np.array_equal(tree["end"], ref["end"]) and ref["level"].max() == 21
    compare_records(L, o, d, 8, 1, np.arange(L.sizes()["n_superclusters"]), np.arange(n), p_off, p_idx)
    cnt = gpu_counts(L, n)[o["perm"]]
    assert np.array_equal(cnt, np.diff(g_off))
    assert cnt[np.argsort(o["perm"])][:100].min() >= 99
    L.free()


def test_invalid_inputs_are_rejected():
    import torch
    d = _tiny(200, seed=9)
    base = {k: d[k].copy() for k in ("x", "y", "z", "h", "m")}

    def run(mod=None, box=None, cluster=8, h=None, jcl=0):
        dd = dict(d)
        for k in base:
            dd[k] = base[k].copy()
        if mod:
            mod(dd)
        if box is not None:
            dd["box"] = box
        from nlcheck import to_dev
        t = to_dev(dd)
        p = nl.make_params(key=1, cluster=cluster, support=2.0, j_cluster=jcl)
        with pytest.raises(nl.NLError) as e:
            nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], dd["box"], p)
        return e.value.status

    def nan_x(dd):
        dd["x"][7] = np.nan

    def out_of_box(dd):
        dd["y"][3] = 1.5

    def zero_h(dd):
        dd["h"][11] = 0.0

    def big_h(dd):
        dd["h"][0] = 0.26     # 2h = 0.52 >= L/2 on a periodic axis

    assert run(nan_x) == 1
    assert run(out_of_box) == 1
    assert run(zero_h) == 1
    assert run(big_h) == 2
    assert run(cluster=6) == 1
    for c, j in ((8, 2), (4, 2), (8, 16), (16, 4), (8, -1)):
        assert run(cluster=c, jcl=j) == 1
    # a good build on the same process still works afterwards
    o = oracle_sorted(d)
    L, t = gpu_build(d)
    keys, perm = L.sorted()
    assert np.array_equal(keys, o["keys"])
    L.free()


@pytest.mark.parametrize("jcl", [8, 4])
def test_overflow_rounds_keep_records_exact(cases, monkeypatch, jcl):
    """Tiny initial staging and list buffers force the redo rounds (staging
    growth and list-buffer growth); records stay byte-exact with no holes."""
    d, o, (g_off, g_idx, p_off, p_idx) = cases["evrard"]
    monkeypatch.setenv("NLGB_STAGE_CAP0", "40")
    monkeypatch.setenv("NLGB_LIST_CAP0", "20000")
    L, t = gpu_build(d, j_cluster=jcl)
    n = len(o["xs"])
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, 8, 1, np.arange(nsc), np.arange(n), p_off, p_idx,
                                      jcluster=jcl)
    assert L.sizes()["list_bytes"] == total
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    assert (np.abs(rho - want) / want).max() <= DENSITY_RTOL
    L.free()


FORCE_RTOL = 1e-5   # |a_gpu - a_64| / sum_j |f_ij|_64, per particle


@pytest.mark.parametrize("cluster,jcl", TILES)
def test_sph_pressure_force(cases, cluster, jcl):
    """Inputs rho and P are the oracle's FP64 density rounded to FP32 and
    P = (gamma - 1) rho u, so both sides read identical values."""
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases["evrard"]
    n = len(o["xs"])
    rho64 = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                        np.arange(n))
    rho32 = rho64.astype(np.float32)
    pres32 = (np.float32(2.0 / 3.0) * rho32 * np.float32(0.05)).astype(np.float32)
    ax, ay, az, fa = orc.sph_force(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"],
                                   rho32.astype(np.float64), pres32.astype(np.float64), d["box"],
                                   p_off, p_idx, np.arange(n))
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    inv = np.empty(n, np.int64)
    inv[o["perm"]] = np.arange(n)
    rho_c = torch.from_numpy(rho32[inv]).cuda()       # caller order
    pres_c = torch.from_numpy(pres32[inv]).cuda()
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_SPH_PRESSURE, *out, m=t["m"], rho=rho_c, pres=pres_c)
    torch.cuda.synchronize()
    got = np.stack([a.cpu().numpy()[o["perm"]] for a in out], 1)
    want = np.stack([ax, ay, az], 1)
    err = np.linalg.norm(got - want, axis=1) / np.maximum(fa, 1e-300)
    assert err.max() <= FORCE_RTOL, err.max()
    # momentum: sum m a vanishes up to FP32 roundoff
    mom = (o["ms"][:, None].astype(np.float64) * got).sum(0)
    assert np.abs(mom).max() <= 1e-5 * (o["ms"][:, None] * fa[:, None]).sum()
    L.free()


@pytest.mark.parametrize("cluster,jcl", TILES)
def test_lj_force(cases, cluster, jcl):
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases["lj_fluid"]
    n = len(o["xs"])
    fx, fy, fz, fa = orc.lj_force(o["xs"], o["ys"], o["zs"], d["box"], 1.0, 0.3, g_off, g_idx,
                                  np.arange(n))
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_LJ, *out, eps=1.0, sigma=0.3)
    torch.cuda.synchronize()
    got = np.stack([a.cpu().numpy()[o["perm"]] for a in out], 1)
    want = np.stack([fx, fy, fz], 1)
    err = np.linalg.norm(got - want, axis=1) / fa
    assert err.max() <= FORCE_RTOL, err.max()
    assert np.abs(got.sum(0)).max() <= 1e-5 * fa.sum()
    L.free()


def test_stage_times_before_and_after_a_pass():
    """Stage timing is readable after a build alone (pass stages zero) and
    after a pass (every stage timed)."""
    d = _tiny(5000, seed=77)
    L, t = gpu_build(d)
    L.set_profiling(True)
    from nlcheck import to_dev
    p = nl.make_params(key=1, cluster=8, support=2.0)
    L.build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    st = L.stage_times()
    assert st["search"] > 0 and st["pass"] == 0
    gpu_density(L, t, 5000)
    st = L.stage_times()
    assert st["pass"] > 0
    L.free()


@pytest.mark.parametrize("name", ["uniform", "plummer"])
@pytest.mark.parametrize("cluster", [4, 8, 16])
def test_full_and_half_search_give_the_same_records(cases, monkeypatch, name, cluster):
    """With j-clusters = i-clusters the default search visits only j-clusters
    from the own super-cluster on and completes the records by transposition;
    the full search must produce the same bytes (both equal the oracle)."""
    d, o, (g_off, g_idx, p_off, p_idx) = cases[name]
    n = len(o["xs"])
    monkeypatch.setenv("NLGB_SEARCH", "full")
    L, t = gpu_build(d, cluster=cluster)
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, cluster, 1, np.arange(nsc), np.arange(n), p_off, p_idx)
    assert L.sizes()["list_bytes"] == total
    full = L.sizes()
    L.free()
    monkeypatch.delenv("NLGB_SEARCH")
    L, t = gpu_build(d, cluster=cluster)
    compare_records(L, o, d, cluster, 1, np.arange(nsc), np.arange(n), p_off, p_idx)
    half = L.sizes()
    assert half["list_bytes"] == full["list_bytes"]
    assert half["n_entries"] == full["n_entries"] and half["n_tiles"] == full["n_tiles"]
    assert half["tile_tests"] < full["tile_tests"]
    L.free()


def test_half_search_buffer_growth_keeps_records_exact(cases, monkeypatch):
    """Tiny upper-entry / tuple buffers force the re-run of every
    super-cluster, tiny staging the partial re-runs, a tiny list the
    re-assembly; the records stay byte-exact."""
    d, o, (g_off, g_idx, p_off, p_idx) = cases["evrard"]
    monkeypatch.setenv("NLGB_HALF_CAP0", "1000")
    monkeypatch.setenv("NLGB_STAGE_CAP0", "40")
    monkeypatch.setenv("NLGB_LIST_CAP0", "20000")
    L, t = gpu_build(d)
    n = len(o["xs"])
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, 8, 1, np.arange(nsc), np.arange(n), p_off, p_idx)
    assert L.sizes()["list_bytes"] == total
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    assert (np.abs(rho - want) / want).max() <= DENSITY_RTOL
    L.free()


@pytest.mark.parametrize("h,per", [(0.004, (1, 1, 1)), (0.15, (1, 1, 1)), (0.02, (1, 0, 1)),
                                   (0.02, (0, 0, 0))])
def test_periodic_interior_and_boundary_super_clusters(h, per):
    """Periodic super-clusters far from the faces run the open-axis kernels,
    the others the periodic ones (tiny radii: almost all interior; large
    radii: all boundary; mixed periodicity per axis).  Records and density
    must not depend on the split."""
    rng = np.random.default_rng(int(h * 1e4) + sum(per))
    n = 6000
    p = rng.random((3, n)).astype(np.float32)
    d = {"x": p[0], "y": p[1], "z": p[2], "h": np.full(n, h, np.float32) *
         (0.5 + rng.random(n)).astype(np.float32),
         "m": np.full(n, 1.0 / n, np.float32),
         "box": {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
                 "periodic": np.array(per, np.int32)}, "kind": 1, "support": 2.0}
    o = oracle_sorted(d)
    g_off, g_idx, p_off, p_idx = full_reference(o, d)
    L, t = gpu_build(d)
    nsc = L.sizes()["n_superclusters"]
    total, so, J, m = compare_records(L, o, d, 8, 1, np.arange(nsc), np.arange(n), p_off, p_idx)
    assert L.sizes()["list_bytes"] == total
    rho = gpu_density(L, t, n)[o["perm"]]
    want = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                       np.arange(n))
    assert (np.abs(rho - want) / want).max() <= DENSITY_RTOL
    assert np.array_equal(gpu_counts(L, n)[o["perm"]], np.diff(g_off))
    L.free()


def test_density_from_host_buffers(cases):
    """The host-buffer entry point (copies inside, masses on a second stream)
    gives bit for bit the density of the device-resident build and pass, for
    pageable and pinned inputs and on repeated calls with changed masses."""
    import torch
    d, o, (g_off, g_idx, p_off, p_idx) = cases["plummer"]
    n = len(o["xs"])
    L, t = gpu_build(d)
    want = gpu_density(L, t, n)
    L.free()
    p = nl.make_params(key=d["kind"], cluster=8, support=d["support"])
    E = nl.NeighborList()
    host = {k: np.ascontiguousarray(d[k], dtype=np.float32) for k in ("x", "y", "z", "h", "m")}
    rho = np.empty(n, np.float32)
    E.density_from_host(host["x"], host["y"], host["z"], host["h"], host["m"], d["box"], p, rho)
    assert np.array_equal(rho, want)
    pin = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    rho_p = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
    for scale in (1.0, 2.0, 0.5):
        pin["m"][:] = host["m"] * np.float32(scale)
        E.density_from_host(pin["x"], pin["y"], pin["z"], pin["h"], pin["m"], d["box"], p, rho_p)
        ref = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"] * np.float32(scale), d["box"],
                          g_off, g_idx, np.arange(n))
        assert (np.abs(rho_p[o["perm"]] - ref) / ref).max() <= DENSITY_RTOL
    E.free()
