"""Lennard-Jones + Coulomb over a Verlet-buffer list (Sec. III-B: the list is
built at a radius holding about 200 neighbors, the interaction cutoff holds
about 150, and the list serves several steps).  The CUDA pass is compared with
the FP64 oracle on the pairs within the cutoff, before and after the
positions are refreshed without a rebuild."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import TILES, gpu_build, gpu_counts, oracle_sorted, to_dev

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5   # |F_gpu - F_64| / sum_j |f_ij|_64, per particle


@pytest.fixture(scope="module")
def fluid():
    d = wl.lj_coulomb(12000, seed=111)
    o = oracle_sorted(d)
    o["q"] = np.asarray(d["q"], np.float32)[o["perm"]]
    return d, o


def _ljc_gpu(L, n, q, d, rc=None, kc=None):
    import torch
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    qd = None if q is None else torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out, m=qd, eps=d["eps"], sigma=d["sigma"],
                 rc=d["rc"] if rc is None else rc, kc=d["kc"] if kc is None else kc)
    torch.cuda.synchronize()
    return np.stack([a.cpu().numpy() for a in out], 1)


def _check(got_sorted, xs, ys, zs, q, d, rc, kc, rows=None):
    n = len(xs)
    hr = np.full(n, np.float32(rc), np.float32)
    if rows is None:
        off, idx = orc.gather_all(xs, ys, zs, hr, d["box"], 1.0)
        rows = np.arange(n)
    else:
        off, idx = orc.brute_neighbors(xs, ys, zs, hr, d["box"], 1.0, 0, rows)
    fx, fy, fz, fa = orc.ljc_force(xs, ys, zs, d["box"], d["eps"], d["sigma"], q, kc, off, idx,
                                   rows)
    want = np.stack([fx, fy, fz], 1)
    err = np.linalg.norm(got_sorted[rows] - want, axis=1) / fa
    assert err.max() <= FORCE_RTOL, err.max()
    return off, fa


@pytest.mark.parametrize("cluster,jcl", TILES)
def test_ljc_force_matches_oracle(fluid, cluster, jcl):
    d, o = fluid
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    got = _ljc_gpu(L, n, d["q"], d)[o["perm"]]
    off, fa = _check(got, o["xs"], o["ys"], o["zs"], o["q"], d, d["rc"], d["kc"])
    assert np.abs(got.sum(0)).max() <= 1e-5 * fa.sum()
    # the Verlet-buffer shape: ~200 listed neighbors, ~150 within the cutoff
    assert abs(gpu_counts(L, n).mean() - 200.0) < 8.0
    assert abs(np.diff(off).mean() - 150.0) < 6.0
    L.free()


def test_ljc_without_cutoff_and_charges_is_lj_at_the_list_radius(fluid):
    d, o = fluid
    n = len(o["xs"])
    L, t = gpu_build(d)
    got = _ljc_gpu(L, n, None, d, rc=0.0, kc=d["kc"])[o["perm"]]
    _check(got, o["xs"], o["ys"], o["zs"], None, d, d["r_list"], 0.0)
    L.free()


def test_ljc_rejects_bad_parameters(fluid):
    import torch
    d, o = fluid
    n = len(o["xs"])
    L, t = gpu_build(d)
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    for kw in ({"sigma": 0.0}, {"rc": -0.1}, {"rc": float("nan")}, {"kc": float("inf")},
               {"eps": float("nan")}):
        args = {"eps": 1.0, "sigma": 0.3, "rc": 0.7, "kc": 1.0}
        args.update(kw)
        with pytest.raises(nl.NLError):
            L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out, **args)
    with pytest.raises(nl.NLError):
        L.refresh_positions(None, t["y"], t["z"])
    L.free()


def _displaced(d, frac, seed):
    """Every particle moved by at most frac * (r_list - rc) in a random
    direction, wrapped into the periodic box."""
    rng = np.random.default_rng(seed)
    n = len(d["x"])
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v *= (frac * (d["r_list"] - d["rc"]) * rng.random(n))[:, None]
    Lf = np.float32(d["L"])
    out = dict(d)
    crossed = 0
    for a, k in enumerate(("x", "y", "z")):
        p = (np.asarray(d[k], np.float64) + v[:, a]).astype(np.float32)
        crossed += int(np.sum((p < 0) | (p >= Lf)))
        p = np.where(p < 0, p + Lf, p)
        p = np.where(p >= Lf, p - Lf, p).astype(np.float32)
        out[k] = np.ascontiguousarray(p)
    return out, crossed


def _max_disp(d0, d1):
    L = float(np.float32(d0["L"]))
    dv = np.stack([np.asarray(d1[k], np.float64) - np.asarray(d0[k], np.float64)
                   for k in ("x", "y", "z")], 1)
    dv -= L * np.round(dv / L)
    return float(np.linalg.norm(dv, axis=1).max())


@pytest.mark.parametrize("cluster,jcl", [(8, 8), (8, 4)])
def test_refreshed_positions_keep_the_list_exact(fluid, cluster, jcl):
    """Two steps of list reuse: after each refresh the pass equals the oracle
    on the pairs within rc at the new positions; max_disp reports the largest
    move from the build positions; a rebuild starts a new reference."""
    import torch
    d, o = fluid
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    md = torch.zeros(1, dtype=torch.float32, device="cuda")
    prev = d
    for step, frac in enumerate((0.2, 0.45)):
        d1, crossed = _displaced(d, frac, seed=200 + step)
        assert crossed > 0  # some particles leave through a face and wrap
        t1 = to_dev(d1, ("x", "y", "z"))
        L.refresh_positions(t1["x"], t1["y"], t1["z"], md)
        torch.cuda.synchronize()
        want = _max_disp(d, d1)
        assert abs(float(md.item()) - want) <= 1e-5 * want + 1e-6
        assert 2 * want < d["r_list"] - d["rc"]
        got = _ljc_gpu(L, n, d["q"], d)[o["perm"]]
        xs, ys, zs = (np.asarray(d1[k], np.float32)[o["perm"]] for k in ("x", "y", "z"))
        off, fa = _check(got, xs, ys, zs, o["q"], d, d["rc"], d["kc"])
        assert np.abs(got.sum(0)).max() <= 1e-5 * fa.sum()
        prev = d1
    # a rebuild on the moved positions: max_disp restarts from them
    t2 = to_dev(prev, ("x", "y", "z", "h"))
    L.build(t2["x"], t2["y"], t2["z"], t2["h"], d["box"],
            nl.make_params(key=d["kind"], cluster=cluster, support=d["support"],
                           j_cluster=jcl))
    L.refresh_positions(t2["x"], t2["y"], t2["z"], md)
    torch.cuda.synchronize()
    assert float(md.item()) == 0.0
    L.free()


def test_lj_coulomb_4m_sampled():
    """Full size in the benchmark's launch configuration (8x8, compressed,
    leaf bucket 256): sampled particles against the oracle's brute force,
    at the build positions and after one refresh."""
    import torch
    d = wl.cached(wl.lj_coulomb, "lj_coulomb_4000000_6", 4_000_000, seed=6)
    o = oracle_sorted(d)
    q = np.asarray(d["q"], np.float32)[o["perm"]]
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=8, compress=1, bucket=256)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 400)]))
    got = _ljc_gpu(L, n, d["q"], d)[o["perm"]]
    off, fa = _check(got, o["xs"], o["ys"], o["zs"], q, d, d["rc"], d["kc"], rows)
    assert abs(np.diff(off).mean() - 150.0) < 6.0
    d1, crossed = _displaced(d, 0.45, seed=12)
    t1 = to_dev(d1, ("x", "y", "z"))
    md = torch.zeros(1, dtype=torch.float32, device="cuda")
    L.refresh_positions(t1["x"], t1["y"], t1["z"], md)
    torch.cuda.synchronize()
    assert 2 * float(md.item()) < d["r_list"] - d["rc"]
    got = _ljc_gpu(L, n, d["q"], d)[o["perm"]]
    xs, ys, zs = (np.asarray(d1[k], np.float32)[o["perm"]] for k in ("x", "y", "z"))
    _check(got, xs, ys, zs, q, d, d["rc"], d["kc"], rows)
    L.free()


def test_refresh_in_a_batch_of_open_and_periodic_systems():
    """A batch mixing periodic cubes and open spheres: after a refresh the
    open systems, the interior and the boundary super-clusters each keep the
    exact pair set within rc (one system at a time through the oracle)."""
    import torch
    systems = []
    for k, n in enumerate((3001, 5200, 4100, 2600, 6000)):
        d = wl.uniform(n, seed=121 + k, n_target=100.0)
        if k % 2:  # the same cube, open
            d["box"] = dict(d["box"], periodic=np.zeros(3, np.int32))
        systems.append(d)
    rng = np.random.default_rng(122)
    r_min = min(float(np.min(2.0 * d["h"])) for d in systems)
    rc = float(np.float32(0.7 * r_min))
    eps, sigma, kc = 1.0, 0.2 * rc, 1.0
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    q = [np.where(rng.random(len(d["x"])) < 0.5, 1.0, -1.0).astype(np.float32) for d in systems]
    moved = []
    for d in systems:
        n = len(d["x"])
        v = rng.normal(size=(n, 3))
        v *= (0.45 * (r_min - rc) * rng.random(n) / np.linalg.norm(v, axis=1))[:, None]
        m = dict(d)
        for a, k in enumerate("xyz"):
            p = (np.asarray(d[k], np.float64) + v[:, a]).astype(np.float32)
            if d["box"]["periodic"][a]:
                lo, hi = np.float32(d["box"]["lo"][a]), np.float32(d["box"]["hi"][a])
                p = np.where(p < lo, p + (hi - lo), p)
                p = np.where(p >= hi, p - (hi - lo), p).astype(np.float32)
            m[k] = np.ascontiguousarray(p, np.float32)
        moved.append(m)
    cat = {k: np.concatenate([d[k] for d in systems]).astype(np.float32) for k in "xyzh"}
    catm = {k: np.concatenate([d[k] for d in moved]).astype(np.float32) for k in "xyz"}
    dev = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    devm = {k: torch.from_numpy(v).cuda() for k, v in catm.items()}
    qd = torch.from_numpy(np.concatenate(q)).cuda()
    p = nl.make_params(key=1, cluster=8, support=2.0)
    L = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs,
                                      [d["box"] for d in systems], p)
    L.refresh_positions(devm["x"], devm["y"], devm["z"])
    n = int(offs[-1])
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out, m=qd, eps=eps, sigma=sigma, rc=rc, kc=kc)
    torch.cuda.synchronize()
    got = np.stack([a.cpu().numpy() for a in out], 1)
    for k, d in enumerate(moved):
        m = len(d["x"])
        xs, ys, zs = (np.asarray(d[a], np.float32) for a in "xyz")
        hr = np.full(m, np.float32(rc), np.float32)
        off, idx = orc.gather_all(xs, ys, zs, hr, d["box"], 1.0)
        fx, fy, fz, fa = orc.ljc_force(xs, ys, zs, d["box"], eps, sigma, q[k], kc, off, idx,
                                       np.arange(m))
        g = got[offs[k]:offs[k + 1]]
        has = fa > 0
        err = np.linalg.norm(g[has] - np.stack([fx, fy, fz], 1)[has], axis=1) / fa[has]
        assert err.max() <= FORCE_RTOL, (k, err.max())
        assert np.all(g[~has] == 0.0)
    L.free()
