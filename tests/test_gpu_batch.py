"""Batches of independent systems: every system built inside one batch must
match the oracle run on that system alone (records byte-exact up to the
system's cluster offset, density, counts), and the batched h iteration
must put every particle of every system in its window."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import DENSITY_RTOL, oracle_sorted

pytestmark = pytest.mark.gpu


def _batch(seed, n_systems=10, log_n=(1.7, 3.6)):
    systems = wl.batched(n_systems=n_systems, seed=seed, log_n=log_n)
    for d in systems:
        d["h"] = d["h"].astype(np.float32)
    return systems


def _concat(systems):
    import torch
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    cat = {k: np.concatenate([d[k] for d in systems]).astype(np.float32) for k in "xyzhm"}
    dev = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    return offs, cat, dev


def _pad_offsets(systems, M):
    sc = 8 * M
    pad = [0]
    for d in systems:
        pad.append(pad[-1] + (len(d["x"]) + sc - 1) // sc * sc)
    return pad


@pytest.mark.parametrize("cluster,jcl", [(4, 4), (8, 8), (8, 4), (16, 16), (16, 8)])
def test_batch_matches_systems_alone(cluster, jcl):
    import torch
    systems = _batch(seed=401 + cluster, log_n=(2.7, 3.6))
    offs, cat, dev = _concat(systems)
    p = nl.make_params(key=1, cluster=cluster, support=2.0, j_cluster=jcl)
    L = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs,
                                      [d["box"] for d in systems], p)
    n = int(offs[-1])
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    L.density_pass(dev["m"], rho)
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    L.neighbor_counts(cnt)
    torch.cuda.synchronize()
    rho, cnt = rho.cpu().numpy(), cnt.cpu().numpy()
    rec_off, data = L.records()
    pad = _pad_offsets(systems, cluster)
    total = 0
    for k, d in enumerate(systems):
        o = oracle_sorted(d, kind=1)
        ns = len(o["xs"])
        g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 2.0)
        p_off, p_idx = orc.symmetrize(g_off, g_idx)
        nsc = (ns + 8 * cluster - 1) // (8 * cluster)
        so, J, m = orc.cluster_lists(ns, cluster, p_off, p_idx, np.arange(ns), np.arange(nsc),
                                     jcluster=jcl)
        sc0, cl0 = pad[k] // (8 * cluster), pad[k] // jcl
        for t in range(nsc):
            want = orc.encode_record(J[so[t]:so[t + 1]] + cl0, m[so[t]:so[t + 1]], 32, True)
            b = int(rec_off[sc0 + t])
            assert np.array_equal(data[b:b + len(want)], want), (k, t)
            total += len(want)
        # per-particle results (caller order inside the batch)
        want_rho = orc.density(o["xs"], o["ys"], o["zs"], o["hs"], o["ms"], d["box"], g_off, g_idx,
                               np.arange(ns))
        got_rho = rho[offs[k]:offs[k + 1]][o["perm"]]
        assert (np.abs(got_rho - want_rho) / want_rho).max() <= DENSITY_RTOL, k
        assert np.array_equal(cnt[offs[k]:offs[k + 1]][o["perm"]], np.diff(g_off)), k
    assert L.sizes()["list_bytes"] == total
    L.free()


def test_batch_of_one_equals_single_build():
    import torch
    d = wl.plummer(9001, n_spheres=2, seed=411, n_target=60)
    offs, cat, dev = _concat([d])
    p = nl.make_params(key=1, cluster=8, support=2.0)
    A = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs, [d["box"]], p)
    B = nl.NeighborList().build(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], p)
    ka, pa = A.sorted()
    kb, pb = B.sorted()
    assert np.array_equal(ka, kb) and np.array_equal(pa, pb)
    oa, da = A.records()
    ob, db = B.records()
    for s in range(len(oa)):
        c = int(da[oa[s]:oa[s] + 4].view(np.uint32)[0])
        assert int(db[ob[s]:ob[s] + 4].view(np.uint32)[0]) == c
    assert A.sizes()["list_bytes"] == B.sizes()["list_bytes"]
    A.free()
    B.free()


def test_batch_h_iteration_window():
    import torch
    systems = _batch(seed=421, n_systems=8, log_n=(2.5, 3.8))
    offs, cat, dev = _concat(systems)
    p = nl.make_params(key=1, cluster=8, support=2.0)
    h = dev["h"].clone()
    conv = torch.zeros(int(offs[-1]), dtype=torch.uint8, device="cuda")
    L = nl.NeighborList()
    info = L.iterate_h_batch(dev["x"], dev["y"], dev["z"], h, offs, [d["box"] for d in systems],
                             p, 100.0, 2.0, max_iter=60, start=nl.NL_HSTART_PLAIN, converged=conv)
    assert info["unconverged"] == 0 and bool(conv.all())
    hc = h.cpu().numpy()
    for k, d in enumerate(systems):
        if len(d["x"]) <= 103:
            continue
        hk = hc[offs[k]:offs[k + 1]]
        q = np.arange(len(hk))
        c = orc.gather_counts_brute(d["x"], d["y"], d["z"], hk, d["box"], 2.0, q)
        assert np.abs(c - 100).max() <= 2, k
    L.free()


def test_batch_rejects_bad_tables():
    import torch
    systems = _batch(seed=431, n_systems=3, log_n=(2.7, 3.0))
    offs, cat, dev = _concat(systems)
    p = nl.make_params(key=1, cluster=8, support=2.0)
    bad = offs.copy()
    bad[1] = bad[0]       # empty system
    with pytest.raises(nl.NLError):
        nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], bad,
                                      [d["box"] for d in systems], p)
    bad = offs.copy()
    bad[-1] += 1          # does not end at n
    with pytest.raises(nl.NLError):
        nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], bad,
                                      [d["box"] for d in systems], p)
