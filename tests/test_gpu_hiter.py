"""GPU smoothing-length iteration: every returned h lies in the neighbor
window according to the oracle's own FP32-predicate counting; degenerate
inputs report NL_ERR_NOT_CONVERGED with per-particle flags."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import oracle_sorted, to_dev

pytestmark = pytest.mark.gpu


def _iterate(d, n_target, tol, start, max_iter=60, cluster=8, jcl=0):
    import torch
    t = to_dev(d)
    p = nl.make_params(key=d["kind"], cluster=cluster, support=d["support"], j_cluster=jcl)
    L = nl.NeighborList()
    conv = torch.zeros(len(d["x"]), dtype=torch.uint8, device="cuda")
    info = L.iterate_h(t["x"], t["y"], t["z"], t["h"], d["box"], p, n_target, tol,
                       max_iter=max_iter, start=start, converged=conv, check=False)
    torch.cuda.synchronize()
    return L, t["h"].cpu().numpy(), conv.cpu().numpy(), info


def _oracle_counts(d, h):
    dd = dict(d)
    dd["h"] = h
    o = oracle_sorted(dd)
    g_off, _ = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], d["support"])
    cnt = np.empty(len(h), np.int64)
    cnt[o["perm"]] = np.diff(g_off)
    return cnt


@pytest.mark.parametrize("name,start", [("evrard", nl.NL_HSTART_PLAIN),
                                        ("plummer", nl.NL_HSTART_PLAIN),
                                        ("uniform", nl.NL_HSTART_GIVEN),
                                        ("plummer", nl.NL_HSTART_GIVEN)])
@pytest.mark.parametrize("cluster,jcl", [(4, 4), (8, 8), (8, 4)])
def test_h_in_window(name, start, cluster, jcl):
    d = {"evrard": lambda: wl.evrard(30011, seed=201, n_target=100),
         "plummer": lambda: wl.plummer(30001, n_spheres=4, seed=202, n_target=100),
         "uniform": lambda: wl.uniform(30011, seed=203, n_target=100)}[name]()
    L, h, conv, info = _iterate(d, 100.0, 2.0, start, cluster=cluster, jcl=jcl)
    assert info["status"] == 0, info
    assert conv.all()
    cnt = _oracle_counts(d, h)
    assert np.abs(cnt - 100).max() <= 2
    assert info["iterations"] >= 1 and info["rebuilds"] >= 1
    L.free()


def test_plain_start_is_close():
    """The plain start (super-cluster box volume) lands within a factor of a
    few of the answer on a smooth distribution."""
    d = wl.uniform(40000, seed=204, n_target=100)
    d["h"][:] = np.float32(1e-3)
    L, h, conv, info = _iterate(d, 100.0, 2.0, nl.NL_HSTART_PLAIN)
    assert info["status"] == 0
    assert info["iterations"] <= 25
    L.free()


def test_degenerate_ties_report_not_converged():
    """300 coincident particles: the count jumps from 0 to 299 at one h, so
    the window around 200 is empty; the cap ends the iteration with flags."""
    n = 600
    rng = np.random.default_rng(5)
    p = rng.random((3, n)).astype(np.float32)
    p[:, :300] = 0.5
    d = {"x": p[0], "y": p[1], "z": p[2], "h": np.full(n, 0.05, np.float32),
         "m": np.full(n, 1.0 / n, np.float32), "kind": 1, "support": 2.0,
         "box": {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
                 "periodic": np.zeros(3, np.int32)}}
    L, h, conv, info = _iterate(d, 200.0, 2.0, nl.NL_HSTART_GIVEN, max_iter=30)
    assert info["status"] == 6
    assert info["unconverged"] >= 300
    assert not conv[:300].any()
    cnt = _oracle_counts(d, h)
    assert (np.abs(cnt[conv == 1] - 200) <= 2).all()
    L.free()


def test_iteration_cap_reports_not_converged():
    d = wl.plummer(20000, n_spheres=2, seed=206, n_target=100)
    d["h"] = d["h"] * np.float32(0.2)
    L, h, conv, info = _iterate(d, 100.0, 2.0, nl.NL_HSTART_GIVEN, max_iter=1)
    assert info["status"] == 6 and info["iterations"] == 1
    assert info["unconverged"] == int((conv == 0).sum()) > 0
    L.free()


def test_iteration_trace_is_consistent():
    """nl_get_hiter_trace: one record per count pass; the first pass counts
    every super-cluster after a rebuild, later ones only the unconverged
    ones, the last leaves none unconverged, and the rebuilt passes are the
    iteration's rebuilds."""
    d = wl.plummer(30001, n_spheres=4, seed=205, n_target=100)
    L, h, conv, info = _iterate(d, 100.0, 2.0, nl.NL_HSTART_PLAIN)
    assert info["status"] == 0
    tr = L.hiter_trace()
    assert len(tr) == info["iterations"]
    assert sum(t["rebuilt"] for t in tr) == info["rebuilds"]
    nsc = L.sizes()["n_superclusters"]
    assert tr[0]["rebuilt"] == 1 and tr[0]["active"] == nsc
    assert all(t["active"] <= nsc and t["entries"] > 0 and t["tiles"] >= t["entries"] for t in tr)
    assert tr[-1]["unconverged"] == 0 and all(t["unconverged"] > 0 for t in tr[:-1])
    assert all(t["ms"] > 0 for t in tr)
    L.free()
