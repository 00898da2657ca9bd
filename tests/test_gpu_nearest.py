"""Distance to the nearest gather neighbor (the pair function of Sec. II-D with
a minimum reduction) against the FP64 oracle, on full and half lists, with
particles that have no neighbor at all (+inf)."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import TILES, gpu_build, oracle_sorted

pytestmark = pytest.mark.gpu

DIST_RTOL = 1e-6   # FP32 sqrt of an FP32 squared distance vs FP64


def _with_isolated(d):
    """Every fifth particle gets a radius too small to hold a neighbor."""
    d = dict(d)
    h = np.asarray(d["h"], np.float32).copy()
    h[::5] *= np.float32(0.01)
    d["h"] = h
    return d


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, d in (("uniform", wl.uniform(20037, seed=141, n_target=60.0)),
                    ("plummer", wl.plummer(24001, n_spheres=3, seed=142, n_target=60.0))):
        d = _with_isolated(d)
        o = oracle_sorted(d)
        g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], d["support"])
        want = orc.nearest(o["xs"], o["ys"], o["zs"], d["box"], g_off, g_idx)
        out[name] = (d, o, want)
    return out


def _gpu_nearest(L, n):
    import torch
    dist = torch.empty(n, dtype=torch.float32, device="cuda")
    L.nearest_distance(dist)
    torch.cuda.synchronize()
    return dist.cpu().numpy()


def _check(got, want):
    fin = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), fin)
    assert fin.sum() > 0.5 * len(want) and (~fin).sum() > 0.1 * len(want)
    rel = np.abs(got[fin] - want[fin]) / want[fin]
    assert rel.max() <= DIST_RTOL, rel.max()


@pytest.mark.parametrize("cluster,jcl", TILES)
@pytest.mark.parametrize("name", ["uniform", "plummer"])
def test_nearest_distance_full_list(cases, name, cluster, jcl):
    d, o, want = cases[name]
    n = len(o["xs"])
    L, t = gpu_build(d, cluster=cluster, j_cluster=jcl)
    _check(_gpu_nearest(L, n)[o["perm"]], want)
    L.free()


@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("name", ["uniform", "plummer"])
def test_nearest_distance_half_list_equals_full(cases, name, cluster):
    """A minimum is the same in any order: the half list gives the full
    list's bits."""
    d, o, want = cases[name]
    n = len(o["xs"])
    H, t = gpu_build(d, cluster=cluster, half_list=1)
    got = _gpu_nearest(H, n)
    _check(got[o["perm"]], want)
    F, _ = gpu_build(d, cluster=cluster)
    assert np.array_equal(got, _gpu_nearest(F, n))
    F.free()
    H.free()
