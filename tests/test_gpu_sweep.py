"""The quantities of the neighbor-count sweep (bench.py --sweep: the stand-in
for the paper's Sec. III-A cluster overhead and Sec. III-C memory footprint),
checked against the oracle on a small LJ fluid at three neighbor counts: for
8x8 and 8x4 tiles, full and half lists, compressed and raw records, the list
bytes the library reports equal the sum of the oracle's own encodings of the
canonical records, and its computed pairs (tiles x M x MJ, the numerator of
the cluster overhead) equal the oracle's; the gather pairs (the denominator)
equal the oracle's count."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import oracle_sorted

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nb", [25, 100, 400])
def test_sweep_sizes_and_pairs_match_oracle(nb):
    import torch
    d = wl.lj_fluid(12000, seed=81)
    n = len(d["x"])
    rc = (3.0 * nb / (4.0 * math.pi * 100.0)) ** (1.0 / 3.0)
    d["h"] = np.full(n, rc, np.float32)
    o = oracle_sorted(d)
    g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], 1.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    assert abs(np.diff(g_off).mean() - nb) < 0.1 * nb
    t = {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda()
         for k in ("x", "y", "z", "h")}
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    for M, MJ, half in ((8, 8, 0), (8, 4, 0), (8, 8, 1)):
        nsc = (n + 8 * M - 1) // (8 * M)
        so, J, m = orc.cluster_lists(n, M, p_off, p_idx, np.arange(n), np.arange(nsc),
                                     jcluster=MJ)
        if half:
            so, J, m = orc.half_lists(so, J, m, np.arange(nsc))
        want_pairs = orc.computed_pairs(m, M, MJ)
        for comp in (1, 0):
            want_bytes = sum(orc.record_bytes(J[so[s]:so[s + 1]], 32, bool(comp))
                             for s in range(nsc))
            p = nl.make_params(key=1, cluster=M, j_cluster=MJ, support=1.0, compress=comp,
                               half_list=half)
            L = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
            sz = L.sizes()
            assert sz["list_bytes"] == want_bytes, (nb, M, MJ, half, comp)
            assert sz["n_tiles"] * M * sz["j_cluster"] == want_pairs, (nb, M, MJ, half, comp)
            if (M, MJ, half, comp) == (8, 8, 0, 1):
                L.neighbor_counts(cnt)
                torch.cuda.synchronize()
                assert int(cnt.to(torch.int64).sum().item()) == int(g_off[-1])
            L.free()
