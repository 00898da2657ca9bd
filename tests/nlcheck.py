"""Shared helpers of the GPU parity tests: run the CUDA library through its
C ABI and compare with the CPU oracle on the same seeded inputs."""
import numpy as np

import oracle as orc
from paper_2602_19873_gb300 import nl

DENSITY_RTOL = 1e-5   # FP32 density vs the FP64 oracle, max relative error

# tile shapes (i-cluster M, j-cluster MJ) the library supports
TILES = [(4, 4), (8, 8), (8, 4), (16, 16), (16, 8)]


def to_dev(d, keys=("x", "y", "z", "h", "m")):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda() for k in keys}


def gpu_build(d, cluster=8, compress=1, bucket=256, kind=None, support=None, j_cluster=0,
              half_list=0):
    import torch
    t = to_dev(d)
    p = nl.make_params(key=d["kind"] if kind is None else kind, cluster=cluster,
                       support=d["support"] if support is None else support, compress=compress,
                       leaf_bucket=bucket, j_cluster=j_cluster, half_list=half_list)
    L = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    torch.cuda.synchronize()
    return L, t


def oracle_sorted(d, kind=None):
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"] if kind is None else kind)
    perm = orc.sort(k)
    out = {"keys": k[perm], "perm": perm}
    for a in ("x", "y", "z", "h", "m"):
        out[a + "s"] = np.ascontiguousarray(np.asarray(d[a], np.float32)[perm])
    return out


def gpu_records(L, sc_ids):
    off, data = L.records()
    out = []
    for s in sc_ids:
        o = int(off[s])
        assert o != 0xffffffff * 4, "super-cluster %d has no record" % s
        cnt = int(data[o:o + 4].view(np.uint32)[0])
        out.append((o, cnt, data))
    return out


def compare_records(L, o, d, cluster, compress, sc_ids, rows, p_off, p_idx, jcluster=None,
                    half=False):
    """Byte-exact comparison of the GPU records of sc_ids with the oracle's
    independent encoding of the canonical lists built from (rows, P); half:
    the oracle's half lists."""
    n = len(o["xs"])
    so, J, m = orc.cluster_lists(n, cluster, p_off, p_idx, rows, sc_ids,
                                 jcluster=jcluster or cluster)
    if half:
        so, J, m = orc.half_lists(so, J, m, sc_ids)
    off, data = L.records()
    total = 0
    for t, s in enumerate(sc_ids):
        want = orc.encode_record(J[so[t]:so[t + 1]], m[so[t]:so[t + 1]], 32, bool(compress))
        b = int(off[s])
        got = data[b:b + len(want)]
        if not np.array_equal(got, want):
            gj, gm = orc.decode_record(data[b:], 32, bool(compress))
            raise AssertionError(
                "record of super-cluster %d differs: oracle J=%s mask=%s; gpu J=%s mask=%s" % (
                    s, J[so[t]:so[t + 1]][:20], m[so[t]:so[t + 1]][:20], gj[:20], gm[:20]))
        total += len(want)
    return total, so, J, m


def full_reference(o, d):
    g_off, g_idx = orc.gather_all(o["xs"], o["ys"], o["zs"], o["hs"], d["box"], d["support"])
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    return g_off, g_idx, p_off, p_idx


def gpu_density(L, t, n):
    import torch
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    L.density_pass(t["m"], rho)
    torch.cuda.synchronize()
    return rho.cpu().numpy()


def gpu_counts(L, n):
    import torch
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    L.neighbor_counts(c)
    torch.cuda.synchronize()
    return c.cpu().numpy()
