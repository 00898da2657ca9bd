"""SFC domain decomposition with a halo exchange (Sec. I key-range domains,
Sec. IV halos), on CPU ranks over gloo.

Each rank runs the decomposition's host logic (paper_2602_19873_gb300.domain)
with the oracle standing in for the device steps: keys, histograms, owner
and halo masks, grouping, and the local build + density pass.  The
densities and neighbor counts of the owned particles, gathered over all
ranks, must equal the single-domain oracle's; every particle must be owned
by exactly one rank, in contiguous ascending key ranges of about N/P
particles each."""
import os
import socket
import tempfile
import types

import numpy as np
import pytest

from paper_2602_19873_gb300 import workloads as wl


class OracleOps:
    """The decomposition's device steps computed by the oracle and numpy on
    CPU tensors (the same contracts as domain.LibraryOps)."""

    def __init__(self, kind):
        self.kind = kind

    def keys(self, x, y, z, h, box, key, support):
        import torch
        import oracle as orc
        k = orc.keys(x.numpy(), y.numpy(), z.numpy(), box, key)
        return torch.from_numpy(k.astype(np.uint64).view(np.int64).copy())

    def histogram(self, keys, lo, shift, nbins):
        import torch
        k = keys.numpy().view(np.uint64)
        sel = k >= np.uint64(lo)
        b = (k[sel] - np.uint64(lo)) >> np.uint64(shift)
        b = b[b < np.uint64(nbins)].astype(np.int64)
        return torch.from_numpy(np.bincount(b, minlength=nbins).astype(np.int64))

    def owner_mask(self, keys, splitters, P):
        import torch
        k = keys.numpy().view(np.uint64)
        own = np.searchsorted(np.array(splitters, np.uint64), k, side="right")
        return torch.from_numpy((np.uint64(1) << own.astype(np.uint64)).view(np.int64))

    def box(self, x, y, z, h, support):
        import torch
        if x.numel() == 0:
            return torch.tensor([np.inf] * 3 + [0.0] + [-np.inf] * 3 + [0.0], dtype=torch.float32)
        r = (np.float32(support) * h.numpy()).astype(np.float32)
        lo = [float(a.min()) for a in (x, y, z)]
        hi = [float(a.max()) for a in (x, y, z)]
        return torch.tensor(lo + [float(r.max())] + hi + [0.0], dtype=torch.float32)

    def halo_mask(self, x, y, z, h, box, support, dom, P, self_rank):
        """Exact FP64 point-to-box distance with a relative margin far above
        FP32 rounding (sending more than needed is harmless)."""
        import torch
        p = np.stack([x.numpy(), y.numpy(), z.numpy()], 1).astype(np.float64)
        r = (np.float32(support) * h.numpy()).astype(np.float64)
        L = np.asarray(box["hi"], np.float64) - np.asarray(box["lo"], np.float64)
        per = np.asarray(box["periodic"]).astype(bool)
        d = dom.numpy().astype(np.float64)
        m = np.zeros(len(p), np.uint64)
        for q in range(P):
            if q == self_rank or not d[q, 0] <= d[q, 4]:
                continue
            lo, hi, rq = d[q, 0:3], d[q, 4:7], d[q, 3]
            g = np.maximum(0.0, np.maximum(lo - p, p - hi))
            for a in range(3):
                if per[a]:
                    for s in (-L[a], L[a]):
                        ga = np.maximum(0.0, np.maximum(lo[a] - (p[:, a] + s), (p[:, a] + s) - hi[a]))
                        g[:, a] = np.minimum(g[:, a], ga)
            near = (g ** 2).sum(1) <= (np.maximum(r, rq) * (1 + 1e-5)) ** 2
            m |= np.where(near, np.uint64(1) << np.uint64(q), np.uint64(0))
        return torch.from_numpy(m.view(np.int64))

    def group(self, mask, P):
        import torch
        m = mask.numpy().view(np.uint64)
        parts, counts = [], []
        for q in range(P):
            sel = np.nonzero((m >> np.uint64(q)) & np.uint64(1))[0]
            parts.append(sel)
            counts.append(len(sel))
        idx = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        return torch.from_numpy(idx.astype(np.int64)), counts

    def local_pass(self, x, y, z, h, m, box, params):
        import torch
        import oracle as orc
        xs, ys, zs, hs, ms = (a.numpy() for a in (x, y, z, h, m))
        k = orc.keys(xs, ys, zs, box, self.kind)
        perm = orc.sort(k)
        srt = [np.ascontiguousarray(a[perm]) for a in (xs, ys, zs, hs, ms)]
        g_off, g_idx = orc.gather_all(*srt[:4], box, params.support)
        rho_s = orc.density(*srt, box, g_off, g_idx, np.arange(len(perm)))
        rho = np.empty(len(perm))
        cnt = np.empty(len(perm), np.int32)
        rho[perm] = rho_s
        cnt[perm] = np.diff(g_off)
        return torch.from_numpy(rho), torch.from_numpy(cnt), {}


def _rank_main(rank, world, port, case, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2602_19873_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = _case(case)
    n = len(d["x"])
    # an arbitrary initial distribution: a seeded random split of the particles
    owner0 = np.random.default_rng(77).integers(0, world, n)
    ids = np.nonzero(owner0 == rank)[0]
    t = {a: torch.from_numpy(np.ascontiguousarray(np.asarray(d[a], np.float32)[ids]))
         for a in "xyzhm"}
    params = types.SimpleNamespace(support=float(d["support"]), key=d["kind"])
    res = domain.decomposed_density(domain.Comm(), OracleOps(d["kind"]), torch.from_numpy(ids),
                                    t["x"], t["y"], t["z"], t["h"], t["m"], d["box"], d["kind"],
                                    params)
    np.savez(os.path.join(out_dir, "r%d.npz" % rank), ids=res["ids"].numpy(),
             rho=res["rho"].numpy(), counts=res["counts"].numpy(),
             splitters=np.array(res["splitters"], np.uint64), n_halo=res["n_halo"],
             n_global=res["n_global"])
    dist.barrier()
    dist.destroy_process_group()


def _case(case):
    if case == "plummer":
        return wl.plummer(6001, n_spheres=3, seed=61, n_target=40)
    if case == "uniform":
        return wl.uniform(5003, seed=62, n_target=40)
    raise KeyError(case)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case,world", [("plummer", 2), ("uniform", 2), ("uniform", 3)])
def test_decomposition_matches_single_domain(orc, case, world):
    import torch.multiprocessing as mp
    d = _case(case)
    n = len(d["x"])
    with tempfile.TemporaryDirectory() as tmp:
        mp.start_processes(_rank_main, args=(world, _free_port(), case, tmp), nprocs=world,
                           join=True, start_method="spawn")
        res = [dict(np.load(os.path.join(tmp, "r%d.npz" % r))) for r in range(world)]
    # every particle owned exactly once
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(n))
    assert all(int(r["n_global"]) == n for r in res)
    # contiguous ascending key ranges, balanced counts
    keys = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    split = res[0]["splitters"]
    assert all(np.array_equal(r["splitters"], split) for r in res)
    for q, r in enumerate(res):
        k = keys[r["ids"]]
        lo = split[q - 1] if q > 0 else np.uint64(0)
        assert np.all(k >= lo)
        if q < world - 1:
            assert np.all(k < split[q])
        assert abs(len(r["ids"]) - n / world) <= 0.02 * n
    # densities and counts equal the single-domain oracle's
    perm = orc.sort(keys)
    srt = [np.ascontiguousarray(np.asarray(d[a], np.float32)[perm]) for a in "xyzhm"]
    g_off, g_idx = orc.gather_all(*srt[:4], d["box"], d["support"])
    rho_s = orc.density(*srt, d["box"], g_off, g_idx, np.arange(n))
    rho = np.empty(n)
    cnt = np.empty(n, np.int64)
    rho[perm] = rho_s
    cnt[perm] = np.diff(g_off)
    for r in res:
        assert np.array_equal(r["counts"], cnt[r["ids"]])
        assert np.max(np.abs(r["rho"] - rho[r["ids"]]) / rho[r["ids"]]) <= 1e-12
        assert int(r["n_halo"]) > 0
