"""The SFC domain decomposition on the GPU (Sec. I key-range domains,
Sec. IV halos): its device steps through the C ABI against plain
definitions, and a whole decomposition run by two ranks -- two processes
sharing this GPU, exchanging over gloo on the host (no kernel waits on
another) -- against the single-domain oracle."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _dev(d):
    import torch
    return {a: torch.from_numpy(np.ascontiguousarray(np.asarray(d[a], np.float32))).cuda()
            for a in "xyzhm"}


@pytest.mark.parametrize("case", ["plummer", "uniform"])
def test_device_steps(case):
    import torch
    from paper_2602_19873_gb300 import domain
    d = (wl.plummer(20011, n_spheres=3, seed=71, n_target=50) if case == "plummer"
         else wl.uniform(17003, seed=72, n_target=50))
    n = len(d["x"])
    t = _dev(d)
    ops = domain.LibraryOps()
    keys = ops.keys(t["x"], t["y"], t["z"], t["h"], d["box"], d["kind"], d["support"])
    want = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    k = keys.cpu().numpy().view(np.uint64)
    assert np.array_equal(k, want)
    # histograms: top 16 bits, then 16 bits inside one bucket
    h1 = ops.histogram(keys, 0, 47, 1 << 16).cpu().numpy()
    assert np.array_equal(h1, np.bincount((k >> np.uint64(47)).astype(np.int64), minlength=1 << 16))
    b = int(np.argmax(h1))
    h2 = ops.histogram(keys, b << 47, 31, 1 << 16).cpu().numpy()
    sel = (k >> np.uint64(47)) == np.uint64(b)
    assert np.array_equal(h2, np.bincount(((k[sel] >> np.uint64(31)) & np.uint64(0xffff)).astype(np.int64),
                                          minlength=1 << 16))
    # owners from three splitters, grouped stably
    split = sorted(int(v) for v in np.sort(k)[[n // 4, n // 2, 3 * n // 4]])
    own = np.searchsorted(np.array(split, np.uint64), k, side="right")
    mask = ops.owner_mask(keys, split, 4)
    assert np.array_equal(mask.cpu().numpy().view(np.uint64), np.uint64(1) << own.astype(np.uint64))
    idx, counts = ops.group(mask, 4)
    assert counts == [int(np.sum(own == q)) for q in range(4)]
    assert np.array_equal(idx.cpu().numpy(), np.concatenate([np.nonzero(own == q)[0] for q in range(4)]))
    # box of rank 0's particles, then halo masks of the others against it
    r0 = torch.from_numpy(np.nonzero(own == 0)[0]).cuda()
    sub = {a: t[a].index_select(0, r0) for a in "xyzh"}
    bx = ops.box(sub["x"], sub["y"], sub["z"], sub["h"], d["support"]).cpu().numpy()
    x0 = np.stack([np.asarray(d[a], np.float32)[own == 0] for a in "xyz"], 1)
    assert np.array_equal(bx[0:3], x0.min(0)) and np.array_equal(bx[4:7], x0.max(0))
    assert bx[3] == np.max(np.float32(d["support"]) * np.asarray(d["h"], np.float32)[own == 0])
    dom = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    dom[0] = torch.from_numpy(bx).cuda()
    dom[1:, 0:3], dom[1:, 4:7] = float("inf"), float("-inf")     # empty boxes are skipped
    hm = ops.halo_mask(t["x"], t["y"], t["z"], t["h"], d["box"], d["support"], dom, 4, 1)
    hm = hm.cpu().numpy().view(np.uint64)
    assert np.all((hm & ~np.uint64(1)) == 0)
    # every particle of the other ranks with a symmetric neighbor in rank 0
    # must be flagged (brute force with the canonical predicate)
    o = np.nonzero(own != 0)[0]
    ks = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    perm = orc.sort(ks)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    srt = [np.ascontiguousarray(np.asarray(d[a], np.float32)[perm]) for a in "xyzh"]
    p_off, p_idx = orc.brute_neighbors(*srt, d["box"], d["support"], 1, inv[o])
    need = np.array([np.any(own[perm[p_idx[p_off[q]:p_off[q + 1]]]] == 0) for q in range(len(o))])
    assert need.any()
    assert np.all(hm[o][need] == 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(case):
    if case == "plummer":
        return wl.plummer(60013, n_spheres=4, seed=73, n_target=60)
    return wl.uniform(50021, seed=74, n_target=60)


def _rank_main(rank, world, port, case, half, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2602_19873_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = _case(case)
    n = len(d["x"])
    ids = np.nonzero(np.random.default_rng(75).integers(0, world, n) == rank)[0]
    t = {a: torch.from_numpy(np.ascontiguousarray(np.asarray(d[a], np.float32)[ids])).cuda()
         for a in "xyzhm"}
    p = nl.make_params(key=d["kind"], cluster=8, support=d["support"], half_list=half)
    res = domain.decomposed_density(domain.Comm(), domain.LibraryOps(),
                                    torch.from_numpy(ids).cuda(), t["x"], t["y"], t["z"], t["h"],
                                    t["m"], d["box"], d["kind"], p)
    torch.cuda.synchronize()
    np.savez(os.path.join(out_dir, "r%d.npz" % rank), ids=res["ids"].cpu().numpy(),
             rho=res["rho"].cpu().numpy(), counts=res["counts"].cpu().numpy(),
             n_halo=res["n_halo"])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,half", [("plummer", 1), ("uniform", 0)])
def test_two_ranks_match_single_domain(case, half):
    import torch.multiprocessing as mp
    from nlcheck import DENSITY_RTOL
    d = _case(case)
    n = len(d["x"])
    with tempfile.TemporaryDirectory() as tmp:
        mp.start_processes(_rank_main, args=(2, _free_port(), case, half, tmp), nprocs=2,
                           join=True, start_method="spawn")
        res = [dict(np.load(os.path.join(tmp, "r%d.npz" % r))) for r in range(2)]
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(n))
    keys = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    perm = orc.sort(keys)
    srt = [np.ascontiguousarray(np.asarray(d[a], np.float32)[perm]) for a in "xyzhm"]
    g_off, g_idx = orc.gather_all(*srt[:4], d["box"], d["support"])
    rho = np.empty(n)
    cnt = np.empty(n, np.int64)
    rho[perm] = orc.density(*srt, d["box"], g_off, g_idx, np.arange(n))
    cnt[perm] = np.diff(g_off)
    for r in res:
        assert int(r["n_halo"]) > 0
        assert np.array_equal(r["counts"], cnt[r["ids"]])
        assert np.max(np.abs(r["rho"] - rho[r["ids"]]) / rho[r["ids"]]) <= DENSITY_RTOL
