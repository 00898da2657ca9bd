"""The batched step as a CUDA graph, and the autotuner.

A replay of the captured build + density step must give exactly the density
of a normal build of the same inputs (same kernels, same order), follow new
input values written in place between replays, and report a capacity
overflow through nl_graph_check instead of returning silently wrong data."""
import numpy as np
import pytest

from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _batch(seed, n_systems=12, log_n=(2.7, 3.7)):
    import torch
    systems = wl.batched(n_systems=n_systems, seed=seed, log_n=log_n)
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    dev = {k: torch.from_numpy(np.concatenate([d[k] for d in systems]).astype(np.float32)).cuda()
           for k in "xyzhm"}
    return systems, offs, dev


def _normal_density(dev, offs, boxes, p, stream):
    import torch
    L = nl.NeighborList().build_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs, boxes, p,
                                      stream)
    rho = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    L.density_pass(dev["m"], rho, stream)
    stream.synchronize()
    L.free()
    return rho.cpu().numpy()


def test_graph_replay_matches_normal_build():
    import torch
    stream = torch.cuda.Stream()
    systems, offs, dev = _batch(501)
    boxes = [d["box"] for d in systems]
    p = nl.make_params(key=1, cluster=8, support=2.0)
    with torch.cuda.stream(stream):
        rho = torch.zeros(int(offs[-1]), dtype=torch.float32, device="cuda")
        L = nl.NeighborList()
        G = nl.Graph(L, dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], rho, offs, boxes, p,
                     stream)
        want = _normal_density(dev, offs, boxes, p, stream)
        rho.zero_()
        for _ in range(3):
            G.launch(stream)
        G.check(stream)
        assert np.array_equal(rho.cpu().numpy(), want)
        # new values written in place: the replay follows them
        g = torch.Generator(device="cuda").manual_seed(3)
        for a, k in enumerate("xyz"):
            lo = torch.from_numpy(np.repeat([b["lo"][a] for b in boxes], np.diff(offs))).cuda()
            hi = torch.from_numpy(np.repeat([b["hi"][a] for b in boxes], np.diff(offs))).cuda()
            j = (torch.rand(dev[k].shape, generator=g, device="cuda") - 0.5) * 1e-4
            dev[k].copy_(torch.minimum(torch.maximum(dev[k] + j * (hi - lo), lo), hi))
        want2 = _normal_density(dev, offs, boxes, p, stream)
        G.launch(stream)
        G.check(stream)
        assert np.array_equal(rho.cpu().numpy(), want2)
        assert L.sizes()["n_entries"] > 0
        # lists that outgrow the reserved buffers are reported
        dev["h"].mul_(3.0)
        G.launch(stream)
        with pytest.raises(nl.NLError) as e:
            G.check(stream)
        assert e.value.status in (2, 5)   # radius limit on a periodic cube, or capacity
        G.free()
        L.free()


@pytest.mark.parametrize("half", [0, 1])
def test_autotuner_returns_a_valid_faster_choice(half):
    import torch
    stream = torch.cuda.Stream()
    systems, offs, dev = _batch(511, n_systems=6, log_n=(3.0, 3.8))
    boxes = [d["box"] for d in systems]
    base = nl.make_params(key=1, cluster=8, support=2.0, half_list=half)
    with torch.cuda.stream(stream):
        best, ms = nl.autotune_batch(dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], offs, boxes,
                                     base, reps=1, stream=stream)
        assert best.cluster in (4, 8, 16) and best.threads_per_block in (128, 256)
        assert best.j_cluster in (best.cluster, best.cluster // 2) and best.j_cluster >= 4
        assert best.half_list == half
        if half:  # half lists need j-clusters of the i-cluster size
            assert best.j_cluster == best.cluster
        assert best.blocks_per_sm in (2, 3, 4) and ms > 0
        # the tuned parameters give the same densities within the FP32 tolerance
        a = _normal_density(dev, offs, boxes, base, stream)
        b = _normal_density(dev, offs, boxes, best, stream)
        assert np.max(np.abs(a - b) / a) < 2e-5


def test_graph_after_staging_growth(monkeypatch):
    """A build whose staging overflowed grows the per-slot capacity during
    redo rounds on a smaller grid; the captured graph then runs the full
    grid.  Its replays must stay within the staging arrays and match a
    normal build."""
    import torch
    monkeypatch.setenv("NLGB_STAGE_CAP0", "64")
    monkeypatch.setenv("NLGB_LIST_CAP0", "100000")
    stream = torch.cuda.Stream()
    systems, offs, dev = _batch(521, n_systems=6)
    boxes = [d["box"] for d in systems]
    p = nl.make_params(key=1, cluster=8, support=2.0)
    with torch.cuda.stream(stream):
        rho = torch.zeros(int(offs[-1]), dtype=torch.float32, device="cuda")
        L = nl.NeighborList()
        G = nl.Graph(L, dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], rho, offs, boxes, p,
                     stream)
        want = _normal_density(dev, offs, boxes, p, stream)
        rho.zero_()
        for _ in range(2):
            G.launch(stream)
        G.check(stream)
        assert np.array_equal(rho.cpu().numpy(), want)
        G.free()
        L.free()
