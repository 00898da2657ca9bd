"""The allocation-free SFC ordering entry point (nl_sfc_order_noalloc), for
callers that cannot allocate device memory where they need the order (a
simulation loop that cannot afford cudaMalloc's implicit synchronisation, or
a framework that owns all device memory and forbids driver allocations).

It must return the same keys and permutation as the allocating path
(nl_build followed by nl_copy_sorted), bit for bit, on two calls in a row
that share its fixed scratch array.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _reference(d, t):
    p = nl.make_params(key=d["kind"], cluster=8, support=d["support"])
    L = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    keys, perm = L.sorted()
    L.free()
    return keys, perm.astype(np.uint32)


def _noalloc(d, t):
    import torch
    n = len(d["x"])
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nl.sfc_order_noalloc(t["x"], t["y"], t["z"], t["h"], d["box"], d["kind"], d["support"],
                         keys, perm)
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32)


def _dev(d):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda()
            for k in ("x", "y", "z", "h")}


def test_noalloc_matches_allocating_path_on_two_calls():
    first = wl.plummer(200003, n_spheres=4, seed=301, n_target=60.0)     # Hilbert, open box
    second = wl.uniform(nl.NL_NOALLOC_MAX_N - 5, seed=302, n_target=60.0)  # Morton, periodic
    for d in (first, second):
        t = _dev(d)
        want_keys, want_perm = _reference(d, t)
        got_keys, got_perm = _noalloc(d, t)
        assert np.array_equal(got_keys, want_keys)
        assert np.array_equal(got_perm, want_perm)


def test_noalloc_rejects_oversize_and_bad_input():
    import torch
    n = nl.NL_NOALLOC_MAX_N + 1
    z = torch.zeros(n, dtype=torch.float32, device="cuda")
    h = torch.ones(n, dtype=torch.float32, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    box = {"lo": [0, 0, 0], "hi": [1, 1, 1], "periodic": [0, 0, 0]}
    with pytest.raises(nl.NLError) as e:
        nl.sfc_order_noalloc(z, z, z, h, box, 1, 2.0, keys, perm)
    assert e.value.status == 1 and "NL_NOALLOC_MAX_N" in str(e.value)
    # a NaN coordinate is reported, and the next good call still succeeds
    d = wl.uniform(5000, seed=303)
    t = _dev(d)
    t["x"][17] = float("nan")
    with pytest.raises(nl.NLError) as e:
        _noalloc(d, t)
    assert e.value.status == 1
    d = wl.uniform(5000, seed=304)
    t = _dev(d)
    want_keys, want_perm = _reference(d, t)
    got_keys, got_perm = _noalloc(d, t)
    assert np.array_equal(got_keys, want_keys) and np.array_equal(got_perm, want_perm)
