"""A key sort whose look-back gave up its bounded wait ends the build with
NL_ERR_TIMEOUT, and the same handle builds correctly afterwards.  The stall
is reported through the library's test knob NLGB_SORT_STALL (the status word
is set on the host's stream, no wait runs out on the GPU)."""
import numpy as np
import pytest

from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import gpu_density, to_dev

pytestmark = pytest.mark.gpu


def test_sort_stall_is_reported_and_the_handle_recovers(monkeypatch):
    import torch
    d = wl.uniform(20000, seed=31, n_target=60.0)
    t = to_dev(d)
    p = nl.make_params(key=d["kind"], cluster=8, support=d["support"])
    L = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    monkeypatch.setenv("NLGB_SORT_STALL", "1")
    for _ in range(2):  # a fresh build and a rebuild of the kept handle
        with pytest.raises(nl.NLError) as err:
            nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p) if _ == 0 else \
                L.build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
        assert err.value.status == 7  # NL_ERR_TIMEOUT
    monkeypatch.delenv("NLGB_SORT_STALL")
    L.build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    torch.cuda.synchronize()
    ref = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    n = len(d["x"])
    assert np.array_equal(gpu_density(L, t, n), gpu_density(ref, t, n))
    L.free()
    ref.free()
