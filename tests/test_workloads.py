"""The seeded input generators and their cache (no method arithmetic)."""
import numpy as np


def test_workload_cache_round_trips_dicts_and_lists(tmp_path, monkeypatch):
    """The generator cache returns what the generator returned, for a single
    system (dict) and a batch (list of dicts), on the first and later calls."""
    import tempfile
    from paper_2602_19873_gb300 import workloads as wl
    monkeypatch.setattr(tempfile, "gettempdir", lambda: str(tmp_path))
    for key, fn, args in (("one", wl.uniform, (300,)), ("many", wl.batched, (3,))):
        a = wl.cached(fn, key, *args, seed=7)
        b = wl.cached(fn, key, *args, seed=7)
        aa = a if isinstance(a, list) else [a]
        bb = b if isinstance(b, list) else [b]
        assert type(a) is type(b) and len(aa) == len(bb)
        for x, y in zip(aa, bb):
            assert np.array_equal(x["x"], y["x"]) and np.array_equal(x["h"], y["h"])
