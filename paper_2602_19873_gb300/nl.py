"""Python binding of the C ABI in include/nl.h (argument marshalling only).

Functions keep the C names and take torch CUDA tensors (float32/int32
contiguous) or raw device pointers; every step of the path runs in
libnlgb.so.  The first call loads the library and raises NLError when it is
missing, when no CUDA device is visible, or when a call fails.  Inspection
helpers return numpy arrays.
"""
import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

NL_OK = 0
NL_KEY_MORTON, NL_KEY_HILBERT = 0, 1
STATUS_NAMES = {0: "NL_OK", 1: "NL_ERR_ARG", 2: "NL_ERR_RADIUS", 3: "NL_ERR_OOM", 4: "NL_ERR_CUDA",
                5: "NL_ERR_CAPACITY", 6: "NL_ERR_NOT_CONVERGED", 7: "NL_ERR_TIMEOUT",
                8: "NL_ERR_UNIMPLEMENTED"}


class NLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class nl_box(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("periodic", C.c_int32 * 3)]


class nl_params(C.Structure):
    _fields_ = [("key", C.c_int32), ("cluster", C.c_int32), ("support", C.c_float),
                ("compress", C.c_int32), ("leaf_bucket", C.c_int32),
                ("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("j_cluster", C.c_int32), ("half_list", C.c_int32)]


class nl_sizes(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_clusters", C.c_int64), ("n_superclusters", C.c_int64),
                ("n_leaves", C.c_int64), ("n_nodes", C.c_int64), ("n_entries", C.c_int64),
                ("n_tiles", C.c_int64), ("list_bytes", C.c_int64), ("cluster", C.c_int32),
                ("compress", C.c_int32), ("node_visits", C.c_int64), ("leaf_visits", C.c_int64),
                ("j_examined", C.c_int64), ("tile_tests", C.c_int64), ("j_cluster", C.c_int32),
                ("pad0", C.c_int32)]


P = C.c_void_p
_SIGS = {
    "nl_default_params": (None, [P]),
    "nl_last_error": (C.c_char_p, []),
    "nl_build": (C.c_int, [P, P, P, P, C.c_int64, P, P, P, P]),
    "nl_rebuild": (C.c_int, [P, P, P, P, P, C.c_int64, P, P, P]),
    "nl_density_pass": (C.c_int, [P, P, P, P]),
    "nl_neighbor_counts": (C.c_int, [P, P, P]),
    "nl_force_pass": (C.c_int, [P, C.c_int32, P, P, P, P, P, P, P, P]),
    "nl_refresh_positions": (C.c_int, [P, P, P, P, P, P]),
    "nl_nearest_distance": (C.c_int, [P, P, P]),
    "nl_free": (C.c_int, [P]),
    "nl_get_sizes": (C.c_int, [P, P]),
    "nl_copy_sorted": (C.c_int, [P, P, P]),
    "nl_copy_octree": (C.c_int, [P, P, P, P, P, P]),
    "nl_copy_records": (C.c_int, [P, P, P]),
    "nl_create": (C.c_int, [P]),
    "nl_set_profiling": (C.c_int, [P, C.c_int32]),
    "nl_get_stage_times": (C.c_int, [P, P, C.c_int32, P]),
    "nl_density_from_host": (C.c_int, [P, P, P, P, P, P, C.c_int64, P, P, P, P]),
    "nl_sfc_order_noalloc": (C.c_int, [P, P, P, P, C.c_int64, P, C.c_int32, C.c_float, P, P,
                                        P]),
    "nl_build_batch": (C.c_int, [P, P, P, P, C.c_int32, P, P, P, P, P]),
    "nl_rebuild_batch": (C.c_int, [P, P, P, P, P, C.c_int32, P, P, P, P]),
    "nl_iterate_h_batch": (C.c_int, [P, P, P, P, P, C.c_int32, P, P, P, C.c_float, C.c_float,
                                     C.c_int32, C.c_float, C.c_int32, P, P, P]),
    "nl_graph_create": (C.c_int, [P, P, P, P, P, P, P, C.c_int32, P, P, P, P, P]),
    "nl_graph_launch": (C.c_int, [P, P]),
    "nl_graph_check": (C.c_int, [P, P]),
    "nl_graph_free": (C.c_int, [P]),
    "nl_autotune_batch": (C.c_int, [P, P, P, P, P, C.c_int32, P, P, P, C.c_int32, P, P, P]),
    "nl_mlp_nparams": (C.c_int64, []),
    "nl_mlp_create": (C.c_int, [C.c_uint64, P]),
    "nl_mlp_free": (C.c_int, [P]),
    "nl_mlp_get_params": (C.c_int, [P, P]),
    "nl_mlp_set_params": (C.c_int, [P, P]),
    "nl_mlp_features": (C.c_int, [P, P, P, P]),
    "nl_mlp_targets": (C.c_int, [P, P, P, P, P, P]),
    "nl_mlp_grad": (C.c_int, [P, P, P, P, C.c_int64, P, P, P]),
    "nl_mlp_train": (C.c_int, [P, P, P, P, C.c_int64, C.c_int32, C.c_int32, C.c_float,
                               C.c_uint64, P, P]),
    "nl_mlp_predict": (C.c_int, [P, P, C.c_int64, P, P]),
    "nl_set_mlp": (C.c_int, [P, P]),
    "nl_probe_fp32_rate": (C.c_int, [C.c_int32, C.c_int32, P, P, P]),
    "nl_get_hiter_trace": (C.c_int, [P, P, C.c_int32, P]),
    "nl_sfc_keys": (C.c_int, [P, P, P, P, C.c_int64, P, C.c_int32, C.c_float, P, P]),
    "nl_key_histogram": (C.c_int, [P, C.c_int64, C.c_uint64, C.c_int32, C.c_int32, P, P]),
    "nl_domain_owner_mask": (C.c_int, [P, C.c_int64, P, C.c_int32, P, P]),
    "nl_domain_box": (C.c_int, [P, P, P, P, C.c_int64, C.c_float, P, P]),
    "nl_domain_halo_mask": (C.c_int, [P, P, P, P, C.c_int64, P, C.c_float, P, C.c_int32,
                                      C.c_int32, P, P]),
    "nl_domain_count": (C.c_int, [P, C.c_int64, C.c_int32, P, P]),
    "nl_domain_group": (C.c_int, [P, C.c_int64, C.c_int32, P, P, P]),
    "nl_iterate_h": (C.c_int, [P, P, P, P, P, C.c_int64, P, P, C.c_float, C.c_float, C.c_int32,
                               C.c_float, C.c_int32, P, P, P]),
}

NL_HSTART_GIVEN, NL_HSTART_PLAIN, NL_HSTART_LEARNED = 0, 1, 2
NL_FORCE_SPH_PRESSURE, NL_FORCE_LJ, NL_FORCE_LJ_COULOMB = 0, 1, 2


class nl_hiter_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("rebuilds", C.c_int32), ("unconverged", C.c_int64)]


class nl_hiter_step(C.Structure):
    _fields_ = [("rebuilt", C.c_int32), ("pad0", C.c_int32), ("active", C.c_int64),
                ("unconverged", C.c_int64), ("entries", C.c_int64), ("tiles", C.c_int64),
                ("ms", C.c_float), ("pad1", C.c_int32)]

STAGES = ["keys", "sort", "permute", "octree", "search", "assemble", "pass_gather", "pass"]


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libnlgb.so (building it first when asked) and bind signatures."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise NLError(8, "native library %s is missing; run build()" % path)
            lib = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st):
    if st != NL_OK:
        raise NLError(st, load().nl_last_error().decode())


def _ptr(t):
    """Device pointer of a torch tensor (or an int pointer / None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_box(box):
    b = nl_box()
    for a in range(3):
        b.lo[a] = float(np.float32(box["lo"][a]))
        b.hi[a] = float(np.float32(box["hi"][a]))
        b.periodic[a] = int(box["periodic"][a])
    return b


def make_params(key=NL_KEY_HILBERT, cluster=8, support=2.0, compress=1, leaf_bucket=256,
                threads_per_block=0, blocks_per_sm=0, j_cluster=0, half_list=0):
    """Build options; j_cluster 0 means j-clusters of `cluster` particles;
    half_list 1 stores every cluster pair once."""
    p = nl_params()
    load().nl_default_params(C.byref(p))
    p.key, p.cluster, p.support = int(key), int(cluster), float(support)
    p.compress, p.leaf_bucket = int(compress), int(leaf_bucket)
    p.threads_per_block, p.blocks_per_sm = int(threads_per_block), int(blocks_per_sm)
    p.j_cluster, p.half_list = int(j_cluster), int(half_list)
    return p


def params_dict(p):
    return {f: getattr(p, f) for f, _ in nl_params._fields_}


NL_NOALLOC_MAX_N = 1048576


def _require(t, name, dtype, n):
    """A contiguous CUDA tensor of `dtype` with at least n elements."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must have dtype %s, not %s" % (name, dtype, t.dtype))
    if t.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), n))


def sfc_order_noalloc(x, y, z, h, box, key, support, keys, perm, stream=None):
    """nl_sfc_order_noalloc: keys (int64 tensor viewed as uint64) and perm
    (int32 tensor) are caller-owned CUDA outputs of n entries."""
    import torch
    n = int(x.numel()) if hasattr(x, "numel") else 0
    for name, t in (("x", x), ("y", y), ("z", z), ("h", h)):
        _require(t, name, torch.float32, n)
    _require(keys, "keys", torch.int64, n)
    _require(perm, "perm", torch.int32, n)
    b = make_box(box) if isinstance(box, dict) else box
    _check(load().nl_sfc_order_noalloc(_ptr(x), _ptr(y), _ptr(z), _ptr(h), int(x.numel()),
                                       C.byref(b), int(key), float(support), _ptr(keys),
                                       _ptr(perm), _stream(stream)))


def autotune_batch(x, y, z, h, m, offsets, boxes, base, reps=2, stream=None):
    """nl_autotune_batch: returns (best nl_params, mean ms)."""
    nsys = len(boxes)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    barr = (nl_box * nsys)(*[make_box(b) for b in boxes])
    best = nl_params()
    ms = C.c_float()
    _check(load().nl_autotune_batch(_ptr(x), _ptr(y), _ptr(z), _ptr(h), _ptr(m), nsys,
                                    offs.ctypes.data, barr, C.byref(base), int(reps),
                                    C.byref(best), C.byref(ms), _stream(stream)))
    return best, ms.value


class Graph:
    """nl_graph: one captured build + density step of a batch."""

    def __init__(self, nlist, x, y, z, h, m, rho, offsets, boxes, params, stream):
        nlist.ensure_handle()
        nsys = len(boxes)
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        barr = (nl_box * nsys)(*[make_box(b) for b in boxes])
        self.handle = C.c_void_p()
        self.nlist = nlist
        _check(load().nl_graph_create(nlist.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(h), _ptr(m),
                                      _ptr(rho), nsys, offs.ctypes.data, barr, C.byref(params),
                                      _stream(stream), C.byref(self.handle)))

    def launch(self, stream=None):
        _check(load().nl_graph_launch(self.handle, _stream(stream)))

    def check(self, stream=None):
        _check(load().nl_graph_check(self.handle, _stream(stream)))

    def free(self):
        if self.handle:
            load().nl_graph_free(self.handle)
            self.handle = None


class MLP:
    """nl_mlp: the smoothing-length network (device parameters)."""

    def __init__(self, seed=0):
        self.handle = C.c_void_p()
        _check(load().nl_mlp_create(int(seed), C.byref(self.handle)))

    @staticmethod
    def nparams():
        return int(load().nl_mlp_nparams())

    def get_params(self):
        out = np.zeros(self.nparams(), np.float32)
        _check(load().nl_mlp_get_params(self.handle, out.ctypes.data))
        return out

    def set_params(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32)
        assert len(arr) == self.nparams()
        _check(load().nl_mlp_set_params(self.handle, arr.ctypes.data))

    def grad(self, X, y, w, grad_out, stream=None):
        loss = C.c_float()
        _check(load().nl_mlp_grad(self.handle, _ptr(X), _ptr(y), _ptr(w), int(y.numel()),
                                  _ptr(grad_out), C.byref(loss), _stream(stream)))
        return loss.value

    def train(self, X, y, w, epochs, batch=4096, lr=3e-3, seed=0, stream=None):
        loss = C.c_float()
        _check(load().nl_mlp_train(self.handle, _ptr(X), _ptr(y), _ptr(w), int(y.numel()),
                                   int(epochs), int(batch), float(lr), int(seed), C.byref(loss),
                                   _stream(stream)))
        return loss.value

    def predict(self, X, out, stream=None):
        _check(load().nl_mlp_predict(self.handle, _ptr(X), int(out.numel()), _ptr(out),
                                     _stream(stream)))

    def free(self):
        if self.handle:
            load().nl_mlp_free(self.handle)
            self.handle = None


class NeighborList:
    """Owner of one nl_list handle.  Positions x, y, z and smoothing lengths h
    are float32 CUDA tensors in caller order."""

    def __init__(self):
        self.handle = None

    def build(self, x, y, z, h, box, params, stream=None):
        L = load()
        b = make_box(box) if isinstance(box, dict) else box
        n = int(x.numel())
        if self.handle is None:
            out = C.c_void_p()
            _check(L.nl_build(_ptr(x), _ptr(y), _ptr(z), _ptr(h), n, C.byref(b), C.byref(params),
                              _stream(stream), C.byref(out)))
            self.handle = out
        else:
            _check(L.nl_rebuild(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(h), n, C.byref(b),
                                C.byref(params), _stream(stream)))
        return self

    def build_batch(self, x, y, z, h, offsets, boxes, params, stream=None):
        """Batch of systems back to back in x..h; offsets: nsys+1 ints;
        boxes: list of box dicts."""
        L = load()
        nsys = len(boxes)
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        assert len(offs) == nsys + 1
        barr = (nl_box * nsys)(*[make_box(b) for b in boxes])
        if self.handle is None:
            out = C.c_void_p()
            _check(L.nl_build_batch(_ptr(x), _ptr(y), _ptr(z), _ptr(h), nsys, offs.ctypes.data,
                                    barr, C.byref(params), _stream(stream), C.byref(out)))
            self.handle = out
        else:
            _check(L.nl_rebuild_batch(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(h), nsys,
                                      offs.ctypes.data, barr, C.byref(params), _stream(stream)))
        return self

    def iterate_h_batch(self, x, y, z, h, offsets, boxes, params, n_target, tol=2.0, max_iter=40,
                        margin=0.15, start=1, converged=None, stream=None, check=True):
        self.ensure_handle()
        nsys = len(boxes)
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        barr = (nl_box * nsys)(*[make_box(b) for b in boxes])
        info = nl_hiter_info()
        st = load().nl_iterate_h_batch(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(h), nsys,
                                       offs.ctypes.data, barr, C.byref(params), float(n_target),
                                       float(tol), int(max_iter), float(margin), int(start),
                                       _ptr(converged), C.byref(info), _stream(stream))
        out = {"iterations": info.iterations, "rebuilds": info.rebuilds,
               "unconverged": info.unconverged, "status": st}
        if st != NL_OK and (check or st != 6):
            _check(st)
        return out

    def ensure_handle(self):
        if self.handle is None:
            out = C.c_void_p()
            _check(load().nl_create(C.byref(out)))
            self.handle = out
        return self

    def set_profiling(self, on=True):
        self.ensure_handle()
        _check(load().nl_set_profiling(self.handle, 1 if on else 0))

    def stage_times(self):
        ms = (C.c_float * 16)()
        cnt = C.c_int32()
        _check(load().nl_get_stage_times(self.handle, ms, 16, C.byref(cnt)))
        return {STAGES[k]: float(ms[k]) for k in range(cnt.value)}

    def density_from_host(self, x, y, z, h, m, box, params, rho, stream=None):
        """x..m, rho: numpy float32 arrays (pinned or pageable host memory)."""
        self.ensure_handle()
        b = make_box(box) if isinstance(box, dict) else box
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z, h, m)]
        assert rho.dtype == np.float32 and rho.flags.c_contiguous
        _check(load().nl_density_from_host(self.handle, *[a.ctypes.data for a in arrs],
                                           len(arrs[0]), C.byref(b), C.byref(params),
                                           rho.ctypes.data, _stream(stream)))

    def iterate_h(self, x, y, z, h, box, params, n_target, tol=2.0, max_iter=40, margin=0.15,
                  start=NL_HSTART_PLAIN, converged=None, stream=None, check=True):
        """h: float32 CUDA tensor (in/out, caller order).  Returns the info
        dict; raises NLError on failure (NL_ERR_NOT_CONVERGED when check)."""
        self.ensure_handle()
        b = make_box(box) if isinstance(box, dict) else box
        info = nl_hiter_info()
        st = load().nl_iterate_h(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(h), int(x.numel()),
                                 C.byref(b), C.byref(params), float(n_target), float(tol),
                                 int(max_iter), float(margin), int(start), _ptr(converged),
                                 C.byref(info), _stream(stream))
        out = {"iterations": info.iterations, "rebuilds": info.rebuilds,
               "unconverged": info.unconverged, "status": st}
        if st != NL_OK and (check or st != 6):
            _check(st)
        return out

    def set_mlp(self, mlp):
        self.ensure_handle()
        _check(load().nl_set_mlp(self.handle, mlp.handle if mlp is not None else None))

    def mlp_features(self, stream=None):
        """(X [n_clusters x 8], e64 [n_superclusters]) CUDA tensors of this list."""
        import torch
        s = self.sizes()
        X = torch.empty((s["n_clusters"], 8), dtype=torch.float32, device="cuda")
        e64 = torch.empty(s["n_superclusters"], dtype=torch.float32, device="cuda")
        _check(load().nl_mlp_features(self.handle, _ptr(X), _ptr(e64), _stream(stream)))
        return X, e64

    def mlp_targets(self, h, e64, stream=None):
        import torch
        nc = self.sizes()["n_clusters"]
        y = torch.empty(nc, dtype=torch.float32, device="cuda")
        w = torch.empty(nc, dtype=torch.float32, device="cuda")
        _check(load().nl_mlp_targets(self.handle, _ptr(h), _ptr(e64), _ptr(y), _ptr(w),
                                     _stream(stream)))
        return y, w

    def density_pass(self, m, rho, stream=None):
        _check(load().nl_density_pass(self.handle, _ptr(m), _ptr(rho), _stream(stream)))

    def force_pass(self, kind, ax, ay, az, m=None, rho=None, pres=None, eps=1.0, sigma=1.0,
                   rc=0.0, kc=0.0, stream=None):
        """nl_force_pass; for NL_FORCE_LJ_COULOMB `m` carries the charges q."""
        prm = (C.c_float * 4)(float(eps), float(sigma), float(rc), float(kc))
        _check(load().nl_force_pass(self.handle, int(kind), prm, _ptr(m), _ptr(rho), _ptr(pres),
                                    _ptr(ax), _ptr(ay), _ptr(az), _stream(stream)))

    def neighbor_counts(self, counts, stream=None):
        _check(load().nl_neighbor_counts(self.handle, _ptr(counts), _stream(stream)))

    def nearest_distance(self, dist, stream=None):
        _check(load().nl_nearest_distance(self.handle, _ptr(dist), _stream(stream)))

    def refresh_positions(self, x, y, z, max_disp=None, stream=None):
        _check(load().nl_refresh_positions(self.handle, _ptr(x), _ptr(y), _ptr(z), _ptr(max_disp),
                                           _stream(stream)))

    def hiter_trace(self):
        """Per-pass records of the last h iteration (nl_get_hiter_trace)."""
        cnt = C.c_int32()
        _check(load().nl_get_hiter_trace(self.handle, None, 0, C.byref(cnt)))
        arr = (nl_hiter_step * max(1, cnt.value))()
        _check(load().nl_get_hiter_trace(self.handle, arr, cnt.value, C.byref(cnt)))
        return [{f: getattr(arr[i], f) for f, _ in nl_hiter_step._fields_ if not f.startswith("pad")}
                for i in range(cnt.value)]

    def sizes(self):
        s = nl_sizes()
        _check(load().nl_get_sizes(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in nl_sizes._fields_}

    def sorted(self):
        n = self.sizes()["n"]
        keys = np.zeros(n, np.uint64)
        perm = np.zeros(n, np.int32)
        _check(load().nl_copy_sorted(self.handle, keys.ctypes.data, perm.ctypes.data))
        return keys, perm

    def octree(self):
        nn = self.sizes()["n_nodes"]
        arrs = [np.zeros(nn, np.int32) for _ in range(5)]
        _check(load().nl_copy_octree(self.handle, *[a.ctypes.data for a in arrs]))
        return dict(zip(["level", "first", "end", "leaf", "skip"], arrs))

    def records(self):
        s = self.sizes()
        off = np.zeros(s["n_superclusters"], np.uint64)
        data = np.zeros(max(1, s["list_bytes"]), np.uint8)
        _check(load().nl_copy_records(self.handle, off.ctypes.data, data.ctypes.data))
        return off, data[:s["list_bytes"]]

    def free(self):
        if self.handle is not None:
            load().nl_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def probe_fp32_rate(packed=False, reps=5, stream=None):
    """nl_probe_fp32_rate: (FP32 element ops per second, ms of the best launch)."""
    ops = C.c_double()
    ms = C.c_double()
    _check(load().nl_probe_fp32_rate(int(bool(packed)), int(reps), C.byref(ops), C.byref(ms),
                                     _stream(stream)))
    return ops.value, ms.value


# ------------------------------------------------------------ domain decomposition
def sfc_keys(x, y, z, h, box, key, support, keys, stream=None):
    """nl_sfc_keys: keys (int64 CUDA tensor of n, viewed as uint64) of the
    particles in caller order."""
    import torch
    n = int(x.numel())
    for name, t in (("x", x), ("y", y), ("z", z), ("h", h)):
        _require(t, name, torch.float32, n)
    _require(keys, "keys", torch.int64, n)
    b = make_box(box) if isinstance(box, dict) else box
    _check(load().nl_sfc_keys(_ptr(x), _ptr(y), _ptr(z), _ptr(h), n, C.byref(b), int(key),
                              float(support), _ptr(keys), _stream(stream)))


def key_histogram(keys, lo, shift, nbins, hist, stream=None):
    """nl_key_histogram into hist (int64 CUDA tensor of nbins)."""
    import torch
    _require(keys, "keys", torch.int64, int(keys.numel()))
    _require(hist, "hist", torch.int64, int(nbins))
    _check(load().nl_key_histogram(_ptr(keys), int(keys.numel()), int(lo), int(shift), int(nbins),
                                   _ptr(hist), _stream(stream)))


def domain_owner_mask(keys, splitters, P, mask, stream=None):
    """nl_domain_owner_mask: splitters int64 CUDA tensor of P-1."""
    import torch
    n = int(keys.numel())
    _require(keys, "keys", torch.int64, n)
    _require(mask, "mask", torch.int64, n)
    if P > 1:
        _require(splitters, "splitters", torch.int64, P - 1)
    _check(load().nl_domain_owner_mask(_ptr(keys), n, _ptr(splitters) if P > 1 else None, int(P),
                                       _ptr(mask), _stream(stream)))


def domain_box(x, y, z, h, support, out, stream=None):
    """nl_domain_box into out (float32 CUDA tensor of 8)."""
    import torch
    n = int(x.numel())
    for name, t in (("x", x), ("y", y), ("z", z), ("h", h)):
        _require(t, name, torch.float32, n)
    _require(out, "out", torch.float32, 8)
    _check(load().nl_domain_box(_ptr(x), _ptr(y), _ptr(z), _ptr(h), n, float(support), _ptr(out),
                                _stream(stream)))


def domain_halo_mask(x, y, z, h, box, support, dom, P, self_rank, mask, stream=None):
    """nl_domain_halo_mask: dom float32 CUDA tensor [P, 8] (nl_domain_box rows)."""
    import torch
    n = int(x.numel())
    for name, t in (("x", x), ("y", y), ("z", z), ("h", h)):
        _require(t, name, torch.float32, n)
    _require(dom, "dom", torch.float32, 8 * int(P))
    _require(mask, "mask", torch.int64, n)
    b = make_box(box) if isinstance(box, dict) else box
    _check(load().nl_domain_halo_mask(_ptr(x), _ptr(y), _ptr(z), _ptr(h), n, C.byref(b),
                                      float(support), _ptr(dom), int(P), int(self_rank), _ptr(mask),
                                      _stream(stream)))


def domain_count(mask, P, counts, stream=None):
    import torch
    _require(mask, "mask", torch.int64, int(mask.numel()))
    _require(counts, "counts", torch.int64, int(P))
    _check(load().nl_domain_count(_ptr(mask), int(mask.numel()), int(P), _ptr(counts),
                                  _stream(stream)))


def domain_group(mask, P, offsets, idx, stream=None):
    """nl_domain_group: offsets int64 CUDA tensor of P, idx int32 CUDA tensor."""
    import torch
    _require(mask, "mask", torch.int64, int(mask.numel()))
    _require(offsets, "offsets", torch.int64, int(P))
    if not (isinstance(idx, torch.Tensor) and idx.is_cuda and idx.dtype == torch.int32):
        raise ValueError("idx must be an int32 CUDA tensor")
    _check(load().nl_domain_group(_ptr(mask), int(mask.numel()), int(P), _ptr(offsets), _ptr(idx),
                                  _stream(stream)))
