"""ctypes marshalling for nl_oracle.c (test infrastructure; see package doc).

Every function takes and returns numpy arrays.  Particle arrays passed to the
neighbor / pass functions are in SFC-sorted order (the oracle sorts with
``sort`` first); ``box`` is a dict ``{"lo": (3,), "hi": (3,), "periodic": (3,)}``.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nl_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "lib", "Box", "quantize", "morton3", "hilbert3", "hilbert3_inverse", "keys",
    "sort", "octree", "brute_neighbors", "gather_all", "symmetrize", "cluster_lists", "half_lists",
    "encode_block", "encode_record", "decode_record", "record_bytes", "stream_nibbles",
    "w", "dw", "W", "density", "sph_force", "lj_force", "lj_energy", "ljc_force", "ljc_energy",
    "nearest", "gather_counts_brute",
    "pred", "dist2", "dist2_row", "num_threads", "pipeline_lists", "mlp_nparams",
    "mlp_forward", "mlp_loss_grad", "mlp_features", "mlp_targets", "h_at_count",
    "computed_pairs", "cluster_overhead",
]


def build(force=False):
    """Compile nl_oracle.c with gcc (FP32 predicate without FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class Box(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("periodic", C.c_int32 * 3)]


def _box(b):
    out = Box()
    for a in range(3):
        out.lo[a] = float(np.float32(b["lo"][a]))
        out.hi[a] = float(np.float32(b["hi"][a]))
        out.periodic[a] = int(b["periodic"][a])
    return out


P = C.c_void_p
I64 = C.c_int64
F32 = C.c_float


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_OUT)
            sig = {
                "orc_quantize": (C.c_uint32, [F32, F32, F32]),
                "orc_morton3": (C.c_uint64, [C.c_uint32] * 3),
                "orc_hilbert3": (C.c_uint64, [C.c_uint32] * 3 + [C.c_int]),
                "orc_hilbert3_inverse": (None, [C.c_uint64, C.c_int, P]),
                "orc_keys": (None, [I64, P, P, P, P, C.c_int, P]),
                "orc_sort": (C.c_int, [I64, P, P]),
                "orc_octree": (I64, [I64, P, C.c_int, P, P, P, P, I64]),
                "orc_pred": (C.c_int, [P, P, P, P, F32, I64, I64, P, C.c_int]),
                "orc_dist2": (F32, [P, P, P, I64, I64, P]),
                "orc_csr_nnz": (I64, [P]),
                "orc_csr_copy": (None, [P, P, P]),
                "orc_csr_free": (None, [P]),
                "orc_csr_from": (P, [I64, P, P]),
                "orc_brute_neighbors": (P, [I64, P, P, P, P, P, F32, C.c_int, I64, P]),
                "orc_gather_all": (P, [I64, P, P, P, P, P, F32]),
                "orc_symmetrize": (P, [P]),
                "orc_cluster_lists": (P, [I64, C.c_int, C.c_int, P, P, I64, P]),
                "orc_clist_nnz": (I64, [P]),
                "orc_clist_copy": (None, [P, P, P, P]),
                "orc_clist_free": (None, [P]),
                "orc_encode_block": (None, [C.c_int, P, P, P, P, P, P]),
                "orc_stream_nibbles": (I64, [I64, P, C.c_int]),
                "orc_record_bytes": (I64, [I64, P, C.c_int, C.c_int]),
                "orc_encode_record": (I64, [I64, P, P, C.c_int, C.c_int, P]),
                "orc_decode_record": (I64, [P, C.c_int, C.c_int, P, P]),
                "orc_w": (C.c_double, [C.c_double]),
                "orc_dw": (C.c_double, [C.c_double]),
                "orc_W": (C.c_double, [C.c_double, C.c_double]),
                "orc_density": (None, [P, P, P, P, P, P, P, P, P]),
                "orc_sph_force": (None, [P] * 14),
                "orc_lj_force": (None, [P, P, P, P, C.c_double, C.c_double, P, P, P, P, P, P]),
                "orc_lj_energy": (C.c_double, [P, P, P, P, C.c_double, C.c_double, P]),
                "orc_ljc_force": (None, [P, P, P, P, C.c_double, C.c_double, P, C.c_double, P,
                                         P, P, P, P, P]),
                "orc_ljc_energy": (C.c_double, [P, P, P, P, C.c_double, C.c_double, P,
                                                C.c_double, P]),
                "orc_nearest": (None, [P, P, P, P, P, P]),
                "orc_gather_counts_brute": (None, [I64, P, P, P, P, P, F32, I64, P, P]),
                "orc_dist2_row": (None, [I64, P, P, P, P, I64, P]),
                "orc_num_threads": (C.c_int, []),
                "orc_mlp_nparams": (I64, []),
                "orc_mlp_forward": (None, [I64, P, P, P]),
                "orc_mlp_loss_grad": (C.c_double, [I64, P, P, P, P]),
                "orc_mlp_features": (C.c_int, [I64, P, P, P, P, C.c_int, P, P]),
                "orc_mlp_targets": (None, [I64, P, C.c_int, P, P, P]),
                "orc_h_at_count": (C.c_int, [I64, P, P, P, P, P, F32, C.c_int, P]),
                "orc_computed_pairs": (I64, [I64, P, C.c_int, C.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def num_threads():
    return lib().orc_num_threads()


# ----------------------------------------------------------------------------- keys
def quantize(x, lo, hi):
    return lib().orc_quantize(float(np.float32(x)), float(np.float32(lo)), float(np.float32(hi)))


def morton3(qx, qy, qz):
    return lib().orc_morton3(int(qx), int(qy), int(qz))


def hilbert3(qx, qy, qz, bits=21):
    return lib().orc_hilbert3(int(qx), int(qy), int(qz), int(bits))


def hilbert3_inverse(key, bits=21):
    q = np.zeros(3, np.uint32)
    lib().orc_hilbert3_inverse(int(key), int(bits), _p(q))
    return tuple(int(v) for v in q)


def keys(x, y, z, box, kind):
    """kind: 0 Morton, 1 Hilbert.  Returns uint64 keys in caller order."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    out = np.zeros(len(x), np.uint64)
    b = _box(box)
    lib().orc_keys(len(x), _p(x), _p(y), _p(z), C.byref(b), int(kind), _p(out))
    return out


def sort(k):
    """Stable sort by (key, original index): perm[k] = original index."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    perm = np.zeros(len(k), np.int64)
    if lib().orc_sort(len(k), _p(k), _p(perm)) != 0:
        raise MemoryError("oracle sort")
    return perm


def octree(sorted_keys, bucket):
    """Pre-order non-empty cells: dict(level, first, end, leaf)."""
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    n = len(k)
    cap = max(16, 4 * n // max(1, bucket) * 22 + 64)
    while True:
        lev = np.zeros(cap, np.int32)
        fst = np.zeros(cap, np.int64)
        end = np.zeros(cap, np.int64)
        leaf = np.zeros(cap, np.int32)
        cnt = lib().orc_octree(n, _p(k), int(bucket), _p(lev), _p(fst), _p(end), _p(leaf), cap)
        if cnt <= cap:
            return {"level": lev[:cnt], "first": fst[:cnt], "end": end[:cnt],
                    "leaf": leaf[:cnt].astype(bool)}
        cap = cnt


# ------------------------------------------------------------------------- neighbors
def _csr_take(h):
    L = lib()
    if not h:
        raise MemoryError("oracle CSR allocation failed")
    n = C.cast(h, C.POINTER(C.c_int64))[0]
    nnz = L.orc_csr_nnz(h)
    off = np.zeros(n + 1, np.int64)
    idx = np.zeros(max(nnz, 1), np.int32)
    L.orc_csr_copy(h, _p(off), _p(idx))
    L.orc_csr_free(h)
    return off, idx[:nnz]


def _csr_make(off, idx):
    off = _i64(off)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if len(idx) == 0:
        idx = np.zeros(1, np.int32)
    return lib().orc_csr_from(len(off) - 1, _p(off), _p(idx)), (off, idx)


def brute_neighbors(xs, ys, zs, hs, box, support, mode, queries):
    """O(n) per query.  mode 0 gather (d2 < ri^2), 1 symmetric (max radius)."""
    xs, ys, zs, hs = _f32(xs), _f32(ys), _f32(zs), _f32(hs)
    q = _i64(queries)
    b = _box(box)
    h = lib().orc_brute_neighbors(len(xs), _p(xs), _p(ys), _p(zs), _p(hs), C.byref(b),
                                  float(support), int(mode), len(q), _p(q))
    return _csr_take(h)


def gather_all(xs, ys, zs, hs, box, support):
    """Gather sets of every particle through the FP64 multi-level cell list."""
    xs, ys, zs, hs = _f32(xs), _f32(ys), _f32(zs), _f32(hs)
    b = _box(box)
    h = lib().orc_gather_all(len(xs), _p(xs), _p(ys), _p(zs), _p(hs), C.byref(b), float(support))
    return _csr_take(h)


def symmetrize(off, idx):
    h, keep = _csr_make(off, idx)
    try:
        s = lib().orc_symmetrize(h)
    finally:
        lib().orc_csr_free(h)
    return _csr_take(s)


def cluster_lists(n, cluster, off, idx, rows, sc_ids, jcluster=None):
    """Canonical (J, mask) lists of the super-clusters sc_ids from the
    symmetric sets (off, idx) of the particles rows; J counts j-clusters of
    `jcluster` particles (default: the i-cluster size)."""
    h, keep = _csr_make(off, idx)
    rows = _i64(rows)
    sc = _i64(sc_ids)
    L = lib()
    jc = cluster if jcluster is None else jcluster
    try:
        c = L.orc_cluster_lists(int(n), int(cluster), int(jc), h, _p(rows), len(sc), _p(sc))
    finally:
        L.orc_csr_free(h)
    nnz = L.orc_clist_nnz(c)
    o = np.zeros(len(sc) + 1, np.int64)
    J = np.zeros(max(nnz, 1), np.int32)
    m = np.zeros(max(nnz, 1), np.uint8)
    L.orc_clist_copy(c, _p(o), _p(J), _p(m))
    L.orc_clist_free(c)
    return o, J[:nnz], m[:nnz]


def half_lists(o, J, m, sc_ids):
    """Half list of the super-clusters sc_ids (j-clusters = i-clusters): each
    record keeps the entries J >= 8 s of the full canonical record of s, with
    their masks, so every pair of clusters of different super-clusters is
    stored once, by the lower super-cluster (Sec. II-D's symmetric lists)."""
    o2 = [0]
    J2, m2 = [], []
    for t, s in enumerate(np.asarray(sc_ids, np.int64)):
        Js, ms = J[o[t]:o[t + 1]], m[o[t]:o[t + 1]]
        keep = Js >= 8 * s
        J2.append(Js[keep])
        m2.append(ms[keep])
        o2.append(o2[-1] + int(keep.sum()))
    cat = (lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
    return np.asarray(o2, np.int64), cat(J2, np.int32), cat(m2, np.uint8)


def pipeline_lists(x, y, z, h, box, support, kind, cluster):
    """Whole canonical list of a small system: keys, sort, symmetric sets,
    per-super-cluster (J, mask).  Returns a dict of sorted arrays."""
    k = keys(x, y, z, box, kind)
    perm = sort(k)
    xs, ys, zs, hs = (_f32(a)[perm] for a in (x, y, z, h))
    g_off, g_idx = gather_all(xs, ys, zs, hs, box, support)
    p_off, p_idx = symmetrize(g_off, g_idx)
    n = len(xs)
    nsc = (n + 8 * cluster - 1) // (8 * cluster)
    o, J, m = cluster_lists(n, cluster, p_off, p_idx, np.arange(n), np.arange(nsc))
    return {"keys": k[perm], "perm": perm, "xs": xs, "ys": ys, "zs": zs, "hs": hs,
            "g_off": g_off, "g_idx": g_idx, "p_off": p_off, "p_idx": p_idx,
            "sc_off": o, "J": J, "mask": m}


# ----------------------------------------------------------------------------- codec
def encode_block(diffs):
    d = np.ascontiguousarray(diffs, dtype=np.uint32)
    mask = np.zeros(1, np.uint64)
    info = np.zeros(64, np.uint8)
    data = np.zeros(512, np.uint8)
    ni = C.c_int()
    nd = C.c_int()
    lib().orc_encode_block(len(d), _p(d), _p(mask), _p(info), C.byref(ni), _p(data), C.byref(nd))
    return int(mask[0]), list(info[:ni.value]), list(data[:nd.value])


def stream_nibbles(J, w=32):
    J = np.ascontiguousarray(J, dtype=np.int32)
    return lib().orc_stream_nibbles(len(J), _p(J) if len(J) else None, int(w))


def record_bytes(J, w=32, compress=True):
    J = np.ascontiguousarray(J, dtype=np.int32)
    return lib().orc_record_bytes(len(J), _p(J) if len(J) else None, int(w), int(compress))


def encode_record(J, mask, w=32, compress=True):
    J = np.ascontiguousarray(J, dtype=np.int32)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nb = record_bytes(J, w, compress)
    out = np.zeros(nb, np.uint8)
    Jp = _p(J) if len(J) else None
    mp = _p(m) if len(m) else None
    lib().orc_encode_record(len(J), Jp, mp, int(w), int(compress), _p(out))
    return out


def decode_record(rec, w=32, compress=True):
    rec = np.ascontiguousarray(rec, dtype=np.uint8)
    L = lib()
    cnt = L.orc_decode_record(_p(rec), int(w), int(compress), None, None)
    J = np.zeros(max(cnt, 1), np.int32)
    m = np.zeros(max(cnt, 1), np.uint8)
    L.orc_decode_record(_p(rec), int(w), int(compress), _p(J), _p(m))
    return J[:cnt], m[:cnt]


# ------------------------------------------------------------------------------- SPH
def w(q):
    return lib().orc_w(float(q))


def dw(q):
    return lib().orc_dw(float(q))


def W(r, h):
    return lib().orc_W(float(r), float(h))


def density(xs, ys, zs, hs, ms, box, off, idx, rows):
    """FP64 density of particles rows from their gather sets (off, idx)."""
    xs, ys, zs, hs, ms = (_f32(a) for a in (xs, ys, zs, hs, ms))
    h, keep = _csr_make(off, idx)
    rows = _i64(rows)
    out = np.zeros(len(rows), np.float64)
    b = _box(box)
    try:
        lib().orc_density(_p(xs), _p(ys), _p(zs), _p(hs), _p(ms), C.byref(b), h, _p(rows), _p(out))
    finally:
        lib().orc_csr_free(h)
    return out


def sph_force(xs, ys, zs, hs, ms, rho, pres, box, off, idx, rows):
    """FP64 pressure acceleration of particles rows over symmetric sets, and
    sum_j |pair term| per row.  rho and pres are full per-particle arrays
    (sorted order)."""
    xs, ys, zs, hs, ms = (_f32(a) for a in (xs, ys, zs, hs, ms))
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    pres = np.ascontiguousarray(pres, dtype=np.float64)
    h, keep = _csr_make(off, idx)
    rows = _i64(rows)
    ax, ay, az, fa = (np.zeros(len(rows)) for _ in range(4))
    b = _box(box)
    try:
        lib().orc_sph_force(_p(xs), _p(ys), _p(zs), _p(hs), _p(ms), _p(rho), _p(pres),
                            C.byref(b), h, _p(rows), _p(ax), _p(ay), _p(az), _p(fa))
    finally:
        lib().orc_csr_free(h)
    return ax, ay, az, fa


def lj_force(xs, ys, zs, box, eps, sigma, off, idx, rows):
    """FP64 LJ force of particles rows; also sum_j |f_ij| per row."""
    xs, ys, zs = (_f32(a) for a in (xs, ys, zs))
    h, keep = _csr_make(off, idx)
    rows = _i64(rows)
    fx, fy, fz, fa = (np.zeros(len(rows)) for _ in range(4))
    b = _box(box)
    try:
        lib().orc_lj_force(_p(xs), _p(ys), _p(zs), C.byref(b), float(eps), float(sigma), h,
                           _p(rows), _p(fx), _p(fy), _p(fz), _p(fa))
    finally:
        lib().orc_csr_free(h)
    return fx, fy, fz, fa


def lj_energy(xs, ys, zs, box, eps, sigma, off, idx):
    xs, ys, zs = (_f32(a) for a in (xs, ys, zs))
    h, keep = _csr_make(off, idx)
    b = _box(box)
    try:
        return lib().orc_lj_energy(_p(xs), _p(ys), _p(zs), C.byref(b), float(eps), float(sigma), h)
    finally:
        lib().orc_csr_free(h)


def ljc_force(xs, ys, zs, box, eps, sigma, q, kc, off, idx, rows):
    """FP64 Lennard-Jones + cutoff Coulomb force of particles rows over the
    interaction sets (off, idx); q None: no Coulomb term.  Also sum_j |f_ij|."""
    xs, ys, zs = (_f32(a) for a in (xs, ys, zs))
    qq = None if q is None else _f32(q)
    h, keep = _csr_make(off, idx)
    rows = _i64(rows)
    if len(rows) != len(off) - 1:
        raise ValueError("one row index per CSR row")
    fx, fy, fz, fa = (np.zeros(len(rows)) for _ in range(4))
    b = _box(box)
    try:
        lib().orc_ljc_force(_p(xs), _p(ys), _p(zs), C.byref(b), float(eps), float(sigma),
                            None if qq is None else _p(qq), float(kc), h, _p(rows), _p(fx),
                            _p(fy), _p(fz), _p(fa))
    finally:
        lib().orc_csr_free(h)
    return fx, fy, fz, fa


def ljc_energy(xs, ys, zs, box, eps, sigma, q, kc, off, idx):
    xs, ys, zs = (_f32(a) for a in (xs, ys, zs))
    qq = None if q is None else _f32(q)
    h, keep = _csr_make(off, idx)
    b = _box(box)
    try:
        return lib().orc_ljc_energy(_p(xs), _p(ys), _p(zs), C.byref(b), float(eps), float(sigma),
                                    None if qq is None else _p(qq), float(kc), h)
    finally:
        lib().orc_csr_free(h)


def nearest(xs, ys, zs, box, off, idx):
    """FP64 distance of every particle (rows 0..n-1) to its nearest member of
    its interaction set (off, idx); +inf for an empty set."""
    xs, ys, zs = (_f32(a) for a in (xs, ys, zs))
    h, keep = _csr_make(off, idx)
    out = np.zeros(len(off) - 1)
    b = _box(box)
    try:
        lib().orc_nearest(_p(xs), _p(ys), _p(zs), C.byref(b), h, _p(out))
    finally:
        lib().orc_csr_free(h)
    return out


def gather_counts_brute(xs, ys, zs, hs, box, support, queries):
    xs, ys, zs, hs = _f32(xs), _f32(ys), _f32(zs), _f32(hs)
    q = _i64(queries)
    out = np.zeros(len(q), np.int64)
    b = _box(box)
    lib().orc_gather_counts_brute(len(xs), _p(xs), _p(ys), _p(zs), _p(hs), C.byref(b),
                                  float(support), len(q), _p(q), _p(out))
    return out


def pred(xs, ys, zs, hs, support, i, j, box, mode):
    xs, ys, zs, hs = _f32(xs), _f32(ys), _f32(zs), _f32(hs)
    b = _box(box)
    return lib().orc_pred(_p(xs), _p(ys), _p(zs), _p(hs), float(support), int(i), int(j),
                          C.byref(b), int(mode))


def dist2(xs, ys, zs, i, j, box):
    xs, ys, zs = _f32(xs), _f32(ys), _f32(zs)
    b = _box(box)
    return lib().orc_dist2(_p(xs), _p(ys), _p(zs), int(i), int(j), C.byref(b))


def dist2_row(xs, ys, zs, box, i):
    xs, ys, zs = _f32(xs), _f32(ys), _f32(zs)
    out = np.zeros(len(xs), np.float32)
    b = _box(box)
    lib().orc_dist2_row(len(xs), _p(xs), _p(ys), _p(zs), C.byref(b), int(i), _p(out))
    return out


# ------------------------------------------------------------------------------ MLP
def mlp_nparams():
    return lib().orc_mlp_nparams()


def mlp_forward(X, P):
    X = np.ascontiguousarray(X, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros(len(X))
    lib().orc_mlp_forward(len(X), _p(X), _p(P), _p(out))
    return out


def mlp_loss_grad(X, t, P):
    X = np.ascontiguousarray(X, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    G = np.zeros(mlp_nparams())
    loss = lib().orc_mlp_loss_grad(len(X), _p(X), _p(t), _p(P), _p(G))
    return loss, G


def mlp_features(xs, ys, zs, box, cluster):
    """Learned-start features of one system in sorted order: (X [clusters x 8],
    e64 [super-clusters]), FP64."""
    xs, ys, zs = _f32(xs), _f32(ys), _f32(zs)
    n = len(xs)
    nsc = (n + 8 * cluster - 1) // (8 * cluster)
    X = np.zeros((8 * nsc, 8))
    e64 = np.zeros(nsc)
    b = _box(box)
    if lib().orc_mlp_features(n, _p(xs), _p(ys), _p(zs), C.byref(b), int(cluster), _p(X),
                              _p(e64)) != 0:
        raise MemoryError("orc_mlp_features")
    return X, e64


def mlp_targets(hs, cluster, e64):
    """Targets (y, w) per cluster from sorted smoothing lengths and e64."""
    hs = _f32(hs)
    e64 = np.ascontiguousarray(e64, dtype=np.float64)
    ncl = 8 * len(e64)
    y, w = np.zeros(ncl), np.zeros(ncl)
    lib().orc_mlp_targets(len(hs), _p(hs), int(cluster), _p(e64), _p(y), _p(w))
    return y, w


def h_at_count(xs, ys, zs, sorted_keys, box, support, k):
    """FP32 smoothing lengths (sorted order) with exactly k gather neighbors:
    halfway, in squared distance, between the k-th and (k+1)-th neighbor."""
    xs, ys, zs = _f32(xs), _f32(ys), _f32(zs)
    keys = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    out = np.zeros(len(xs), np.float32)
    b = _box(box)
    if lib().orc_h_at_count(len(xs), _p(xs), _p(ys), _p(zs), _p(keys), C.byref(b),
                            float(support), int(k), _p(out)) != 0:
        raise ValueError("orc_h_at_count: n <= k or out of memory")
    return out


def computed_pairs(mask, cluster, jcluster=None):
    """Particle pairs a list's tiles evaluate: set mask bits x M x MJ."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return int(lib().orc_computed_pairs(len(m), _p(m), int(cluster), int(jcluster or cluster)))


def cluster_overhead(mask, cluster, n_pairs, n, jcluster=None):
    """Computed pairs / (ordered neighbor pairs + self terms)."""
    return computed_pairs(mask, cluster, jcluster) / float(n_pairs + n)
