"""Seeded synthetic particle systems (inputs only; no neighbor-list arithmetic).

Shared by the tests, the benchmark and the oracle's callers, so that the CUDA
library and the CPU oracle read identical FP32 bytes.  This module imports
nothing from the library or the oracle.  Each generator returns a dict with
float32 ``x, y, z, m, h`` (``h`` is an initial smoothing length taken from the
analytic number density of the distribution, a workload property, not a
converged value), the ``box`` (lo, hi, periodic), the SFC ``kind``
(0 Morton, 1 Hilbert), the pair ``support`` (r = support * h) and metadata.

Workloads (stand-ins for the paper's LJ 4M-atom fluid of Sec. III-B and its
Evrard sphere of Sec. IV; none of the paper's data ships):
  uniform     -- uniform random points in a periodic unit cube.
  evrard      -- unit sphere with number density proportional to 1/r
                 (radius r = u^(1/2)), non-periodic.
  lj_fluid    -- cubic lattice at 100 particles/nm^3 in a periodic cube,
                 Gaussian jitter 0.05 nm, single cutoff.
  lj_coulomb  -- the same fluid with charges +-1 (neutral) and two radii:
                 the list radius (about 200 neighbors) and the shorter
                 interaction cutoff (about 150), the Verlet-buffer shape.
  plummer     -- several Plummer spheres with log-uniform scale radii,
                 centres uniform in the unit box, non-periodic, bbox box.
  batched     -- many independent systems of log-uniform size, alternating
                 uniform cubes and single Plummer spheres.
"""
import math

import numpy as np

KIND_MORTON = 0
KIND_HILBERT = 1


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _h_from_density(nd, n_target):
    """h such that the sphere of radius 2h holds n_target particles at number
    density nd (support 2h)."""
    nd = np.maximum(nd, 1e-30)
    return 0.5 * np.cbrt(3.0 * n_target / (4.0 * math.pi * nd))


def _box(lo, hi, periodic):
    return {"lo": np.asarray(lo, np.float32), "hi": np.asarray(hi, np.float32),
            "periodic": np.asarray(periodic, np.int32)}


def _bbox(x, y, z):
    lo = [float(np.min(a)) for a in (x, y, z)]
    hi = [float(np.max(a)) for a in (x, y, z)]
    for a in range(3):
        if hi[a] <= lo[a]:
            hi[a] = lo[a] + 1.0
    return lo, hi


def uniform(n=32768, seed=1, n_target=100.0):
    """Uniform random points in a periodic unit cube; constant h giving
    n_target expected neighbors within 2h."""
    rng = np.random.default_rng(seed)
    p = rng.random((3, n), dtype=np.float64).astype(np.float32)
    p = np.where(p >= 1.0, np.float32(0.0), p)
    h = np.float32(0.5 * (3.0 * n_target / (4.0 * math.pi * n)) ** (1.0 / 3.0))
    return {"name": "uniform", "x": _f32(p[0]), "y": _f32(p[1]), "z": _f32(p[2]),
            "m": np.full(n, 1.0 / n, np.float32), "h": np.full(n, h, np.float32),
            "box": _box([0, 0, 0], [1, 1, 1], [1, 1, 1]), "kind": KIND_MORTON,
            "support": 2.0, "n_target": n_target}


def evrard(n=1 << 21, seed=2, n_target=200.0):
    """Evrard-sphere initial condition: rho ~ 1/r inside the unit sphere."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    r = np.sqrt(u)
    cz = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    x, y, z = r * s * np.cos(phi), r * s * np.sin(phi), r * cz
    nd = n / (2.0 * math.pi * np.maximum(r, 1e-6))
    h = _h_from_density(nd, n_target)
    return {"name": "evrard", "x": _f32(x), "y": _f32(y), "z": _f32(z),
            "m": np.full(n, 1.0 / n, np.float32), "h": _f32(h),
            "box": _box([-1, -1, -1], [1, 1, 1], [0, 0, 0]), "kind": KIND_HILBERT,
            "support": 2.0, "n_target": n_target, "u": 0.05, "gamma": 5.0 / 3.0}


def lj_fluid(n=4_000_000, seed=3, density=100.0, rc=0.9, jitter=0.05):
    """Jittered lattice at `density` per nm^3, periodic cube of side
    (n/density)^(1/3); one cutoff rc for every particle (h = rc, support 1)."""
    rng = np.random.default_rng(seed)
    L = (n / density) ** (1.0 / 3.0)
    k = int(math.ceil(n ** (1.0 / 3.0)))
    sites = rng.permutation(k ** 3)[:n]
    ix, iy, iz = sites // (k * k), (sites // k) % k, sites % k
    a = L / k
    p = np.stack([ix, iy, iz]).astype(np.float64) * a + 0.5 * a
    p += rng.normal(0.0, jitter, size=p.shape)
    p = np.mod(p, L)
    p = p.astype(np.float32)
    Lf = np.float32(L)
    p = np.where(p >= Lf, np.float32(0.0), p)
    return {"name": "lj_fluid", "x": _f32(p[0]), "y": _f32(p[1]), "z": _f32(p[2]),
            "m": np.ones(n, np.float32), "h": np.full(n, np.float32(rc), np.float32),
            "box": _box([0, 0, 0], [Lf, Lf, Lf], [1, 1, 1]), "kind": KIND_HILBERT,
            "support": 1.0, "rc": rc, "eps": 1.0, "sigma": 0.3, "L": float(Lf)}


def lj_coulomb(n=4_000_000, seed=6, density=100.0, n_list=200.0, n_int=150.0, jitter=0.05):
    """lj_fluid with charges and a Verlet buffer: h = r_list holds n_list
    expected neighbors, rc = r_int holds n_int (spheres at `density`); charges
    +1 on a random half and -1 on the rest (zero for an odd one out).  kc is
    the Coulomb constant in kJ mol^-1 nm e^-2."""
    r_list = (3.0 * n_list / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    r_int = (3.0 * n_int / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    d = lj_fluid(n, seed=seed, density=density, rc=r_list, jitter=jitter)
    rng = np.random.default_rng(seed + 1000)
    q = np.zeros(n, np.float32)
    order = rng.permutation(n)
    half = n // 2
    q[order[:half]] = 1.0
    q[order[half:2 * half]] = -1.0
    d.update({"name": "lj_coulomb", "q": q, "rc": float(np.float32(r_int)),
              "r_list": float(np.float32(r_list)), "kc": 138.935458})
    return d


def _plummer_radii(rng, n, a):
    out = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        u = rng.random(len(todo))
        u = np.clip(u, 1e-12, 1.0 - 1e-12)
        r = a * (u ** (-2.0 / 3.0) - 1.0) ** -0.5
        ok = r <= 20.0 * a
        out[todo[ok]] = r[ok]
        todo = todo[~ok]
    return out


def plummer(n=1 << 24, n_spheres=64, seed=4, n_target=200.0, a_range=(-3.0, -1.0)):
    """n_spheres Plummer spheres (scale radii log-uniform), centres in [0,1)^3,
    equal masses, non-periodic box = particle bounding box."""
    rng = np.random.default_rng(seed)
    per = n // n_spheres
    counts = np.full(n_spheres, per)
    counts[: n - per * n_spheres] += 1
    a = 10.0 ** rng.uniform(a_range[0], a_range[1], n_spheres)
    cen = rng.random((n_spheres, 3))
    xs, ys, zs = [], [], []
    for s in range(n_spheres):
        c = int(counts[s])
        r = _plummer_radii(rng, c, a[s])
        cz = 2.0 * rng.random(c) - 1.0
        phi = 2.0 * math.pi * rng.random(c)
        st = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        xs.append(cen[s, 0] + r * st * np.cos(phi))
        ys.append(cen[s, 1] + r * st * np.sin(phi))
        zs.append(cen[s, 2] + r * cz)
    x, y, z = _f32(np.concatenate(xs)), _f32(np.concatenate(ys)), _f32(np.concatenate(zs))
    # number density of the whole mixture at every particle
    nd = np.empty(n)
    P = np.stack([x, y, z], 1).astype(np.float64)
    coef = 3.0 * counts / (4.0 * math.pi * a ** 3)
    inva2 = 1.0 / a ** 2
    cenf = cen
    step = 1 << 15
    for b in range(0, n, step):
        q = P[b:b + step]
        d2 = (q * q).sum(1)[:, None] - 2.0 * (q @ cenf.T) + (cenf * cenf).sum(1)[None, :]
        t = 1.0 / (1.0 + np.maximum(d2, 0.0) * inva2[None, :])
        nd[b:b + step] = (t * t * np.sqrt(t)) @ coef
    h = _h_from_density(nd, n_target)
    lo, hi = _bbox(x, y, z)
    return {"name": "plummer", "x": x, "y": y, "z": z, "m": np.full(n, 1.0 / n, np.float32),
            "h": _f32(h), "box": _box(lo, hi, [0, 0, 0]), "kind": KIND_HILBERT,
            "support": 2.0, "n_target": n_target, "scale_radii": a, "centres": cen}


def batched(n_systems=256, seed=5, n_target=100.0, log_n=(3.0, 6.0), scale=1.0):
    """List of independent systems: even index uniform periodic unit cube,
    odd index one Plummer sphere in its bounding box.  `scale` shrinks every
    system size (tests)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(10.0 ** rng.uniform(log_n[0], log_n[1], n_systems) * scale).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    out = []
    for s in range(n_systems):
        sub = int(rng.integers(0, 2 ** 31))
        if s % 2 == 0:
            d = uniform(int(sizes[s]), seed=sub, n_target=n_target)
            d["kind"] = KIND_HILBERT
        else:
            d = plummer(int(sizes[s]), n_spheres=1, seed=sub, n_target=n_target)
        out.append(d)
    return out


def cached(fn, key, *args, **kw):
    """Call a generator once per machine: results are kept as .npz files
    under $TMPDIR (inputs only; safe to delete)."""
    import os
    import tempfile
    d = os.path.join(tempfile.gettempdir(), "nlgb_workloads")
    path = os.path.join(d, key + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=True)
        v = z["d"]
        return v.item() if v.shape == () else list(v)
    out = fn(*args, **kw)
    os.makedirs(d, exist_ok=True)
    tmp = path + ".%d.tmp.npz" % os.getpid()
    box = np.empty((), dtype=object)  # a 0-d holder keeps lists and dicts whole
    box[()] = out
    np.savez(tmp, d=box)
    os.replace(tmp, path)
    return out


def config(name, scale=1.0, seed=None):
    """The six named workloads at full size (scale=1) or shrunk for tests."""
    if name == "uniform_periodic_32k":
        return uniform(max(8, int(32768 * scale)), seed=1 if seed is None else seed)
    if name == "evrard_2m":
        return evrard(max(8, int((1 << 21) * scale)), seed=2 if seed is None else seed)
    if name == "lj_fluid_4m":
        return lj_fluid(max(8, int(4_000_000 * scale)), seed=3 if seed is None else seed)
    if name == "lj_coulomb_4m":
        return lj_coulomb(max(8, int(4_000_000 * scale)), seed=6 if seed is None else seed)
    if name == "plummer64_16m":
        n = max(64, int((1 << 24) * scale))
        return plummer(n, n_spheres=64 if n >= 64 * 64 else max(1, n // 64),
                       seed=4 if seed is None else seed)
    if name == "batched_256":
        return batched(seed=5 if seed is None else seed, scale=scale)
    raise KeyError(name)
