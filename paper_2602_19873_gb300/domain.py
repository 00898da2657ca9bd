"""SFC domain decomposition with a halo exchange across ranks.

The paper's method runs inside a distributed code: the particles are split
into contiguous ranges of the space-filling curve (Sec. I, the Cornerstone
domain decomposition the method builds on), and every rank builds its list
over the particles it owns plus a halo received from the other ranks before
its neighborhood passes (Sec. IV, the Evrard runs on up to 1024 GPUs).

One call of ``decomposed_density`` on every rank of a process group:

1. keys of the local particles in the global box (``nl_sfc_keys``);
2. splitters from two global key histograms (two all-reduces): 16 key bits,
   then 16 more bits inside each bucket that holds a splitter, so the ranks'
   counts differ from N/P by at most the population of one 32-bit key prefix;
3. each particle to the rank whose key range holds it (one all-to-all);
4. the owned particles' box and largest radius (one all-gather);
5. every owned particle that may be a symmetric neighbor of a particle
   inside another rank's box goes to that rank (one all-to-all), decided by
   the search's conservative point-box test, so no pair is lost;
6. ``nl_build`` over owned + halo particles, then the density and neighbor
   count passes; the owned particles' results are exact.

The device steps go through the C ABI (``LibraryOps``); the exchanges go
through ``torch.distributed`` (NCCL keeps tensors on the GPU; with gloo they
pass through host memory).  ``ops`` can be any object with the methods of
``LibraryOps``.
"""
import numpy as np

KEY_BITS = 63
L1_BITS, L1_SHIFT = 16, 47     # first histogram: the top 16 key bits
L2_BITS, L2_SHIFT = 16, 31     # second histogram: the next 16 bits
MAX_RANKS = 64                 # destinations are bits of a 64-bit mask


class Comm:
    """The collectives of the decomposition over a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.host = dist.get_backend(group) == "gloo"

    def _out(self, t):
        return t.cpu() if self.host else t

    def all_reduce_sum(self, t):
        c = self._out(t).clone()
        self.dist.all_reduce(c, op=self.dist.ReduceOp.SUM, group=self.group)
        return c.to(t.device)

    def all_gather(self, t):
        """[size, *t.shape] of every rank's t."""
        import torch
        c = self._out(t).contiguous()
        parts = [torch.empty_like(c) for _ in range(self.size)]
        self.dist.all_gather(parts, c, group=self.group)
        return torch.stack(parts).to(t.device)

    def all_to_all(self, rows, send_counts):
        """rows [n, w] grouped by destination with send_counts[q] rows for
        rank q; returns the received rows, grouped by source rank, and the
        per-source counts."""
        import torch
        sc_d = self._out(torch.tensor(send_counts, dtype=torch.int64, device=rows.device))
        rc_d = torch.empty_like(sc_d)
        self.dist.all_to_all_single(rc_d, sc_d, group=self.group)
        rc = [int(v) for v in rc_d.cpu().tolist()]
        src = self._out(rows).contiguous()
        out = torch.empty((sum(rc),) + tuple(rows.shape[1:]), dtype=rows.dtype, device=src.device)
        self.dist.all_to_all_single(out, src, rc, list(send_counts), group=self.group)
        return out.to(rows.device), rc


class LibraryOps:
    """Per-rank device steps through the CUDA library's C ABI."""

    def __init__(self, stream=None):
        self.stream = stream

    def keys(self, x, y, z, h, box, key, support):
        import torch
        from . import nl
        k = torch.empty(x.numel(), dtype=torch.int64, device=x.device)
        nl.sfc_keys(x, y, z, h, box, key, support, k, self.stream)
        return k

    def histogram(self, keys, lo, shift, nbins):
        import torch
        from . import nl
        out = torch.empty(nbins, dtype=torch.int64, device=keys.device)
        nl.key_histogram(keys, lo, shift, nbins, out, self.stream)
        return out

    def owner_mask(self, keys, splitters, P):
        import torch
        from . import nl
        sp = torch.tensor(splitters, dtype=torch.int64, device=keys.device)
        m = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
        nl.domain_owner_mask(keys, sp, P, m, self.stream)
        return m

    def box(self, x, y, z, h, support):
        import torch
        from . import nl
        out = torch.empty(8, dtype=torch.float32, device=x.device)
        nl.domain_box(x, y, z, h, support, out, self.stream)
        return out

    def halo_mask(self, x, y, z, h, box, support, dom, P, self_rank):
        import torch
        from . import nl
        m = torch.empty(x.numel(), dtype=torch.int64, device=x.device)
        nl.domain_halo_mask(x, y, z, h, box, support, dom.contiguous(), P, self_rank, m,
                            self.stream)
        return m

    def group(self, mask, P):
        """(indices grouped by destination, ascending within each; counts)."""
        import torch
        from . import nl
        cnt = torch.empty(P, dtype=torch.int64, device=mask.device)
        nl.domain_count(mask, P, cnt, self.stream)
        counts = [int(v) for v in cnt.cpu().tolist()]
        total = sum(counts)
        idx = torch.empty(total, dtype=torch.int32, device=mask.device)
        if total:
            off = torch.tensor(np.concatenate([[0], np.cumsum(counts)[:-1]]), dtype=torch.int64,
                               device=mask.device)
            nl.domain_group(mask, P, off, idx, self.stream)
        return idx.to(torch.int64), counts

    def local_pass(self, x, y, z, h, m, box, params):
        """Build over the local particles; density and gather counts."""
        import torch
        from . import nl
        n = x.numel()
        L = nl.NeighborList().build(x, y, z, h, box, params, self.stream)
        rho = torch.empty(n, dtype=torch.float32, device=x.device)
        cnt = torch.empty(n, dtype=torch.int32, device=x.device)
        L.density_pass(m, rho, self.stream)
        L.neighbor_counts(cnt, self.stream)
        sizes = L.sizes()
        L.free()
        return rho, cnt, sizes


def splitters(comm, ops, keys, n_local):
    """P-1 ascending key splitters balancing the global particle count; the
    owner of key k is the number of splitters <= k."""
    import torch
    P = comm.size
    dev = keys.device
    N = int(comm.all_reduce_sum(torch.tensor([n_local], dtype=torch.int64, device=dev)).item())
    if P == 1:
        return [], N
    h1 = comm.all_reduce_sum(ops.histogram(keys, 0, L1_SHIFT, 1 << L1_BITS)).cpu().numpy()
    c1 = np.cumsum(h1)
    targets = [r * N // P for r in range(1, P)]
    b = [int(np.searchsorted(c1, t, side="right")) for t in targets]
    b = [min(v, (1 << L1_BITS) - 1) for v in b]
    buckets = sorted(set(b))
    h2 = torch.stack([ops.histogram(keys, v << L1_SHIFT, L2_SHIFT, 1 << L2_BITS) for v in buckets])
    h2 = comm.all_reduce_sum(h2).cpu().numpy()
    out = []
    for t, v in zip(targets, b):
        before = int(c1[v] - h1[v])
        c2 = np.cumsum(h2[buckets.index(v)])
        c = int(np.searchsorted(c2, t - before, side="right"))
        out.append((v << L1_SHIFT) + (min(c, (1 << L2_BITS) - 1) << L2_SHIFT))
    for r in range(1, len(out)):          # ascending (equal splitters leave a rank empty)
        out[r] = max(out[r], out[r - 1])
    return out, N


def _pack(x, y, z, h, m, ids):
    import torch
    f = torch.stack([x, y, z, h, m], 1).contiguous().view(torch.int32)
    return torch.cat([f, ids.contiguous().view(torch.int32).view(-1, 2)], 1)


def _unpack(rows):
    import torch
    f = rows[:, :5].contiguous().view(torch.float32)
    ids = rows[:, 5:7].contiguous().view(torch.int64).view(-1)
    return [f[:, k].contiguous() for k in range(5)], ids


def decomposed_density(comm, ops, ids, x, y, z, h, m, box, key, params):
    """One decomposition step and the density pass of the owned particles.

    Every rank passes its local particles (any subset; ids are their global
    indices, int64) and the same global box, key kind and nl_params.  Returns
    a dict with the owned particles' ids, densities and gather-neighbor
    counts (same order), the splitters, the global count and the halo size."""
    import torch
    P, me = comm.size, comm.rank
    if P > MAX_RANKS:
        raise ValueError("at most %d ranks" % MAX_RANKS)
    support = float(params.support)
    keys = ops.keys(x, y, z, h, box, key, support)
    split, N = splitters(comm, ops, keys, int(x.numel()))
    # particles to their owners
    idx, counts = ops.group(ops.owner_mask(keys, split, P), P)
    rows, _ = comm.all_to_all(_pack(x, y, z, h, m, ids).index_select(0, idx), counts)
    (ox, oy, oz, oh, om), oid = _unpack(rows)
    n_own = int(ox.numel())
    # halo: owned particles that may be neighbors of another rank's particles
    dom = comm.all_gather(ops.box(ox, oy, oz, oh, support))
    hidx, hcounts = ops.group(ops.halo_mask(ox, oy, oz, oh, box, support, dom, P, me), P)
    hrows, _ = comm.all_to_all(_pack(ox, oy, oz, oh, om, oid).index_select(0, hidx), hcounts)
    (hx, hy, hz, hh, hm), hid = _unpack(hrows)
    n_halo = int(hx.numel())
    out = {"ids": oid, "n_global": N, "splitters": split, "n_owned": n_own, "n_halo": n_halo,
           "halo_sent": int(sum(hcounts))}
    if n_own == 0:
        out["rho"] = torch.empty(0, dtype=torch.float32, device=x.device)
        out["counts"] = torch.empty(0, dtype=torch.int32, device=x.device)
        return out
    cat = [torch.cat([a, b]) for a, b in ((ox, hx), (oy, hy), (oz, hz), (oh, hh), (om, hm))]
    rho, cnt, sizes = ops.local_pass(*cat, box, params)
    out["rho"], out["counts"] = rho[:n_own], cnt[:n_own]
    out["list_bytes"] = sizes.get("list_bytes") if isinstance(sizes, dict) else None
    return out
