"""Benchmark: neighbor-list build + SPH density pass on one GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

One step = the whole hot path on one batch of synthetic input: SFC keys,
stable radix sort, permute + cluster boxes, octree, cluster-pair search with
list encoding, and the decode + density pass, on the 2^24-particle
64-Plummer-sphere system (inputs resident in HBM, larger than L2).  `value`
is Mparticles/s over all ranks (weak scaling: every rank builds its own
replica); `e2e` repeats the measurement through nl_density_from_host with
pinned host buffers, copies included.  `--impl reference` times the CPU
oracle on a bounded sample of the same workload generator.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("build+density Mparticles/s at 16M, learned-h vs plain, rel err ≤1e-5; %HBM peak")
UNIT = "Mparticles/s"
WORKLOAD = "plummer64_16m"
N_FULL = 1 << 24
ALU_OPS_PER_PAIR_SEARCH = 9      # predicate: 3 sub, 3 mul, 2 add, 1 compare (non-periodic)
ALU_OPS_PER_DENSITY_SIDE = 12    # gather pair in range: square root, scale, spline, weighted add
ALGO_BYTES_PER_PARTICLE = 145    # keygen 20 + sort 24 + permute 49 + octree 2 + search 19 + density 31
# DRAM bytes (read + write) of one k_search launch per particle, from an ncu
# capture on this generator at 2^21 particles (8x8 clusters, leaf bucket 256,
# half list: packed tile and node tests, the range test of the half search
# ending at the first accepted leaf), 44.87 MB + 1.13 MB, scaled by the
# particle count (the traffic grows with the particles).  Valid for that kernel
# version only; a list kind without a capture of the current kernel reports no
# traffic.
SEARCH_DRAM_BYTES_PER_PARTICLE = {"half": 46.0e6 / 2097152}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


def fp32_peak(stream, device_index=0):
    """Measured FP32 rate of this GPU (element ops/s, scalar and packed
    fused multiply-add chains on every lane, CUDA events), with the SM clock
    sampled while the probe runs.  The peak is the faster of the two forms;
    the nominal figure (SMs x 128 lanes x max clock) is given beside it."""
    import torch
    from paper_2602_19873_gb300 import nl
    clocks = Clocks(device_index)
    clocks.start()
    scalar, scalar_ms = nl.probe_fp32_rate(False, 10, stream)
    packed, packed_ms = nl.probe_fp32_rate(True, 10, stream)
    clk = clocks.stop()
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    _, _, sm_max = peaks()
    return {"tops": max(scalar, packed) / 1e12, "scalar_tops": scalar / 1e12,
            "packed_tops": packed / 1e12, "scalar_ms": scalar_ms, "packed_ms": packed_ms,
            "sms": sms, "nominal_tops": sms * 128 * sm_max * 1e6 / 1e12,
            "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
            "how": "nl_probe_fp32_rate: 8 independent FMA chains per thread on every lane of "
                   "every SM, best of 10 launches (CUDA events); one element FMA = one op"}


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def quiesce_host():
    """Flush dirty file pages (cache files written while preparing inputs)
    so that their writeback does not delay the host thread in the timed
    region: a build reads status words back from the device between its
    stages, so host stalls show up as idle GPU time."""
    if hasattr(os, "sync"):
        os.sync()


def init_ranks(backend):
    """(world size, rank, local rank); joins the process group when there
    are several ranks (one process per GPU, env rendezvous)."""
    ws, rank, local = dist_init()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest x over all ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws, device):
    """The sum of x over all ranks."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank, ws, ms):
    """Whole-job throughput in millions of units per second: every rank
    processes units_per_rank units in the slowest rank's ms."""
    return ws * units_per_rank / (ms * 1e-3) / 1e6


def reference_sample(steps, warmup, requested=None):
    """Particles per oracle step: the requested size, else a size that keeps
    warmup + steps oracle steps near 100 s on the host (0.11 Mparticles/s
    measured for the oracle), between 2^16 and 2^20."""
    if requested:
        return requested
    return int(min(1 << 20, max(1 << 16, 0.11e6 * 100.0 / max(1, steps + warmup))))


def launches_per_step(sizes, batched, mixed=False, half_list=False):
    """Kernels of one build + density step (graph replay when batched): keys
    (which also count the sort's digits), the key sort (digit starts and 8
    passes; in batches a histogram, the starts and one pass by system),
    permute, octree (10), search (open, interior and boundary launches plus a
    classification when a batch mixes open and periodic systems), and for the
    half search the tuple sort (histogram, starts, one pass per 8 key bits,
    plus the fill of unused slots in a graph), the lower-entry scan (3) and
    the record assembly; then the pass input gather and the pass (three when
    mixed); a half list stores the search's records directly and adds the
    pass's finishing kernel."""
    sort_launches = 1 + 8 + (3 if batched else 0)
    # mixed batches: open, interior and boundary launches of the search and
    # the pass, plus the interior classification
    n = 1 + sort_launches + 1 + 10 + (3 + 1 if mixed else 1) + (2 if mixed else 0)
    if half_list:
        return n + 3
    if sizes["j_cluster"] == sizes["cluster"]:
        nsc = sizes["n_superclusters"]
        bits = 1
        while bits < 64 and (nsc * 8 * nsc) >> bits:
            bits += 1
        n += 2 + (bits + 7) // 8 + 3 + 1 + (1 if batched else 0)
    return n + 2


def workload(seed, n=N_FULL):
    from paper_2602_19873_gb300 import workloads as wl
    return wl.cached(wl.plummer, "plummer64_%d_%d" % (n, seed), n, n_spheres=64, seed=seed)


def converge_h(L, dev, d, params, start, stream):
    """Exact h iteration to 200 +- 2 neighbors; returns (h tensor, info, ms).
    The learned start runs its feature and MLP kernels inside the timing."""
    import torch
    h = dev["h"].clone()
    torch.cuda.synchronize()
    t = time.perf_counter()
    info = L.iterate_h(dev["x"], dev["y"], dev["z"], h, d["box"], params, 200.0, 2.0,
                       max_iter=60, margin=0.15, start=start, stream=stream)
    torch.cuda.synchronize()
    return h, info, (time.perf_counter() - t) * 1e3


def time_h_iteration(H, dev, d, params, start, stream, reps):
    """One warm-up and `reps` timed h iterations from `start`: the median,
    spread and per-pass trace (list sizes and times) of the runs."""
    converge_h(H, dev, d, params, start, stream)       # warm-up
    runs = []
    for _ in range(max(1, reps)):
        h, info, ms = converge_h(H, dev, d, params, start, stream)
        runs.append(ms)
    trace = H.hiter_trace()
    return h, {"ms": statistics.median(runs), "ms_min": min(runs), "ms_max": max(runs),
               "runs": len(runs), "iterations": info["iterations"],
               "rebuilds": info["rebuilds"], "unconverged": info["unconverged"],
               "passes": [{"rebuilt": t["rebuilt"], "active_superclusters": t["active"],
                           "unconverged": t["unconverged"], "entries": t["entries"],
                           "computed_pairs": t["tiles"] * params.cluster * params.cluster,
                           "ms": t["ms"]} for t in trace]}


TRAIN_SEEDS = list(range(100, 108))
TRAIN_N = 1 << 19


def train_mlp(params, stream, reuse):
    """Train the smoothing-length MLP on the GPU: 8 systems of the benchmark
    generator (2^19 particles, seeds 100..107), h from the exact iteration,
    per-cluster features and targets from the list kernels, Adam."""
    import torch
    from paper_2602_19873_gb300 import nl
    cache = os.path.join(__import__("tempfile").gettempdir(), "nlgb_workloads",
                         "mlp_%d_%d.npy" % (TRAIN_N, len(TRAIN_SEEDS)))
    mlp = nl.MLP(seed=0)
    if reuse and os.path.exists(cache):
        mlp.set_params(np.load(cache))
        return mlp, {"cached": True}
    t0 = time.perf_counter()
    Xs, ys, ws = [], [], []
    for seed in TRAIN_SEEDS:
        d = workload(seed, TRAIN_N)
        dev = {k: torch.from_numpy(d[k]).cuda() for k in ("x", "y", "z", "h")}
        L = nl.NeighborList()
        h = dev["h"].clone()
        L.iterate_h(dev["x"], dev["y"], dev["z"], h, d["box"], params, 200.0, 2.0, max_iter=60,
                    start=nl.NL_HSTART_PLAIN, stream=stream)
        X, e64 = L.mlp_features(stream)
        y, w = L.mlp_targets(h, e64, stream)
        Xs.append(X), ys.append(y), ws.append(w)
        L.free()
    X, y, w = torch.cat(Xs), torch.cat(ys), torch.cat(ws)
    t1 = time.perf_counter()
    loss = mlp.train(X, y, w, epochs=40, batch=8192, lr=3e-3, seed=1, stream=stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    np.save(cache, mlp.get_params())
    return mlp, {"samples": int(y.numel()), "epochs": 40, "final_loss": loss,
                 "data_ms": (t1 - t0) * 1e3, "train_ms": (t2 - t1) * 1e3,
                 "systems": "%d x %d particles, seeds %d..%d" % (len(TRAIN_SEEDS), TRAIN_N,
                                                                 TRAIN_SEEDS[0], TRAIN_SEEDS[-1])}


def run_native(args):
    import torch
    from paper_2602_19873_gb300 import nl

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    init_ranks("nccl")
    if ws > 1:
        import torch.distributed as dist
    d = workload(4 + rank, args.n)
    n = len(d["x"])
    dev = {k: torch.from_numpy(d[k]).cuda() for k in ("x", "y", "z", "h", "m")}
    M, MJ = (int(v) for v in args.tile.split("x"))
    params = nl.make_params(key=d["kind"], cluster=M, support=d["support"], compress=1,
                            leaf_bucket=args.leaf_bucket, j_cluster=MJ,
                            threads_per_block=args.threads, blocks_per_sm=args.blocks_per_sm,
                            half_list=int(args.list == "half"))
    L = nl.NeighborList()
    stream = torch.cuda.current_stream()
    # smoothing lengths at 200 +- 2 neighbors from the plain start (untimed
    # input preparation; the iteration is reported separately)
    H = nl.NeighborList()
    hcache = os.path.join(__import__("tempfile").gettempdir(), "nlgb_workloads",
                          "hconv_%d_%d.npy" % (n, 4 + rank))
    learned = None
    if args.h_source == "generator":
        # profiling runs: the generator's h (no iteration, no learned start)
        hconv = dev["h"].clone()
        hinfo, hms = {"iterations": None, "rebuilds": None, "unconverged": None}, None
        plain = None
    elif args.reuse_h and os.path.exists(hcache):
        hconv = torch.from_numpy(np.load(hcache)).cuda()
        hinfo, hms = {"iterations": None, "rebuilds": None, "unconverged": None}, None
        plain = None
    else:
        hconv, plain = time_h_iteration(H, dev, d, params, nl.NL_HSTART_PLAIN, stream,
                                        args.h_reps)
        hinfo, hms = plain, plain["ms"]
        np.save(hcache, hconv.cpu().numpy())
        if not args.no_learned:
            mlp, tinfo = train_mlp(params, stream, args.reuse_h)
            H.set_mlp(mlp)
            _, learned = time_h_iteration(H, dev, d, params, nl.NL_HSTART_LEARNED, stream,
                                          args.h_reps)
            learned["training"] = tinfo
            learned["speedup_vs_plain"] = hms / learned["ms"]
            cost = (tinfo.get("data_ms") or 0.0) + (tinfo.get("train_ms") or 0.0)
            gain = hms - learned["ms"]
            learned["break_even_runs"] = (cost / gain) if (cost > 0 and gain > 0) else None
            learned["break_even_note"] = ("training cost (data generation + training, ms) over "
                                          "the median time saved per h iteration of this system")
            H.set_mlp(None)
            mlp.free()
    H.free()
    dev["h"] = hconv
    d["h"] = hconv.cpu().numpy()
    L.set_profiling(True)
    rho = torch.empty(n, dtype=torch.float32, device="cuda")

    def step():
        L.build(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], params, stream)
        L.density_pass(dev["m"], rho, stream)

    # input files written above (workload, h and MLP caches) are flushed now,
    # not by background writeback competing with the host thread while timed
    quiesce_host()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    stage_acc = {}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step()
        for k, v in L.stage_times().items():
            stage_acc[k] = stage_acc.get(k, 0.0) + v
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, "cuda")
    if ws > 1:
        dist.barrier()
    stages = {k: v / args.steps for k, v in stage_acc.items()}
    sizes = L.sizes()

    # the minimum-reduction pass on the same list (nearest gather neighbor)
    dist = torch.empty(n, dtype=torch.float32, device="cuda")
    L.nearest_distance(dist, stream)
    t0.record(stream)
    for _ in range(args.steps):
        L.nearest_distance(dist, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    near_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, "cuda")

    # the other storage of the same list (full <-> half), timed the same way
    alt_kind = "full" if args.list == "half" else "half"
    alt_params = nl.make_params(key=d["kind"], cluster=M, support=d["support"], compress=1,
                                leaf_bucket=args.leaf_bucket, j_cluster=MJ,
                                threads_per_block=args.threads, blocks_per_sm=args.blocks_per_sm,
                                half_list=int(alt_kind == "half"))
    alt = None
    if alt_kind == "full" or MJ == M:
        A = nl.NeighborList()
        A.set_profiling(True)

        def alt_step():
            A.build(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], alt_params, stream)
            A.density_pass(dev["m"], rho, stream)

        quiesce_host()
        for _ in range(args.warmup):
            alt_step()
        torch.cuda.synchronize()
        a_acc = {}
        t0.record(stream)
        for _ in range(args.steps):
            alt_step()
            for k, v in A.stage_times().items():
                a_acc[k] = a_acc.get(k, 0.0) + v
        t1.record(stream)
        torch.cuda.synchronize()
        a_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, "cuda")
        asz = A.sizes()
        alt = {"list": alt_kind, "ms_per_step": a_ms, "value": job_rate(n, ws, a_ms),
               "unit": UNIT, "stages_ms": {k: v / args.steps for k, v in a_acc.items()},
               "bytes_per_particle": asz["list_bytes"] / n, "entries": asz["n_entries"]}
        A.free()
    # gather pairs of the timed list (the density pass evaluates the kernel
    # once per gather pair and particle): one count pass after the timing
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    L.neighbor_counts(cnt, stream)
    torch.cuda.synchronize()
    gather_pairs = int(cnt.to(torch.int64).sum().item())
    del cnt

    # end to end through the host-buffer entry point (pinned memory)
    pin = {k: torch.from_numpy(d[k]).pin_memory().numpy() for k in ("x", "y", "z", "h", "m")}
    rho_h = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
    E = nl.NeighborList()
    for _ in range(0 if args.no_e2e else max(1, args.warmup)):
        E.density_from_host(pin["x"], pin["y"], pin["z"], pin["h"], pin["m"], d["box"], params,
                            rho_h, stream)
    torch.cuda.synchronize()
    te = time.perf_counter()
    esteps = max(1, min(args.steps, 5))
    for _ in range(0 if args.no_e2e else esteps):
        E.density_from_host(pin["x"], pin["y"], pin["z"], pin["h"], pin["m"], d["box"], params,
                            rho_h, stream)
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - te) * 1e3 / esteps
    e_ms = max_over_ranks(e_ms, ws, "cuda")

    hbm, hbm_kind, sm_max = peaks()
    fp32 = fp32_peak(stream, local)
    alu_peak = fp32["tops"]
    search_ms = stages.get("search", float("nan"))
    pass_ms = stages.get("pass", float("nan"))
    # computed pairs of the timed list: its tiles with the mask bit set x M x MJ
    pairs = sizes["n_tiles"] * params.cluster * sizes["j_cluster"]
    achieved = pairs * ALU_OPS_PER_PAIR_SEARCH / (search_ms * 1e-3) / 1e12
    pass_ops = pairs * ALU_OPS_PER_PAIR_SEARCH + (gather_pairs + n) * ALU_OPS_PER_DENSITY_SIDE
    pass_achieved = pass_ops / (pass_ms * 1e-3) / 1e12
    step_bytes = ALGO_BYTES_PER_PARTICLE * n
    out = {
        "metric": METRIC, "value": job_rate(n, ws, ms), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "%s: 2^24 particles in 64 Plummer spheres (scale radii "
                               "log-uniform 1e-3..1e-1), Hilbert keys, %dx%d clusters, "
                               "compressed %s list" % (WORKLOAD, M, MJ, args.list),
                   "n": n, "cluster": params.cluster, "j_cluster": sizes["j_cluster"],
                   "leaf_bucket": params.leaf_bucket,
                   "h": ("iterated on the GPU to 200 +- 2 gather neighbors (plain start)"
                         if args.h_source == "iterated" else "the generator's (not iterated)"),
                   "l2": "inputs larger than L2 (268 MB of positions), no flush",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "stages_ms": stages,
        "roofline": {"bound": "alu", "kernel": "k_search (cluster-pair search + encode)",
                     "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "peak_kind": "measured FP32 rate (nl_probe_fp32_rate, faster of scalar "
                                  "and packed FMA chains)",
                     "frac": achieved / alu_peak,
                     "traffic": (SEARCH_DRAM_BYTES_PER_PARTICLE[args.list] * n
                                 if (M, MJ) == (8, 8) and params.leaf_bucket == 256
                                 and SEARCH_DRAM_BYTES_PER_PARTICLE.get(args.list) else None),
                     "algorithmic": "%d FP32 ops per computed pair, %d computed pairs (tiles of "
                                    "the timed %s list with the mask bit set x M x MJ)"
                                    % (ALU_OPS_PER_PAIR_SEARCH, pairs, args.list)},
        "roofline_pass": {"bound": "alu", "kernel": "k_pass (decode + density)",
                          "achieved": pass_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                          "frac": pass_achieved / alu_peak,
                          "algorithmic": "%d FP32 ops per computed pair (%d) + %d per gather "
                                         "pair or self term in range (%d + %d)"
                                         % (ALU_OPS_PER_PAIR_SEARCH, pairs,
                                            ALU_OPS_PER_DENSITY_SIDE, gather_pairs, n)},
        "fp32_peak": fp32,
        "hbm_step": {"achieved_gbs": step_bytes / (ms * 1e-3) / 1e9, "peak_gbs": hbm,
                     "peak_kind": hbm_kind,
                     "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm,
                     "bytes_per_particle": ALGO_BYTES_PER_PARTICLE},
        "list": {"kind": args.list, "bytes_per_particle": sizes["list_bytes"] / n,
                 "entries": sizes["n_entries"],
                 "computed_pairs": sizes["n_tiles"] * params.cluster * sizes["j_cluster"],
                 "nodes": sizes["n_nodes"], "leaves": sizes["n_leaves"],
                 "search_node_visits": sizes["node_visits"],
                 "search_leaf_visits": sizes["leaf_visits"],
                 "search_j_examined": sizes["j_examined"],
                 "search_tile_tests": sizes["tile_tests"]},
        "e2e": None if args.no_e2e else {
            "value": job_rate(n, ws, e_ms), "unit": UNIT,
            "h2d_bytes_per_step": 20 * n, "d2h_bytes_per_step": 4 * n},
        "h_iteration": {"plain": plain if plain is not None else {
                                  "ms": hms, "iterations": hinfo["iterations"],
                                  "rebuilds": hinfo["rebuilds"],
                                  "unconverged": hinfo["unconverged"]},
                        "learned": learned,
                        "end_to_end_ms": None if hms is None else {
                            "plain": hms + ms,
                            "learned": None if learned is None else learned["ms"] + ms}},
        "gpu_launches": None,
        "clocks": clk,
        "other_list": alt,
        "nearest_distance_pass_ms": near_ms,
    }
    out["gpu_launches"] = args.steps * launches_per_step(sizes, False,
                                                         half_list=args.list == "half")
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample or (1 << 20))
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def run_batched(args):
    """256 independent systems (log-uniform sizes 1e3..1e6, alternating periodic
    cubes and Plummer spheres), h at 100 +- 2 neighbors, one captured graph
    per step (persistent search and pass launches), autotuned parameters."""
    import torch
    import oracle
    from paper_2602_19873_gb300 import nl
    from paper_2602_19873_gb300 import workloads as wl

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    init_ranks("nccl")
    systems = wl.cached(wl.batched, "batched256_%d" % (5 + rank), 256, seed=5 + rank)
    offs = np.zeros(len(systems) + 1, np.int64)
    offs[1:] = np.cumsum([len(d["x"]) for d in systems])
    boxes = [d["box"] for d in systems]
    n = int(offs[-1])
    dev = {k: torch.from_numpy(np.concatenate([d[k] for d in systems]).astype(np.float32)).cuda()
           for k in "xyzhm"}
    stream = torch.cuda.Stream()
    base = nl.make_params(key=1, cluster=8, support=2.0, half_list=int(args.list == "half"))
    with torch.cuda.stream(stream):
        H = nl.NeighborList()
        t = time.perf_counter()
        info = H.iterate_h_batch(dev["x"], dev["y"], dev["z"], dev["h"], offs, boxes, base, 100.0,
                                 2.0, max_iter=60, start=nl.NL_HSTART_PLAIN, stream=stream)
        stream.synchronize()
        hms = (time.perf_counter() - t) * 1e3
        H.free()
        best, tune_ms = nl.autotune_batch(dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], offs,
                                          boxes, base, reps=1, stream=stream)
        rho = torch.zeros(n, dtype=torch.float32, device="cuda")
        L = nl.NeighborList()
        G = nl.Graph(L, dev["x"], dev["y"], dev["z"], dev["h"], dev["m"], rho, offs, boxes, best,
                     stream)
        quiesce_host()
        for _ in range(args.warmup):
            G.launch(stream)
        stream.synchronize()
        clocks = Clocks(local)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            G.launch(stream)
        e1.record(stream)
        stream.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws, "cuda")
        n_job = sum_over_ranks(n, ws, "cuda")
        clk = clocks.stop()
        G.check(stream)
        sizes = L.sizes()
        got = rho.cpu().numpy()
    # per-system error against the oracle on a sample of systems (the 3
    # smallest and the median): each is built alone with the tuned parameters
    # at the oracle's own smoothing lengths (exactly 100 gather neighbors), so
    # that no oracle input comes from the GPU; the full-size test covers the
    # largest systems through the graph
    order = np.argsort(np.diff(offs))
    sample = list(order[:3]) + list(order[len(order) // 2:len(order) // 2 + 1])
    worst = 0.0
    for k in sample:
        d = dict(systems[k])
        kk = oracle.keys(d["x"], d["y"], d["z"], d["box"], 1)
        perm = oracle.sort(kk)
        srt = [np.ascontiguousarray(np.asarray(d[a], np.float32)[perm]) for a in "xyzm"]
        hs = oracle.h_at_count(*srt[:3], kk[perm], d["box"], 2.0, 100)
        h = np.empty_like(hs)
        h[perm] = hs
        g_off, g_idx = oracle.gather_all(*srt[:3], hs, d["box"], 2.0)
        want = oracle.density(*srt[:3], hs, srt[3], d["box"], g_off, g_idx, np.arange(len(perm)))
        t = {a: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
             for a, v in (("x", d["x"]), ("y", d["y"]), ("z", d["z"]), ("h", h), ("m", d["m"]))}
        S = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], best)
        r = torch.empty(len(perm), dtype=torch.float32, device="cuda")
        S.density_pass(t["m"], r)
        torch.cuda.synchronize()
        S.free()
        worst = max(worst, float(np.max(np.abs(r.cpu().numpy()[perm] - want) / want)))
    out = {"metric": "batched build+density Mparticles/s (256 systems, one CUDA graph per step)",
           "value": job_rate(n_job, 1, ms), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batched_256: 256 systems, N log-uniform in [1e3, 1e6], "
                                  "even periodic uniform cubes, odd Plummer spheres, h at 100 +- 2",
                      "n": n, "systems": len(systems), "tuned": nl.params_dict(best),
                      "l2": "inputs larger than L2, no flush"},
           "h_iteration": {"plain": {"ms": hms, **{k: info[k] for k in ("iterations", "rebuilds",
                                                                         "unconverged")}}},
           "autotune_best_ms": tune_ms,
           "list": {"bytes_per_particle": sizes["list_bytes"] / n, "entries": sizes["n_entries"],
                    "computed_pairs": sizes["n_tiles"] * best.cluster * sizes["j_cluster"]},
           "per_system_max_rel_density_err": worst,
           "per_system_error_sample": [int(len(systems[k]["x"])) for k in sample],
           "gpu_launches": args.steps * launches_per_step(
               sizes, True, mixed=len({bool(np.any(b["periodic"])) for b in boxes}) > 1,
               half_list=args.list == "half"),
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


CONFIGS = {
    "uniform_32k": ("uniform_periodic_32k", "2^15 uniform particles in a periodic unit cube, "
                    "constant h for 100 neighbors, Morton keys; build + density"),
    "evrard_2m": ("evrard_2m", "2^21-particle Evrard sphere (rho ~ 1/r), h iterated to 200 +- 2; "
                  "build + density + SPH pressure force (P = 2/3 rho u, u = 0.05)"),
    "lj_fluid_4m": ("lj_fluid_4m", "4,000,000-atom jittered lattice at 100 nm^-3, periodic, "
                    "rc = 0.9 nm (about 305 neighbors); build + Lennard-Jones force"),
    "lj_coulomb_4m": ("lj_coulomb_4m", "4,000,000-atom jittered lattice at 100 nm^-3, periodic, "
                      "charges +-1; list radius 0.7816 nm (about 200 neighbors), interaction "
                      "cutoff 0.7102 nm (about 150); build + Lennard-Jones + Coulomb force, the "
                      "list rebuilt every step; 'reuse' times refresh + force on a kept list"),
}


def reuse_timing(L, d, dev, out0, args, stream, ws):
    """Steps on a kept list (Verlet buffer): positions moved by up to 0.45 of
    the skin r_list - rc, then per step nl_refresh_positions + the LJ +
    Coulomb force, timed like the rebuild steps."""
    import torch
    from paper_2602_19873_gb300 import nl
    rng = np.random.default_rng(17)
    n = len(d["x"])
    v = rng.normal(size=(n, 3))
    v *= (0.45 * (d["r_list"] - d["rc"]) * rng.random(n) / np.linalg.norm(v, axis=1))[:, None]
    Lf = np.float32(d["L"])
    moved = {}
    for a, k in enumerate(("x", "y", "z")):
        p = (np.asarray(d[k], np.float64) + v[:, a]).astype(np.float32)
        p = np.where(p < 0, p + Lf, p)
        p = np.where(p >= Lf, p - Lf, p).astype(np.float32)
        moved[k] = torch.from_numpy(np.ascontiguousarray(p)).cuda()
    md = torch.zeros(1, dtype=torch.float32, device="cuda")

    def step():
        L.refresh_positions(moved["x"], moved["y"], moved["z"], md, stream)
        L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out0, m=dev["q"], eps=d["eps"], sigma=d["sigma"],
                     rc=d["rc"], kc=d["kc"], stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, "cuda")
    return {"ms_per_step": ms, "value": job_rate(n, ws, ms), "unit": UNIT,
            "max_disp_nm": float(md.item()), "skin_nm": d["r_list"] - d["rc"]}


def run_config(args):
    """The other workloads: one step = build + the workload's passes."""
    import torch
    from paper_2602_19873_gb300 import nl
    from paper_2602_19873_gb300 import workloads as wl

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    init_ranks("nccl")
    gen, desc = CONFIGS[args.workload]
    seed = {"uniform_periodic_32k": 1, "evrard_2m": 2, "lj_fluid_4m": 3,
            "lj_coulomb_4m": 6}[gen] + 100 * rank
    d = wl.cached(wl.config, "%s_%d" % (gen, seed), gen, seed=seed)
    n = len(d["x"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda()
           for k in ("x", "y", "z", "h", "m") + (("q",) if "q" in d else ())}
    params = nl.make_params(key=d["kind"], cluster=8, support=d["support"], compress=1,
                            leaf_bucket=args.leaf_bucket, half_list=int(args.list == "half"))
    stream = torch.cuda.current_stream()
    if gen == "evrard_2m":  # smoothing lengths at 200 +- 2 neighbors (untimed input preparation)
        H = nl.NeighborList()
        H.iterate_h(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], params, 200.0, 2.0,
                    max_iter=60, margin=0.15, start=nl.NL_HSTART_PLAIN, stream=stream)
        H.free()
    L = nl.NeighborList()
    L.set_profiling(True)
    out0 = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    pres = None
    if gen == "evrard_2m":  # pressure from a density pass (an input field of the force pass)
        L.build(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], params, stream)
        L.density_pass(dev["m"], rho, stream)
        pres = rho * (2.0 / 3.0 * 0.05)

    def step():
        L.build(dev["x"], dev["y"], dev["z"], dev["h"], d["box"], params, stream)
        if gen == "lj_fluid_4m":
            L.force_pass(nl.NL_FORCE_LJ, *out0, eps=1.0, sigma=0.3, stream=stream)
        elif gen == "lj_coulomb_4m":
            L.force_pass(nl.NL_FORCE_LJ_COULOMB, *out0, m=dev["q"], eps=d["eps"],
                         sigma=d["sigma"], rc=d["rc"], kc=d["kc"], stream=stream)
        else:
            L.density_pass(dev["m"], rho, stream)
            if gen == "evrard_2m":
                L.force_pass(nl.NL_FORCE_SPH_PRESSURE, *out0, m=dev["m"], rho=rho, pres=pres,
                             stream=stream)

    quiesce_host()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, "cuda")
    clk = clocks.stop()
    sizes = L.sizes()
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    L.neighbor_counts(cnt, stream)
    useful = int(cnt.sum().item())
    pairs = sizes["n_tiles"] * params.cluster * sizes["j_cluster"]
    out = {"metric": "build+pass Mparticles/s (%s)" % args.workload,
           "value": job_rate(n, ws, ms), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%s: %s" % (args.workload, desc), "n": n, "list": args.list,
                      "l2": "inputs larger than L2 except uniform_32k (no flush)"},
           "stages_ms": L.stage_times(),
           "list": {"bytes_per_particle": sizes["list_bytes"] / n, "entries": sizes["n_entries"],
                    "computed_pairs": pairs, "gather_pairs": useful,
                    "cluster_overhead": pairs / float(useful + n)},
           "e2e": None, "gpu_launches": None, "clocks": clk}
    if gen == "lj_coulomb_4m":
        out["reuse"] = reuse_timing(L, d, dev, out0, args, stream, ws)
    if rank == 0 and not args.no_cpu_baseline:
        ns = min(n, args.cpu_sample or (1 << 18))
        samp = wl.config(gen, scale=ns / float(n), seed=seed)
        import oracle
        oracle.build()
        t = time.perf_counter()
        oracle_step(samp)
        dt = time.perf_counter() - t
        out["cpu_baseline"] = {"value": len(samp["x"]) / dt / 1e6, "unit": UNIT,
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "oracle build + %s of the same generator at %d "
                                         "particles, %.1f s" % (
                                             "LJ + Coulomb force" if "q" in samp else "density",
                                             len(samp["x"]), dt)}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args):
    """List size and cluster overhead against the neighbor count on the LJ
    fluid (100 nm^-3): 8x8 and 8x4 tiles, compressed and raw lists, full and
    (8x8) half lists, build and pass times (Lennard-Jones on full lists,
    density on half lists)."""
    import torch
    from paper_2602_19873_gb300 import nl
    from paper_2602_19873_gb300 import workloads as wl
    torch.cuda.set_device(0)
    d = wl.cached(wl.config, "lj_fluid_4m_3", "lj_fluid_4m", seed=3)
    n = len(d["x"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda()
           for k in ("x", "y", "z", "m")}
    stream = torch.cuda.current_stream()
    out0 = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    rows = []
    quiesce_host()
    for nb in (25, 50, 100, 200, 400, 800, 1600):
        rc = (3.0 * nb / (4.0 * math.pi * 100.0)) ** (1.0 / 3.0)
        h = torch.full((n,), rc, dtype=torch.float32, device="cuda")
        for (M, MJ, half) in ((8, 8, 0), (8, 4, 0), (8, 8, 1)):
            for comp in (1, 0):
                p = nl.make_params(key=1, cluster=M, j_cluster=MJ, support=1.0, compress=comp,
                                   half_list=half)
                L = nl.NeighborList()
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                for r in range(4):
                    if r == 3:
                        e[0].record(stream)
                    L.build(dev["x"], dev["y"], dev["z"], h, d["box"], p, stream)
                    if r == 3:
                        e[1].record(stream)
                    if half:  # half lists serve the density and count passes
                        L.density_pass(dev["m"], out0[0], stream)
                    else:
                        L.force_pass(nl.NL_FORCE_LJ, *out0, eps=1.0, sigma=0.3, stream=stream)
                    if r == 3:
                        e[2].record(stream)
                torch.cuda.synchronize()
                sz = L.sizes()
                if (M, MJ, comp, half) == (8, 8, 1, 0):
                    L.neighbor_counts(cnt, stream)
                    useful = int(cnt.sum().item())
                pairs = sz["n_tiles"] * M * MJ
                rows.append({"neighbors_target": nb, "rc_nm": rc, "tile": "%dx%d" % (M, MJ),
                             "list": "half" if half else "full",
                             "compressed": bool(comp),
                             "mean_neighbors": useful / n,
                             "bytes_per_particle": sz["list_bytes"] / n,
                             "full_list_bytes_per_particle": 4.0 * useful / n,
                             "cluster_overhead": pairs / float(useful + n) * (2 if half else 1),
                             "build_ms": e[0].elapsed_time(e[1]),
                             ("density_pass_ms" if half else "lj_pass_ms"): e[1].elapsed_time(e[2])})
                L.free()
    print(json.dumps({"sweep": "LJ fluid 4,000,000 atoms at 100 nm^-3, periodic, Hilbert keys, "
                               "leaf bucket 256; list radius for the target neighbor count",
                      "rows": rows}))


def oracle_step(d):
    """The oracle's build + density on one system: keys, stable sort, FP64
    cell-list gather sets, symmetric sets, per-super-cluster records, density."""
    import oracle
    k = oracle.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    perm = oracle.sort(k)
    s = [np.ascontiguousarray(d[a][perm]) for a in ("x", "y", "z", "h", "m")]
    g_off, g_idx = oracle.gather_all(*s[:4], d["box"], d["support"])
    p_off, p_idx = oracle.symmetrize(g_off, g_idx)
    n = len(s[0])
    nsc = (n + 63) // 64
    so, J, m = oracle.cluster_lists(n, 8, p_off, p_idx, np.arange(n), np.arange(nsc))
    nbytes = 0
    for t in range(nsc):
        nbytes += len(oracle.encode_record(J[so[t]:so[t + 1]], m[so[t]:so[t + 1]], 32, True))
    if "q" in d:  # LJ + Coulomb over the pairs within the interaction cutoff
        hr = np.full(n, np.float32(d["rc"]), np.float32)
        i_off, i_idx = oracle.gather_all(*s[:3], hr, d["box"], 1.0)
        f = oracle.ljc_force(*s[:3], d["box"], d["eps"], d["sigma"], d["q"][perm], d["kc"],
                             i_off, i_idx, np.arange(n))
        return f, nbytes
    rho = oracle.density(*s, d["box"], g_off, g_idx, np.arange(n))
    return rho, nbytes


def cpu_baseline(n_sample):
    import oracle
    from paper_2602_19873_gb300 import workloads as wl
    oracle.build()
    d = wl.plummer(n_sample, n_spheres=64, seed=4)
    t = time.perf_counter()
    oracle_step(d)
    dt = time.perf_counter() - t
    return {"value": n_sample / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "one oracle build+density of the same generator at %d particles "
                      "(64 Plummer spheres), %.1f s" % (n_sample, dt)}


def run_reference(args):
    ws, rank, local = dist_init()
    if rank != 0:
        return
    import oracle
    from paper_2602_19873_gb300 import workloads as wl
    oracle.build()
    ns = reference_sample(args.steps, args.warmup, args.cpu_sample)
    d = wl.plummer(ns, n_spheres=64, seed=4)
    for _ in range(args.warmup):
        oracle_step(d)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(d)
    dt = (time.perf_counter() - t) / args.steps
    v = ns / dt / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "%s generator at %d particles (bounded CPU sample)" % (
               WORKLOAD, ns)},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle",
                            "sample": "%d particles of the 64-Plummer-sphere generator" % ns},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="particles of the CPU oracle sample (default: 2^20 for cpu_baseline; "
                         "sized to the step count for --impl reference)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=N_FULL,
                    help="particles (smaller cases are for profiling only)")
    ap.add_argument("--reuse-h", action="store_true",
                    help="reuse converged h cached by an earlier run with the same n")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--threads", type=int, default=0, choices=[0, 128, 256],
                    help="search / pass block size of the single-system bench (0: library default)")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="persistent blocks per SM of the single-system bench (0: library default)")
    ap.add_argument("--leaf-bucket", type=int, default=256,
                    help="octree leaf capacity of the single-system bench")
    ap.add_argument("--tile", default="8x8", choices=["8x8", "8x4", "16x8", "16x16", "4x4"],
                    help="i-cluster x j-cluster size of the single-system bench")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-h comparison")
    ap.add_argument("--h-source", default="iterated", choices=["iterated", "generator"],
                    help="smoothing lengths of the timed step: iterated to 200 +- 2 (the "
                         "benchmark), or the generator's (short profiling runs)")
    ap.add_argument("--h-reps", type=int, default=5,
                    help="timed h iterations per start (median and spread reported)")
    ap.add_argument("--list", default="half", choices=["full", "half"],
                    help="full lists, or half lists (every cluster pair once; density workloads)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batched_256"] + sorted(CONFIGS))
    ap.add_argument("--sweep", action="store_true",
                    help="list size / cluster overhead / times against the neighbor count (LJ fluid)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.workload == "batched_256":
        run_batched(args)
    elif args.workload in CONFIGS:
        run_config(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
