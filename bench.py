"""Benchmark: tets/s of VT+VV+ET+TT built for every cluster of the 256^3
Freudenthal grid (16.97M vertices, 100.7M tets, jitter +-0.3 cell, permuted
ids, kd-tree leaves of <= 512 vertices -> 65,536 clusters), batched form.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one full build of all four relations of all clusters
(gale_build_clusters(all, VT|VV|ET|TT, batched)), the mesh already loaded
and resident in HBM.  Prints one JSON line (rank 0).

* value      device-timed throughput (CUDA events on the context stream,
             max over ranks); inputs (1.97 GB of cluster working sets) and
             outputs (8.1 GB) are far larger than L2, so no flush is needed.
* e2e        the same metric through the C ABI with host buffers: every
             step copies the requested cluster ids from host memory, builds,
             and copies every relation array back to pinned host memory
             (gale_build_export: chunks of clusters are copied out while the
             next chunk builds).
* roofline   algorithmic bytes of the build (working sets read once,
             relations written once) / measured step time, against the
             measured HBM copy bandwidth.
* cpu_baseline  the CPU oracle on a bounded sample of the same recipe (a
             96^3 grid), one copy per host core at once, tets/s (and the
             single-thread figure).
* per_cluster   the baseline form: one kernel launch per cluster, timed on
             a subset of the clusters.

--impl reference times the CPU oracle (the only reference this method has)
on bounded samples of the same workload family, one copy per host core.
N > 1 (torchrun): every rank builds its own replica of the mesh (weak
scaling, no data-path collective; only the timing barrier).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "tets/s of VT+VV+ET+TT built; p50/p99 cluster latency vs per-cluster launches"
UNIT = "tets/s"
N_GRID = 256
CPU_SAMPLE_N = 96        # the global-definition oracle, one copy per host core
LOCAL_SAMPLE_N = 128     # the per-cluster localized oracle on every host core
LOCAL_SINGLE_N = 64      # ... and on one core
REF_SAMPLE_N = 64


def read_bytes(info):
    """Algorithmic reads of a full build: every owned tet row once (16 B),
    and for every external and halo tet its index and its gathered row
    (4 + 16 B).  The writes are the relation arrays themselves."""
    return 16 * int(info.nt) + 20 * int(info.ext_tets) + 20 * int(info.halo_tets)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self._stop = threading.Event()
        self._th = None
        self._proc = None

    def _run(self):
        for line in self._proc.stdout:
            row = [c.strip() for c in line.split(",")]
            if len(row) >= 5 and not self._stop.is_set():
                self.rows.append(row)

    def __enter__(self):
        # one nvidia-smi process that prints a line every 50 ms
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                           "--format=csv,noheader,nounits", "-lms", "50"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return self
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_setup(n_gpus: int):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_oracle(n: int, seed: int = 3, mesh=None):
    """Whole oracle pipeline (checks, canonical numbering, VT/VV/ET/TT) on an
    n^3 grid of the same recipe (or on `mesh`); returns (tets, seconds,
    clusters)."""
    import gen
    import oracle
    m = mesh if mesh is not None else gen.freudenthal_mesh(n, 512, seed=seed, jitter=0.3, with_field=False)
    t0 = time.perf_counter()
    oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    return m.nt, time.perf_counter() - t0, m.nclusters


def time_oracle_cores(mesh, threads: int, warm: bool = True):
    """The whole oracle pipeline run `threads` times at once, one copy per
    host thread, on the same sample mesh (the C oracle holds no shared state
    and its calls release the interpreter lock); returns (tets, seconds)."""
    import concurrent.futures as cf
    import oracle
    if warm:
        oracle.build_all(mesh.nv, mesh.tv, mesh.seg, mesh.nclusters)  # library loaded, pages warm
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda _: oracle.build_all(mesh.nv, mesh.tv, mesh.seg, mesh.nclusters), range(threads)))
    return threads * mesh.nt, time.perf_counter() - t0


def time_localized(mesh, threads: int):
    """The oracle's per-cluster localized producer on `mesh` with `threads`
    threads over the clusters: (tets, initialisation seconds, build
    seconds).  The canonical numbering is the oracle's own and is not timed;
    the initialisation gathers every cluster's working set once."""
    import oracle
    canon = oracle.canonicalize(mesh.nv, mesh.tv, mesh.seg, mesh.nclusters)
    _, _, (init_s, build_s) = oracle.localized_build(canon, threads, digests=False)
    return mesh.nt, init_s, build_s


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def ref_config(args) -> dict:
    """The workload our arm measures (the reference arm times bounded samples
    of it): the grid's vertex and tet counts in closed form, and its kd leaf
    count (halving to <= 512 vertices gives a power of two)."""
    n = args.grid
    nv, nt = (n + 1) ** 3, 6 * n ** 3
    k = 1
    while nv / k > 512:
        k *= 2
    return {"workload": f"grid{n}^3-jitter0.3-kd512: {nv} vertices, {nt} tets, {k} clusters",
            "relations": "VT+VV+ET+TT, canonical sorted CSR",
            "mode": "CPU oracle, one copy per host thread, on bounded grid samples of the same recipe",
            "parallelism": "rank 0 only"}


def run_reference(args, rank, dist):
    if rank != 0:
        return
    import gen
    # each step is the oracle's per-cluster localized producer on one grid
    # sample of the same recipe, on every host core; the sample keeps the
    # whole run near a minute (the producer builds a few M tets/s)
    budget_s = 60.0 / max(1, args.steps + args.warmup)
    n = int(max(16, min(REF_SAMPLE_N, round((budget_s * 2e6 / 6.0) ** (1.0 / 3.0)))))
    mesh = gen.freudenthal_mesh(n, 512, seed=3, jitter=0.3, with_field=False)
    cores = host_cores()
    for _ in range(args.warmup):
        time_localized(mesh, cores)
    tets, secs, init = 0, 0.0, 0.0
    for _ in range(args.steps):
        t, i_s, b_s = time_localized(mesh, cores)
        tets += t
        secs += b_s
        init += i_s
    v = tets / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": ref_config(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle per-cluster localized",
                             "sample": f"each step: the oracle's per-cluster localized producer on a {n}^3 grid "
                                       f"of the same recipe ({tets // args.steps} tets, kd leaves <= 512), "
                                       f"{cores} threads over the clusters; the per-cluster builds are timed, "
                                       f"the working-set initialisation ({init / args.steps:.2f} s per step) "
                                       f"is not, as the GPU value leaves out the mesh load"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100,
                    help="timed build steps (100 x ~9 ms keeps the clock sampler running through about a second)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=N_GRID, help="grid cubes per axis (256 = the at-scale workload)")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--per-cluster-sample", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default block sizes")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 24-mesh mixed serving leg (about two minutes)")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the irregular batched leg (2M-point Delaunay, uneven kd leaves)")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="also sweep serving prefetch depth x cache budget on the 256^3 mesh (minutes)")
    ap.add_argument("--no-coboundary", action="store_true", help="skip timing VE, VF, EF, FT (128^3 grid)")
    ap.add_argument("--coboundary-grid", type=int, default=128)
    ap.add_argument("--discrete-gradient", action="store_true",
                    help="also time the discrete-gradient consumer and the relations it reads")
    ap.add_argument("--dg-grid", type=int, default=128)
    ap.add_argument("--dg-threads", type=int, default=0, help="consumer threads (0: the host's cores)")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: each rank builds a balanced shard of the clusters (strong scaling) "
                         "instead of a whole replica")
    ap.add_argument("--mixed-scale", type=float, default=1.0)
    ap.add_argument("--mixed-requests", type=int, default=4000)
    ap.add_argument("--mixed-budget-gb", type=float, default=20.0)
    ap.add_argument("--serve-threads", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    ap.add_argument("--serve-stress-gb", type=float, default=1.0,
                    help="cache budget of the LRU stress variant of the serving leg (0: skip it)")
    ap.add_argument("--serve-baseline-clusters", type=int, default=2048)
    ap.add_argument("--serve-prefetch", type=int, default=4, help="prefetch depth of the serving variant (0: off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch

    import gen
    import paper_2507_15230_gb300 as gale

    torch.cuda.set_device(local)
    mesh = gen.scale_grid(args.grid)
    ctx = gale.Context.load(mesh, device=local, cache_budget_bytes=int(args.serve_budget_gb * (1 << 30)))
    info = ctx.info()
    stream = torch.cuda.ExternalStream(ctx.stream_handle)
    tuned = None
    if not args.no_autotune:
        # block size and CTAs per SM of every size bin, chosen by timing
        tuned = {"best_ms_per_bin": ctx.autotune(gale.ALL)}

    # which clusters this rank builds: all of them (replicas, weak scaling),
    # or its balanced contiguous shard (--shard, strong scaling)
    shard_ids, shard_info = None, None
    if args.shard and world > 1:
        from paper_2507_15230_gb300 import shard as gshard
        I_V, I_T, sizes = ctx.intervals()
        lo_k, hi_k = gshard.shard_ranges(np.diff(I_T) + 1, world)[rank]
        shard_ids = np.arange(lo_k, hi_k, dtype=np.int32)
        edge0, edges = gshard.edge_base(int(sizes[lo_k:hi_k, 2].sum()), dist)
        shard_info = {"clusters": [int(lo_k), int(hi_k)], "first_global_edge": edge0, "edges": edges}
    my_tets = mesh.nt if shard_ids is None else int(np.diff(ctx.intervals()[1])[shard_ids].sum())

    # warm-up (also captures the batched graph)
    for _ in range(args.warmup):
        ctx.build(shard_ids, gale.ALL, gale.MODE_BATCHED)
    ctx.synchronize()
    _, lens = ctx.bulk_arrays()
    out_bytes = 4 * sum(lens.values())
    in_bytes = read_bytes(info)
    if shard_ids is not None:  # this rank's working sets, in proportion to its tets
        in_bytes = int(in_bytes * my_tets / mesh.nt)
    alg_bytes = in_bytes + out_bytes

    # timed region: device throughput
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for a, b in step_ev:
            a.record(stream)
            ctx.build(shard_ids, gale.ALL, gale.MODE_BATCHED)
            b.record(stream)
            launches += ctx.last_launch_count()
        e1.record(stream)
        ctx.synchronize()
        torch.cuda.synchronize()
    barrier(dist)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(dist, ms)
    per_step = [a.elapsed_time(b) for a, b in step_ev]
    step_ms = statistics.mean(per_step)
    # every rank's work counts: replicas build the whole mesh each, shards
    # split it (the slowest rank's time, max over ranks)
    value = (world * mesh.nt if shard_ids is None else mesh.nt) / (ms / 1000.0)
    peak, peak_src = load_peaks()
    achieved = alg_bytes / (step_ms / 1000.0) / 1e9

    # end to end through the C ABI with host buffers
    ids = (torch.arange(ctx.K, dtype=torch.int32) if shard_ids is None
           else torch.from_numpy(shard_ids.copy())).pin_memory()
    ids_np = ids.numpy()
    host = {n: torch.empty(lens[n], dtype=torch.int32).pin_memory() for n in lens}
    host_np = {n: t.numpy() for n, t in host.items()}
    for _ in range(5):  # untimed: first touch of the pinned pages, warm paths
        ctx.build_export(ids_np, gale.ALL, out=host_np)
    barrier(dist)
    e2e_step_s = []
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            # ids in, every relation array out; chunk copies overlap the build
            ts = time.perf_counter()
            ctx.build_export(ids_np, gale.ALL, out=host_np)  # blocks until the copies are done
            e2e_step_s.append(time.perf_counter() - ts)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(dist, e2e_s)
    e2e_value = (world * mesh.nt if shard_ids is None else mesh.nt) / e2e_s

    # baseline form: one launch per cluster, on a subset
    per_cluster = None
    if rank == 0 and args.per_cluster_sample > 0:
        sub = np.arange(min(args.per_cluster_sample, ctx.K), dtype=np.int32)
        ctx.build(sub, gale.ALL, gale.MODE_PER_CLUSTER)
        ctx.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.build(sub, gale.ALL, gale.MODE_PER_CLUSTER)
        b.record(stream)
        ctx.synchronize()
        pms = a.elapsed_time(b)
        _, I_T, _ = ctx.intervals()
        sub_tets = int(I_T[sub[-1] + 1] - I_T[sub[0]])
        # the same subset, batched
        ctx.build(sub, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        a.record(stream)
        ctx.build(sub, gale.ALL, gale.MODE_BATCHED)
        b.record(stream)
        ctx.synchronize()
        bms = a.elapsed_time(b)
        per_cluster = {"clusters": int(sub.size), "tets": sub_tets,
                       "per_cluster_launch_tets_per_s": sub_tets / (pms / 1000.0),
                       "batched_same_subset_tets_per_s": sub_tets / (bms / 1000.0),
                       "per_cluster_ms": pms, "batched_ms": bms}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import gen as _gen
        cores = host_cores()
        big = _gen.freudenthal_mesh(LOCAL_SAMPLE_N, 512, seed=3, jitter=0.3, with_field=False)
        lt, li, lb = time_localized(big, cores)
        small = _gen.freudenthal_mesh(LOCAL_SINGLE_N, 512, seed=3, jitter=0.3, with_field=False)
        st_t, _, st_b = time_localized(small, 1)
        # the global-definition oracle, one copy per core (a second figure)
        sample = _gen.freudenthal_mesh(CPU_SAMPLE_N, 512, seed=3, jitter=0.3, with_field=False)
        gtets, gsecs = time_oracle_cores(sample, cores, warm=True)
        cpu = {"value": lt / lb, "unit": UNIT, "cores": cores, "kind": "oracle per-cluster localized",
               "sample": f"grid{LOCAL_SAMPLE_N}^3-jitter0.3-kd512 ({big.nt} tets, {big.nclusters} clusters): the "
                         f"oracle's per-cluster localized producer, {cores} threads over the clusters; per-cluster "
                         f"builds timed ({lb:.2f} s), working-set initialisation not ({li:.2f} s)",
               "single_thread_value": st_t / st_b,
               "single_thread_sample": f"grid{LOCAL_SINGLE_N}^3 ({small.nt} tets), one thread",
               "global_oracle_copies": {"value": gtets / gsecs, "cores": cores,
                                        "sample": f"grid{CPU_SAMPLE_N}^3 ({sample.nt} tets): the whole global-"
                                                  f"definition oracle pipeline, one copy per host thread"}}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serve_leg(args, mesh, ctx, gale)
    mixed = None
    if rank == 0 and not args.no_mixed:
        mixed = mixed_leg(args, gale)
    config3 = None
    if rank == 0 and not args.no_config3:
        config3 = config3_leg(args, gale, gen)
    sweep = None
    if rank == 0 and args.serve_sweep:
        sweep = serve_sweep_leg(args, mesh, ctx, gale)
    cobound = None
    if rank == 0 and not args.no_coboundary:
        cobound = coboundary_leg(args, gale, gen)
    dgrad = None
    if rank == 0 and args.discrete_gradient:
        dgrad = gradient_leg(args, gale, gen)

    traffic = None
    tp = os.path.join(ROOT, "profiles", "build_kernel_traffic.json")
    if os.path.exists(tp):
        try:
            with open(tp) as f:
                t = json.load(f)
            if t.get("kernel_source_sha") == gale_kernel_sha() and t.get("grid") == args.grid:
                traffic = t.get("bytes_per_launch")
        except Exception:
            traffic = None

    if rank == 0:
        clocks = clk.summary()
        clocks["e2e_region"] = clk_e2e.summary()
        clk.rows += clk_e2e.rows
        both = clk.summary()
        clocks["both_regions"] = {"sm_mhz": both["sm_mhz"], "samples": both["samples"], "reasons": both["reasons"]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak" if shard_ids is None else "strong",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"grid{args.grid}^3-jitter0.3-kd512: {mesh.nv} vertices, {mesh.nt} tets, "
                                   f"{mesh.nclusters} clusters",
                       "relations": "VT+VV+ET+TT, canonical sorted CSR", "mode": "batched persistent kernels, "
                       "CUDA graph replay",
                       "parallelism": f"replicas x{world}" if shard_ids is None else f"cluster shards x{world}",
                       "l2": f"no flush: {in_bytes / 1e9:.2f} GB of inputs and {out_bytes / 1e9:.2f} GB of outputs "
                             f"per step exceed the 129 MB L2"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(ids.numel() * 4),
                    "d2h_bytes_per_step": int(out_bytes), "ms_per_step": [1e3 * x for x in e2e_step_s]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_src},
            "cpu_baseline": cpu,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "per_cluster": per_cluster,
            "serving": serving,
            "mixed_serving": mixed,
            "config3": config3,
            "serve_sweep": sweep,
            "coboundary": cobound,
            "discrete_gradient": dgrad,
            "shard": shard_info,
            "load_seconds": {"host": info.load_host_seconds, "device": info.load_device_seconds},
            "bins": ctx.bins(),
            "autotune": None if tuned is None else {"best_ms_per_bin": tuned["best_ms_per_bin"]},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def serve_leg(args, mesh, ctx, gale):
    """Critical-point consumers (16 threads) classify every vertex through
    gale_request (VT+VV+TT, HBM-budgeted cache, device-resident loop); the
    baseline serves a bounded subset with one kernel launch per request."""
    import consumers
    import gen
    n = args.grid
    field = gen.gaussian_field(mesh.xyz, 16, [0, 0, 0], [n, n, n], 4)
    vperm, _ = ctx.permutations()
    f_c, inid = consumers.canonical_inputs(field, vperm)
    rows = ctx.rows()
    I_V, I_T, _ = ctx.intervals()
    mask = gale.VT | gale.VV | gale.TT

    def summarize(lat, st, nclusters):
        lat = lat[:nclusters]
        tets = int(I_T[nclusters] - I_T[0])
        return {"requests": st["requests"], "failures": st["failures"],
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "wall_s": st["wall"], "tets_per_s": tets / st["wall"], "d2h_bytes": st["d2h_bytes"]}

    def breakdown(s, st):
        """Mean waiting time per request by stage, the stages of the paper's
        breakdown (Section 5.3): enqueue, in queue, preparation, device
        (kernel), copy to host, integration; plus the request's whole wait."""
        n = max(1, int(s.requests))
        us = lambda ns: ns / n / 1e3
        return {"per_request_us": {"enqueue": us(s.t_enqueue_ns), "in_queue": us(s.t_queue_ns),
                                   "preparation": us(s.t_prepare_ns), "device": us(s.t_build_ns),
                                   "device_build_alone": us(s.t_kernel_ns),
                                   "copy_to_host": st["copy_s"] * 1e6 / n, "integration": st["integrate_s"] * 1e6 / n,
                                   "request_wait": us(s.t_wait_ns)},
                "max_request_wait_ms": s.max_wait_ns / 1e6,
                "queue_depth_hist": {f"{1 << b}-{(2 << b) - 1}" if b < 11 else "2048+": int(s.depth_hist[b])
                                     for b in range(12) if s.depth_hist[b]}}

    ctx.serve_configure(gale.SERVE_LOOP)
    cls, lat, st = consumers.serve_run(ctx, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask)
    loop = summarize(lat, st, ctx.K)
    s = ctx.serve_stats()
    loop.update({"builds": s.builds, "hits": s.hits, "evictions": s.evictions, "loop_launches": s.batches,
                 "critical_points": {str(c): int((cls == c).sum()) for c in (0, 1, 2, 3, 4)},
                 "wait_breakdown": breakdown(s, st)})
    # proactive prefetch (Section 4.5): each request also queues the next
    # clusters, which the kd-order walks request next
    pref = None
    if args.serve_prefetch > 0:
        with gale.Context.load(mesh, device=0, cache_budget_bytes=int(args.serve_budget_gb * (1 << 30))) as cp:
            cp.serve_configure(gale.SERVE_LOOP, prefetch=args.serve_prefetch)
            _, latp, stp = consumers.serve_run(cp, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask)
            pref = summarize(latp, stp, cp.K)
            sp = cp.serve_stats()
            pref.update({"prefetch_depth": args.serve_prefetch, "builds": sp.builds, "hits": sp.hits,
                         "prefetches": sp.prefetches, "prefetch_hits": sp.prefetch_hits,
                         "prefetch_dropped": sp.prefetch_dropped, "evictions": sp.evictions,
                         "wait_breakdown": breakdown(sp, stp)})
    # LRU stress: the same walk under a small budget, so finished clusters
    # are evicted to admit new ones
    stress = None
    if args.serve_stress_gb > 0:
        with gale.Context.load(mesh, device=0, cache_budget_bytes=int(args.serve_stress_gb * (1 << 30))) as cs:
            cs.serve_configure(gale.SERVE_LOOP)
            _, lats, sts = consumers.serve_run(cs, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask)
            stress = summarize(lats, sts, cs.K)
            ss = cs.serve_stats()
            stress.update({"budget_gb": args.serve_stress_gb, "builds": ss.builds, "hits": ss.hits,
                           "evictions": ss.evictions, "wait_breakdown": breakdown(ss, sts)})
    base = None
    nb = min(args.serve_baseline_clusters, ctx.K)
    if nb > 0:
        with gale.Context.load(mesh, device=0, cache_budget_bytes=int(args.serve_budget_gb * (1 << 30))) as c2:
            c2.serve_configure(gale.SERVE_SINGLE)
            _, lat2, st2 = consumers.serve_run(c2, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask,
                                               max_clusters=nb)
            base = summarize(lat2, st2, nb)
            base["clusters"] = nb
            base["wait_breakdown"] = breakdown(c2.serve_stats(), st2)
        # the same subset through the loop, fresh cache
        with gale.Context.load(mesh, device=0, cache_budget_bytes=int(args.serve_budget_gb * (1 << 30))) as c3:
            c3.serve_configure(gale.SERVE_LOOP)
            _, lat3, st3 = consumers.serve_run(c3, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask,
                                               max_clusters=nb)
            loop_sub = summarize(lat3, st3, nb)
            loop_sub["clusters"] = nb
            loop_sub["wait_breakdown"] = breakdown(c3.serve_stats(), st3)
    # the producer alone: the same walks with consumers that release each
    # view as soon as it is served (no copy to host, no classification)
    producer = {}
    for key, mode, ncl in (("device_loop", gale.SERVE_LOOP, ctx.K), ("device_loop_subset", gale.SERVE_LOOP, nb),
                           ("per_request_launch_subset", gale.SERVE_SINGLE, nb)):
        if ncl <= 0:
            continue
        with gale.Context.load(mesh, device=0, cache_budget_bytes=int(args.serve_budget_gb * (1 << 30))) as cn:
            cn.serve_configure(mode)
            _, latn, stn = consumers.serve_run(cn, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask,
                                               max_clusters=ncl, null_work=True)
            r = summarize(latn, stn, ncl)
            r.update({"clusters": ncl, "req_per_s": stn["requests"] / stn["wall"],
                      "wait_breakdown": breakdown(cn.serve_stats(), stn)})
            producer[key] = r
    return {"workload": f"{args.serve_threads} critical-point consumer threads, kd-order walks with 10% random "
                        f"jumps, VT+VV+TT requests, {args.serve_budget_gb:g} GB cache budget, field = 16 Gaussians",
            "device_loop": loop, "device_loop_prefetch": pref, "device_loop_lru_stress": stress,
            "per_request_launch_subset": base,
            "device_loop_same_subset": loop_sub if nb > 0 else None,
            "producer_only": producer}


def serve_sweep_leg(args, mesh, ctx, gale):
    """Prefetch depth x cache budget on the 256^3 serving workload (16
    critical-point consumers, VT+VV+TT): p50/p99 request latency, builds,
    prefetch hits and drops, evictions, wall time."""
    import consumers
    import gen
    n = args.grid
    field = gen.gaussian_field(mesh.xyz, 16, [0, 0, 0], [n, n, n], 4)
    vperm, _ = ctx.permutations()
    f_c, inid = consumers.canonical_inputs(field, vperm)
    rows = ctx.rows()
    I_V, I_T, _ = ctx.intervals()
    mask = gale.VT | gale.VV | gale.TT
    out = []
    for budget_gb in (8.0, 1.0):
        for depth in (0, 1, 2, 4, 8):
            with gale.Context.load(mesh, device=0, cache_budget_bytes=int(budget_gb * (1 << 30))) as c:
                c.serve_configure(gale.SERVE_LOOP, prefetch=depth)
                _, lat, st = consumers.serve_run(c, f_c, inid, rows, I_V, nthreads=args.serve_threads, mask=mask)
                s = c.serve_stats()
                out.append({"budget_gb": budget_gb, "prefetch_depth": depth,
                            "p50_ms": float(np.percentile(lat, 50) * 1e3),
                            "p99_ms": float(np.percentile(lat, 99) * 1e3), "wall_s": st["wall"],
                            "tets_per_s": int(I_T[-1] - I_T[0]) / st["wall"], "builds": s.builds,
                            "prefetches": s.prefetches, "prefetch_hits": s.prefetch_hits,
                            "prefetch_dropped": s.prefetch_dropped, "evictions": s.evictions})
    return {"workload": f"grid{n}^3 serving, {args.serve_threads} critical-point consumers, VT+VV+TT", "runs": out}


def config3_leg(args, gale, gen):
    """Irregular batched workload: the Delaunay tetrahedralisation of 2M
    Gaussian-mixture points with uneven kd leaves of 32 to 2,048 vertices.
    All clusters are built by the size-binned persistent kernels replayed
    from a captured CUDA graph, with block sizes and CTAs per SM chosen by
    the autotuner; reported: tets/s, the roofline fraction of the build,
    each bin's time alone, and the one-launch-per-cluster form on the same
    clusters."""
    import torch
    t0 = time.perf_counter()
    mesh = gen.delaunay_mesh(2_000_000, seed=5, with_field=False)
    gen_s = time.perf_counter() - t0
    with gale.Context.load(mesh, device=0) as c:
        info = c.info()
        stream = torch.cuda.ExternalStream(c.stream_handle)
        tuned = c.autotune(gale.ALL)
        for _ in range(3):
            c.build(None, gale.ALL, gale.MODE_BATCHED)
        c.synchronize()
        _, lens = c.bulk_arrays()
        alg = read_bytes(info) + 4 * sum(lens.values())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 20
        a.record(stream)
        for _ in range(steps):
            c.build(None, gale.ALL, gale.MODE_BATCHED)
        b.record(stream)
        c.synchronize()
        ms = a.elapsed_time(b) / steps
        # the baseline form on the same clusters: one launch per cluster
        c.build(None, gale.ALL, gale.MODE_PER_CLUSTER)
        c.synchronize()
        a.record(stream)
        c.build(None, gale.ALL, gale.MODE_PER_CLUSTER)
        b.record(stream)
        c.synchronize()
        pms = a.elapsed_time(b)
        I_V, _, _ = c.intervals()
        leaf = np.diff(I_V)
        bins = c.bins()
    peak, _ = load_peaks()
    return {"workload": f"delaunay 2M points (70% 8 Gaussians, 30% uniform): {mesh.nv} vertices, {mesh.nt} tets, "
                        f"{mesh.nclusters} kd leaves of {int(leaf.min())}..{int(leaf.max())} vertices",
            "generation_s": gen_s,
            "load_seconds": {"host": info.load_host_seconds, "device": info.load_device_seconds,
                             "parts": int(info.nparts)},
            "ms_per_step": ms, "tets_per_s": mesh.nt / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peak, "algorithmic_bytes_per_launch": alg},
            "per_cluster_launch": {"ms": pms, "tets_per_s": mesh.nt / (pms / 1e3), "launches": int(mesh.nclusters)},
            "bins": bins, "best_ms_per_bin": tuned}


def mixed_meshes(scale: float = 1.0):
    """The mixed serving workload: Freudenthal grids n = 32, 48, ..., 192 (kd
    leaves <= 512, jitter 0.3, seed 7 + i) and Delaunay meshes of 100k .. 1M
    Gaussian-mixture points, log-spaced (uneven kd leaves, seed 18 + i).
    scale < 1 shrinks every mesh (grid edge and point count) for quick runs."""
    import gen
    meshes = []
    for i, n in enumerate(range(32, 193, 16)):
        nn = max(4, int(round(n * scale)))
        meshes.append(gen.freudenthal_mesh(nn, 512, seed=7 + i, field_seed=100 + i, jitter=0.3, with_field=False,
                                           name=f"grid{nn}^3"))
    for i, p in enumerate(np.geomspace(1e5, 1e6, 13)):
        npts = max(2000, int(p * scale ** 3))
        meshes.append(gen.delaunay_mesh(npts, seed=18 + i, with_field=False))
    return meshes


def open_loop(ctxs, sizes, rate, nreq, seed, workers=64):
    """Poisson arrivals at `rate` requests/s; each request asks one uniform
    mesh for one uniform cluster and a mask uniform over the 15 non-empty
    subsets of VT, VV, ET, TT.  Latency runs from the scheduled arrival to the
    view being ready (queueing included).  rate = None: closed loop, every
    request at time zero (capacity).  The dispatch runs in native threads
    (consumers.open_loop) so that the driver is not the bottleneck."""
    import consumers
    rng = np.random.default_rng(seed)
    mi = rng.integers(len(ctxs), size=nreq).astype(np.int32)
    ks = np.array([rng.integers(ctxs[m].K) for m in mi], dtype=np.int32)
    masks = rng.integers(1, 16, size=nreq).astype(np.uint32)
    st0 = [(x.builds, x.hits) for x in (c.serve_stats() for c in ctxs)]
    lat, wall, fails, first = consumers.open_loop(ctxs, mi, ks, masks, rate, seed=seed + 1000, workers=workers)
    tets = int(sum(sizes[m][k] for m, k in zip(mi, ks)))
    st1 = [(x.builds, x.hits) for x in (c.serve_stats() for c in ctxs)]
    return {"requests": nreq, "failures": fails,
            "first_failure": None if first < 0 else f"mesh {int(mi[first])} cluster {int(ks[first])} "
                                                      f"mask {int(masks[first])}",
            "wall_s": wall, "req_per_s": nreq / wall, "tets_per_s": tets / wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "builds": int(sum(b[0] - a[0] for a, b in zip(st0, st1))),
            "hits": int(sum(b[1] - a[1] for a, b in zip(st0, st1)))}


def mixed_leg(args, gale):
    """24 meshes loaded at once, Poisson-arriving requests for random masks at
    0.25, 0.5 and 0.9 of the measured capacity of the device-loop form,
    admitted against one budget split across the meshes in proportion to
    their tet counts; the same arrivals then meet one kernel launch per
    request."""
    meshes = mixed_meshes(args.mixed_scale)
    budget = int(args.mixed_budget_gb * (1 << 30))
    nreq = args.mixed_requests

    def load_all(mode):
        # the budget is split in proportion to tet counts (relation bytes per
        # tet are nearly the same across these meshes)
        tot = sum(m.nt for m in meshes)
        ctxs = [gale.Context.load(m, device=0, cache_budget_bytes=max(1 << 20, budget * m.nt // tot)) for m in meshes]
        # every mesh's loop resident at once, even at one CTA per SM
        loop_ctas = max(1, torch_sm_count() // len(ctxs))
        for c in ctxs:
            c.serve_configure(mode, loop_ctas=loop_ctas if mode == gale.SERVE_LOOP else 0)
        sizes = []
        for c in ctxs:
            _, I_T, _ = c.intervals()
            sizes.append(np.diff(I_T))
        return ctxs, sizes, loop_ctas

    out = {"workload": f"{len(meshes)} meshes (Freudenthal 32^3..192^3 kd<=512, Delaunay 100k..1M points "
                       f"uneven kd) x scale {args.mixed_scale:g}, Poisson arrivals, masks uniform over 15 "
                       f"subsets, {args.mixed_budget_gb:g} GB budget split by tet counts",
           "tets": int(sum(m.nt for m in meshes)), "clusters": int(sum(m.nclusters for m in meshes)),
           "requests_per_phase": nreq,
           "phases": "warm-up (seed 1), closed-loop capacity (seed 2), then Poisson arrivals at 0.25, 0.5 and "
                     "0.9 of the device loop's capacity (seeds 11, 12, 13); both forms see the same requests "
                     "from a cold cache"}
    fracs = (0.25, 0.5, 0.9)
    rates = None
    for mode, key in ((gale.SERVE_LOOP, "device_loop"), (gale.SERVE_SINGLE, "per_request_launch")):
        ctxs, sizes, loop_ctas = load_all(mode)
        res = {"loop_ctas_per_mesh": loop_ctas if mode == gale.SERVE_LOOP else None}
        open_loop(ctxs, sizes, None, min(nreq, 1000), seed=1)
        res["capacity"] = open_loop(ctxs, sizes, None, nreq, seed=2)
        if rates is None:
            rates = [f * res["capacity"]["req_per_s"] for f in fracs]
            out["rates_req_per_s"] = rates
        for j, (f, r) in enumerate(zip(fracs, rates)):
            res[f"at_{f:g}"] = open_loop(ctxs, sizes, r, nreq, seed=11 + j)
        res["evictions"] = int(sum(c.serve_stats().evictions for c in ctxs))
        out[key] = res
        for c in ctxs:
            c.close()
    return out


def torch_sm_count() -> int:
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def coboundary_leg(args, gale, gen):
    """VE, VF, EF, FT (gale_build_coboundary) on a grid of the same recipe,
    in sorted enumeration ids: device time of the whole pass (count, scan,
    fill and row-sort kernels over the enumeration and the tet rows), output
    bytes over that time against the HBM copy peak, and the oracle timed on a
    12^3 sample."""
    import torch
    n = args.coboundary_grid
    mesh = gen.freudenthal_mesh(n, 512, seed=3, field_seed=4, jitter=0.3, with_field=False)
    with gale.Context.load(mesh, device=0) as c:
        t0 = time.perf_counter()
        c.enumerate(gale.ENUM_SORTED)
        enum_s = time.perf_counter() - t0
        cb = gale.Coboundary()
        lib = c._lib
        stream = torch.cuda.ExternalStream(c.stream_handle)
        gale._check(lib.gale_build_coboundary(c._h, 15, ctypes.byref(cb)))  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 3
        a.record(stream)
        for _ in range(steps):
            gale._check(lib.gale_build_coboundary(c._h, 15, ctypes.byref(cb)))
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out_bytes = int(sum(4 * (cb.rows[i] + 1 + cb.len[i]) for i in range(4)))
        # what the pass must read: the enumeration's lists and the tet rows
        in_bytes = 4 * (2 * int(cb.rows[2]) + 3 * int(cb.rows[3]) + 4 * mesh.nt)
    peak, _ = load_peaks()
    # the oracle on a small sample of the same recipe
    import oracle
    small = gen.freudenthal_mesh(12, 512, seed=3, field_seed=4, jitter=0.3, with_field=False)
    t0 = time.perf_counter()
    canon = oracle.canonicalize(small.nv, small.tv, small.seg, small.nclusters)
    oracle.coboundary(canon, oracle.enumerate_simplices(canon, "sorted"))
    osec = time.perf_counter() - t0
    return {"workload": f"grid{n}^3-jitter0.3-kd512: {mesh.nt} tets; VE+VF+EF+FT in sorted enumeration ids",
            "ms": ms, "tets_per_s": mesh.nt / (ms / 1e3), "host_enumeration_s": enum_s,
            "roofline": {"bound": "hbm", "achieved": out_bytes / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": out_bytes / (ms / 1e3) / 1e9 / peak,
                         "algorithmic_bytes": out_bytes, "note": "output bytes only",
                         "frac_reads_and_writes": (out_bytes + in_bytes) / (ms / 1e3) / 1e9 / peak,
                         "read_bytes": in_bytes},
            "oracle": {"sample": f"grid12^3 ({small.nt} tets), enumeration + coboundary, Python, single thread",
                       "tets_per_s": small.nt / osec}}


def gradient_leg(args, gale, gen):
    """The discrete gradient of a Gaussian-mixture field on a grid of the
    same recipe (Section 5.1, DiscreteGradient): wall time of each step -
    the enumeration with its lists fetched into host arrays, VE + VF on the
    GPU and their copy to the host, the VT build and export with the TV
    rows, and the consumer threads
    (which answer FE / TF themselves) - and the oracle on an 8^3 sample."""
    import torch
    import consumers
    n = args.dg_grid
    threads = args.dg_threads or os.cpu_count() or 1
    mesh = gen.freudenthal_mesh(n, 512, seed=3, field_seed=4, jitter=0.3, ngauss=16)
    out = {"workload": f"grid{n}^3-jitter0.3-kd512 + 16-Gaussian field: {mesh.nv} vertices, {mesh.nt} tets",
           "threads": threads}
    with gale.Context.load(mesh, device=0) as c:
        vp, _ = c.permutations()
        f_c, inid = consumers.canonical_inputs(mesh.field, vp)
        consumers._load()  # builds / loads the consumer library outside the timed steps
        t = {}
        t0 = time.perf_counter()
        en = c.enumerate(gale.ENUM_SORTED)
        t["enumeration_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        cb = c.coboundary(gale.CB_VE | gale.CB_VF)
        torch.cuda.synchronize()
        t["ve_vf_gpu_and_copy_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        I_V, _, _ = c.intervals()
        c.build(None, gale.VT, gale.MODE_BATCHED)
        c.synchronize()
        b = c.export(gale.VT)
        vt = consumers.csr_from_bulk(b["vt_off"], b["vt_val"], I_V)
        rows = c.rows()
        t["vt_export_s"] = time.perf_counter() - t0
        g, wall = consumers.discrete_gradient_arrays(f_c, inid, cb["VE"], cb["VF"], vt, en["E"], en["F"], rows,
                                                     nthreads=threads)
        t["consumer_s"] = wall
    crit = [int((g["v_up"] < 0).sum()), int(((g["e_down"] < 0) & (g["e_up"] < 0)).sum()),
            int(((g["f_down"] < 0) & (g["f_up"] < 0)).sum()), int((g["t_down"] < 0).sum())]
    out.update(t)
    out["total_s"] = sum(t.values())
    out["consumer_vertices_per_s"] = mesh.nv / t["consumer_s"]
    out["critical_cells"] = crit
    out["euler"] = crit[0] - crit[1] + crit[2] - crit[3]
    import oracle
    small = gen.freudenthal_mesh(8, 512, seed=3, field_seed=4, jitter=0.3, ngauss=16)
    canon = oracle.canonicalize(small.nv, small.tv, small.seg, small.nclusters)
    vp = np.asarray(canon["vperm"])
    t0 = time.perf_counter()
    oracle.lower_star_gradient(canon, np.asarray(small.field, np.float32)[vp].astype(np.float64), vp)
    osec = time.perf_counter() - t0
    out["oracle"] = {"sample": f"grid8^3 ({small.nv} vertices), Python, single thread",
                     "vertices_per_s": small.nv / osec}
    return out


def gale_kernel_sha() -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2507_15230_gb300", "csrc", "gale_kernels.cu"), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


if __name__ == "__main__":
    main()
