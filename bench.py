#!/usr/bin/env python
"""Throughput of the spherical-harmonics hot path on GB300.

Step = one forward pass (values + Cartesian gradients, FP32, l_max = 8) over
N = 4,194,304 synthetic points (directions uniform on the sphere, radii
~ U[0.5, 5.0]), written as sph [N, 81] and dsph [N, 3, 81]: 5.49 GB of output
per step. Metric: points/s, with the dominant kernel's achieved HBM bandwidth
against the measured copy bandwidth.

Also reported (separate keys): the fused recompute-backward against the
materialise-then-contract backward (N = 4,194,304 edge vectors, |r| ~ U[0.7, 6],
l_max = 6, upstream g ~ N(0,1)) with their mutual difference (both are checked
against the FP64 oracle by the test suite); the double backward; the
end-to-end throughput from pinned host memory; and the FP64 oracle timed on
the host cores (the only legs that run the oracle are the CPU baseline and
--impl reference).

Multi-GPU: one process per GPU (torchrun); each rank evaluates its own N
points (weak scaling, no collective on the data path); timing is the max
over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "points/s, Y_lm + grad FP32 l_max=8 (forward values+Cartesian gradients)"
N_POINTS = 4_194_304
L_MAX = 8
BWD_N = 4_194_304
BWD_L = 6
FLUSH_BYTES = 256 << 20  # > 129 MB L2


# ---------------------------------------------------------------- CPU (oracle)
def _oracle_chunk(args):
    n, seed, l_max = args
    import numpy as np

    import oracle
    from paper_2302_08381_gb300 import inputs

    xyz = inputs.shell_points(n, 0.5, 5.0, seed=seed).astype(np.float64)
    v, g = oracle.spherical_harmonics_grad(xyz, l_max, False)
    return float(v.sum() + g.sum())


class OraclePool:
    """A spawn pool over all host cores running the FP64 oracle on chunks of
    the benchmark distribution (values + gradients); workers return checksums
    only, so nothing large crosses process boundaries."""

    def __init__(self, l_max: int):
        import multiprocessing as mp

        self.l_max = l_max
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_chunk, [(256, 1, l_max)] * self.cores)  # import + warm every worker

    def run(self, total_points: int, chunk: int = 16384, seed0: int = 1000):
        nchunks = max(1, total_points // chunk)
        work = [(chunk, seed0 + i, self.l_max) for i in range(nchunks)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_chunk, work, chunksize=1)
        dt = time.perf_counter() - t0
        return nchunks * chunk / dt, nchunks * chunk, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_subset(kind: str):
    """One 10,000-point subset through the FP64 oracle in this process;
    returns seconds."""
    import numpy as np

    import oracle
    from paper_2302_08381_gb300 import inputs

    if kind == "l8":  # the benchmark distribution, values + gradients
        xyz = inputs.shell_points(10_000, 0.5, 5.0, seed=3).astype(np.float64)
        t0 = time.perf_counter()
        oracle.spherical_harmonics_grad(xyz, 8, False)
    elif kind == "l50":  # half uniform on the sphere, half within 1e-4 rad of the poles, normalized
        xyz = inputs.pole_mix_points(10_000, seed=4)
        t0 = time.perf_counter()
        oracle.spherical_harmonics_grad(xyz, 50, True)
    else:  # ragged sets: 2,500 points at each l_max of {3, 6, 8, 12}
        sets = [(inputs.normal_points(2_500, seed=10 + i), L) for i, L in enumerate((3, 6, 8, 12))]
        t0 = time.perf_counter()
        for xyz, L in sets:
            oracle.spherical_harmonics_grad(xyz, L, False)
    return time.perf_counter() - t0


def time_oracle_single_thread():
    """ns per point of the FP64 oracle on one host core (a spawned
    one-process pool) for 10,000-point subsets: l_max 8 values + gradients
    (the benchmark), l_max 50 normalized at the pole mix, and the ragged
    l_max mix {3, 6, 8, 12}."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(1) as pool:
        pool.map(_oracle_subset, ["batch"])  # import + warm the worker
        secs = pool.map(_oracle_subset, ["l8", "l50", "batch"], chunksize=1)
    return {
        "cores": 1,
        "l8_values_gradients_ns_per_point": secs[0] * 1e9 / 10_000,
        "l50_normalized_pole_mix_ns_per_point": secs[1] * 1e9 / 10_000,
        "ragged_lmax_3_6_8_12_ns_per_point": secs[2] * 1e9 / 10_000,
        "sample": "10,000 points each, FP64 oracle, one spawned process",
    }


def time_oracle(total_points: int, l_max: int, chunk: int = 16384):
    """Times the FP64 oracle over total_points on all host cores.
    Returns (points/s, cores, seconds)."""
    op = OraclePool(l_max)
    try:
        vps, _, dt = op.run(total_points, chunk)
    finally:
        op.close()
    return vps, op.cores, dt


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""

    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)],
                stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL,
                text=True,
            )
            self.t0 = time.time()
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(
                    {
                        "sm": float(parts[1]),
                        "max": float(parts[2]),
                        "power": float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else None,
                        "hw_slowdown": parts[5] == "Active",
                        "hw_thermal_slowdown": parts[6] == "Active",
                        "sw_thermal_slowdown": parts[7] == "Active",
                        "sw_power_cap": parts[8] == "Active",
                    }
                )
            except ValueError:
                continue
        if not rows:
            return None
        loaded = [r for r in rows if r["power"] is None or r["power"] > 300] or rows
        reasons = sorted(
            {k for r in loaded for k in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap") if r[k]}
        )
        return {
            "sm_mhz": statistics.median(r["sm"] for r in loaded),
            "sm_max_mhz": max(r["max"] for r in rows),
            "reasons": reasons,
            "samples": len(rows),
            "samples_under_load": len(loaded),
        }


def physical_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(kernel_tag: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    ent = rec.get(kernel_tag)
    if not ent:
        return None
    # hash of the files that define the kernel (listed in the record)
    h = hashlib.sha256()
    for rel in ent.get("source_files", []):
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return None
        with open(path, "rb") as f:
            h.update(rel.encode() + f.read())
    if not ent.get("source_files") or ent.get("sources_sha256") != h.hexdigest():
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    sample = 131_072
    op = OraclePool(L_MAX)
    cores = op.cores
    times = []
    try:
        for i in range(args.warmup + args.steps):
            _, pts, dt = op.run(sample, seed0=1000 + 97 * i)
            if i >= args.warmup:
                times.append(dt)
    finally:
        op.close()
    step = statistics.median(times)
    value = sample / step
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "forward values+gradients l_max=8, FP64 oracle on a sample", "points_per_step": sample},
        "cpu_baseline": {
            "value": value,
            "unit": "points/s",
            "cores": cores,
            "kind": "oracle",
            "sample": f"{sample} points per step of the benchmark distribution, spawn pool of {cores} processes",
        },
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ranks
def launch_ranks(nproc: int) -> int:
    """Runs this script with the same arguments as `nproc` ranks on this node
    (torch.distributed.run, rendezvous on 127.0.0.1); returns their exit code."""
    import socket

    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr=127.0.0.1", f"--master-port={port}", "--", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def rank_shard(n: int, rank: int, world: int):
    """Weak scaling: the global cloud holds world * n points and rank r owns
    the contiguous range shard.point_range gives it (n points each)."""
    from paper_2302_08381_gb300 import shard

    return shard.point_range(world * n, rank, world)


def run_dry(args, rank, world):
    """The multi-rank logic without a GPU: shard ranges, a gloo barrier around
    stand-in timed steps, and the max over ranks, as the GPU arm does it."""
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("gloo")
    start, end = rank_shard(args.n, rank, world)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        time.sleep(0.001 * (1 + rank))  # stand-in step; rank-dependent so the max is visible
    step_ms = (time.perf_counter() - t0) * 1e3 / max(args.steps, 1)
    if world > 1:
        dist.barrier()
    t = torch.tensor([step_ms], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ranges = [None] * world
        dist.all_gather_object(ranges, (start, end))
    else:
        ranges = [(start, end)]
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step_max": float(t.item()), "value": world * args.n / (float(t.item()) * 1e-3),
                          "unit": "points/s (stand-in steps)", "scaling": "weak", "shards": ranges}), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the library's default launch shape")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / backward / oracle legs")
    ap.add_argument(
        "--profile",
        choices=["fwd", "fwd64", "bwd", "dbwd", "batch", "batched", "expansion", "slice20", "degree20", "row20",
                 "hess", "degree50_f64"],
        help="launch only this kernel family warmup+steps times (for ncu), print a short line",
    )
    ap.add_argument("--lmax", type=int, default=0, help="with --profile: l_max of the captured launches (0: the mode's own)")
    ap.add_argument("--dry-run", action="store_true",
                    help="host-only run of the multi-rank logic (gloo, no GPU): sharding, barrier, max over ranks")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: relaunch this script under torch.distributed.run
        sys.exit(launch_ranks(args.gpus))

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and rank == 0:
        print(f"bench.py: WORLD_SIZE={world} differs from --gpus {args.gpus}; running {world} rank(s)",
              file=sys.stderr, flush=True)
    if args.dry_run:
        run_dry(args, rank, world)
        return

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile:
        run_profile(args)
        return

    # CPU baseline first: the spawn pool is created before any CUDA call.
    cpu = None
    cpu_single = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.no_extras:
        sample = 1_048_576
        vps, cores, dt = time_oracle(sample, L_MAX)
        cpu_single = time_oracle_single_thread()
        cpu = {
            "value": vps,
            "unit": "points/s",
            "cores": cores,
            "kind": "oracle",
            "sample": f"{sample} points of the benchmark distribution, l_max=8 values+gradients, FP64, "
            f"spawn pool of {cores} processes ({dt:.1f} s)",
        }

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2302_08381_gb300 import _capi, api, inputs
    from paper_2302_08381_gb300 import build as _build

    if not os.path.exists(_capi.LIB_PATH):
        _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    n, L = args.n, L_MAX
    K = (L + 1) ** 2
    shard_start, shard_end = rank_shard(n, rank, world)
    xyz_np = inputs.shell_points(n, 0.5, 5.0, seed=8 + rank)
    xyz = torch.from_numpy(xyz_np).to(dev)
    sph = torch.empty((n, K), device=dev)
    dsph = torch.empty((n, 3, K), device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # The library's autotuner picks the launch shape for this workload
    # (outside the timed region); the timed steps use the installed shape.
    tuned, tuned_ms = None, None
    if not args.no_autotune:
        tuned, tuned_ms = _capi.sphericart_autotune(
            xyz.data_ptr(), n, L, 0, _capi.SPH_F32, _capi.SPH_OUT_SAME, sph.data_ptr(), dsph.data_ptr(),
            stream.cuda_stream, 3,
        )

    def step():
        api.spherical_harmonics(xyz, L, False, gradients=True, out=(sph, dsph))

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(physical_gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed launches (outside the events)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    # Keep the GPU under the same load a little longer for clock samples.
    t_extra = time.perf_counter()
    while time.perf_counter() - t_extra < 1.0:
        for _ in range(20):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    clocks = sampler.stop()

    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    kernel_ms = sum(per) / len(per)
    t_max = torch.tensor([kernel_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms = float(t_max.item())
    value = world * n / (ms * 1e-3)

    bytes_per_launch = n * (3 * 4 + K * 4 * 4)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (ms * 1e-3) / 1e9
    roof = {
        "bound": "hbm",
        "achieved": achieved,
        "peak": peak,
        "unit": "GB/s",
        "frac": achieved / peak,
        "traffic": recorded_traffic("point_fwd_L8_grad_f32"),
        "kernel": "point_fwd_kernel<8, GRAD, scaled, f32>",
        "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
        "algorithmic_bytes_per_launch": bytes_per_launch,
        "frac_of_8TBs": achieved / 8000.0,
    }

    extras = {}
    if not args.no_extras:
        # every rank runs the end-to-end leg on its own GPU; the slowest counts
        e2e_s = run_e2e(torch, api, inputs, dev, n, L, K, seed=8 + rank)
        t_e2e = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
        e2e_s = float(t_e2e.item())
        extras["e2e"] = {
            "value": world * n / e2e_s,
            "unit": "points/s",
            "h2d_bytes_per_step": world * n * 12,
            "d2h_bytes_per_step": world * n * K * 16,
            "ms_per_step": e2e_s * 1e3,
            "path": "sphericart_compute_host: 512Ki-point chunks, H2D / kernel / D2H overlapped on 3 streams; "
            "bound by the device-to-host link (193.6 GB/s measured on this machine)",
        }
        if rank == 0 and world == 1:
            extras.update(run_extras(torch, np, api, inputs, dev, stream, n, L, K, sph, dsph, flush))

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "points/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": f"forward values+gradients, l_max={L}, N={n} per GPU, FP32, scaled (r^l Y), "
                "directions uniform, r~U[0.5,5]",
                "n_points_per_gpu": n,
                "l_max": L,
                "outputs": f"sph [N,{K}] + dsph [N,3,{K}] FP32",
                "l2": "flushed between timed launches (256 MB zero fill outside the timed events)",
                "parallelism": f"points sharded, {world} independent rank(s); rank 0 owns points "
                f"[{shard_start}, {shard_end}) of {world * n} (contiguous ranges, no collective on the data path)",
                "launch_shape": (
                    {"points_per_tile": tuned.points_per_tile, "warps_per_block": tuned.warps_per_block,
                     "blocks_per_sm": tuned.blocks_per_sm, "source": "sphericart_autotune"}
                    if tuned is not None else "library default"
                ),
            },
            "roofline": roof,
            "clocks": clocks,
            "gpu_launches": args.steps,
            "wall_s_timed_region": wall,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if cpu_single:
            line["oracle_single_thread"] = cpu_single
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_profile(args):
    """Minimal launches of one kernel family for profiler captures."""
    import numpy as np
    import torch

    from paper_2302_08381_gb300 import _capi, api, inputs
    from paper_2302_08381_gb300 import build as _build

    if not os.path.exists(_capi.LIB_PATH):
        _build.build()
    dev = torch.device("cuda", 0)
    n = args.n
    if args.profile in ("fwd", "fwd64", "batch", "batched", "hess"):
        L = L_MAX
    elif args.profile in ("slice20", "degree20", "row20"):
        L = 20
    elif args.profile == "degree50_f64":
        L = 50
    else:
        L = BWD_L  # backward kernels and the expansion: l_max = 6
    if args.lmax > 0 and args.profile not in ("batch", "batched"):
        L = args.lmax
    K = (L + 1) ** 2
    x = torch.from_numpy(inputs.shell_points(n, 0.5, 5.0, seed=8)).to(dev)
    if args.profile == "fwd":
        sph = torch.empty((n, K), device=dev)
        dsph = torch.empty((n, 3, K), device=dev)
        fn = lambda: api.spherical_harmonics(x, L, False, gradients=True, out=(sph, dsph))  # noqa: E731
    elif args.profile == "degree50_f64":
        x64d = x.double()
        fn = lambda: api.spherical_harmonics(x64d, L, True, gradients=True)  # noqa: E731  (AUTO: DEGREE)
    elif args.profile == "fwd64":
        x64 = x.double()
        fn = lambda: api.spherical_harmonics(x64, L, False, gradients=True)  # noqa: E731
    elif args.profile == "slice20":
        fn = lambda: api.spherical_harmonics(x, L, True, gradients=True, kernel="slice")  # noqa: E731
    elif args.profile == "degree20":
        fn = lambda: api.spherical_harmonics(x, L, True, gradients=True, kernel="degree")  # noqa: E731
    elif args.profile == "row20":
        fn = lambda: api.spherical_harmonics(x, L, True, gradients=True, kernel="row")  # noqa: E731
    elif args.profile == "hess":
        fn = lambda: api.spherical_harmonics(x, L, gradients=True, hessians=True)  # noqa: E731
    elif args.profile in ("bwd", "dbwd"):
        g = torch.from_numpy(inputs.upstream(n, K, seed=33)).to(dev)
        v = torch.from_numpy(inputs.upstream(n, 3, seed=34)).to(dev)
        dx = torch.empty_like(x)
        if args.profile == "bwd":
            fn = lambda: api.backward(x, g, L, out=dx)  # noqa: E731
        else:
            fn = lambda: api.double_backward(x, g, v, L)  # noqa: E731
    elif args.profile == "expansion":
        nr, ncent = 8, max(1, n // 40)
        counts = np.full(ncent, n // ncent, dtype=np.int64)
        offs = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)).to(dev)
        E = int(counts.sum())
        R = torch.from_numpy(inputs.upstream(E, nr * (L + 1), seed=612)).to(dev).view(E, nr, L + 1)
        xe = x[:E].contiguous()
        c = torch.empty((ncent, nr, K), device=dev)
        fn = lambda: api.expansion(xe, R, offs, L, out=c)  # noqa: E731
    else:
        sizes, lmax, xyz = inputs.ragged_sets(512, [3, 6, 8, 12], 1000, 200_000, seed=5)
        scale = n / float(sizes.sum())
        sizes = np.maximum(1, (sizes * scale).astype(np.int64))
        offs = np.concatenate([[0], np.cumsum(sizes)])
        xt = torch.from_numpy(xyz[: offs[-1]]).to(dev)
        xs = [xt[offs[i]:offs[i + 1]] for i in range(len(sizes))]
        ls = [int(v) for v in lmax]
        if args.profile == "batch":  # the plan: one launch per l_max class
            plan = api.BatchPlan(xs, ls)
            fn = plan.execute
        else:  # sphericart_compute_batched: one launch
            outs = [(torch.empty((x.shape[0], (L + 1) ** 2), device=dev),
                     torch.empty((x.shape[0], 3, (L + 1) ** 2), device=dev)) for x, L in zip(xs, ls)]
            fn = lambda: api.compute_batched(xs, ls, outputs=outs)  # noqa: E731
    for _ in range(args.warmup + args.steps):
        fn()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n": n, "launches": args.warmup + args.steps}), flush=True)


def _events_ms(torch, stream, fn, reps, flush=None):
    times = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    return statistics.median(times)


def run_batch_leg(torch, np, api, inputs, dev, stream, flush):
    """512 ragged sets (sizes log-uniform in [1e3, 2e5], l_max from {3,6,8,12},
    N(0,1) FP32 points), values + gradients: the plan's persistent launches
    (one per l_max class, and one for all sets), sphericart_compute_batched on
    a device descriptor array (one launch), each eager and replayed from a
    CUDA graph, vs one launch per set (eager and captured in one graph)."""
    sizes, lmax, xyz = inputs.ragged_sets(512, [3, 6, 8, 12], 1000, 200_000, seed=5)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xt = torch.from_numpy(xyz).to(dev)
    xs = [xt[offs[i]:offs[i + 1]] for i in range(len(sizes))]
    ls = [int(v) for v in lmax]
    plan = api.BatchPlan(xs, ls)
    outs = list(zip(plan.sph, plan.dsph))
    # the batch autotuner picks the per-warp budget, warps per block and CTAs per SM
    import ctypes

    from paper_2302_08381_gb300 import _capi as C

    arr = (C.sph_batch_set * len(xs))()
    for i, (x, L) in enumerate(zip(xs, ls)):
        arr[i] = C.sph_batch_set(x.data_ptr(), plan.sph[i].data_ptr(), plan.dsph[i].data_ptr(), x.shape[0], L, 0)
    best = C.sph_launch()
    best_ms = ctypes.c_float()
    C.check("sphericart_batch_autotune", C.lib().sphericart_batch_autotune(
        arr, len(xs), stream.cuda_stream, 2, ctypes.byref(best), ctypes.byref(best_ms)))
    plan.close()
    plan = api.BatchPlan(xs, ls, launch=best, outputs=outs)  # one persistent launch per l_max class
    one = api.BatchPlan(xs, ls, outputs=outs, mode="one_launch")
    # the device-descriptor entry point: one launch over every set
    desc = api.batch_descriptors(xs, ls, [o[0] for o in outs], [o[1] for o in outs])

    def batched():
        C.check("sphericart_compute_batched", C.lib().sphericart_compute_batched(
            desc.data_ptr(), len(xs), C.SPH_BATCHED_GRADIENTS, stream.cuda_stream))

    def per_set():
        for x, L, o in zip(xs, ls, outs):
            api.spherical_harmonics(x, L, gradients=True, out=o)

    plan.execute()
    one.execute()
    batched()
    per_set()
    torch.cuda.synchronize()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    g_plan = torch.cuda.CUDAGraph()
    g_one = torch.cuda.CUDAGraph()
    g_batched = torch.cuda.CUDAGraph()
    g_sets = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g_plan, stream=side):
            plan.execute()
        with torch.cuda.graph(g_one, stream=side):
            one.execute()
        with torch.cuda.graph(g_batched, stream=side):
            C.check("sphericart_compute_batched", C.lib().sphericart_compute_batched(
                desc.data_ptr(), len(xs), C.SPH_BATCHED_GRADIENTS, side.cuda_stream))
        with torch.cuda.graph(g_sets, stream=side):
            per_set()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    total = int(sizes.sum())
    nbytes = int(sum(s * (12 + 16 * (l + 1) ** 2) for s, l in zip(sizes, lmax)))
    res = {
        "workload": f"512 sets, {total} points, l_max from {{3,6,8,12}}, values+gradients FP32",
        "tuned_shape": {"budget_rows": best.points_per_tile, "warps_per_block": best.warps_per_block,
                        "blocks_per_sm": best.blocks_per_sm},
        "points": total,
        "algorithmic_bytes": nbytes,
    }
    for name, fn in (
        ("persistent_per_lmax", plan.execute),
        ("persistent_per_lmax_graph", g_plan.replay),
        ("persistent_one_launch", one.execute),
        ("persistent_one_launch_graph", g_one.replay),
        ("compute_batched_device_desc", batched),
        ("compute_batched_device_desc_graph", g_batched.replay),
        ("per_set_launches", per_set),
        ("per_set_graph", g_sets.replay),
    ):
        for _ in range(2):
            fn()
        ms = _events_ms(torch, stream, fn, 7, flush)
        res[name + "_ms"] = ms
        res[name + "_points_per_s"] = total / (ms * 1e-3)
        res[name + "_GBs"] = nbytes / (ms * 1e-3) / 1e9
    plan.close()
    one.close()
    return res


def run_variants_leg(torch, api, inputs, dev, stream, flush):
    """Forward variants, each timed alone (median of 10 launches, L2 flushed)."""
    res = {}
    for n, L, label, kw, elem, ddims in (
        (4_194_304, 8, "l8_values_only_f32", dict(), 4, 1),
        (4_194_304, 8, "l8_grad_f32_normalized", dict(normalized=True, gradients=True), 4, 4),
        (4_194_304, 8, "l8_grad_bf16_store", dict(gradients=True, out_dtype=torch.bfloat16), 2, 4),
        (4_194_304, 8, "l8_grad_f64", dict(gradients=True), 8, 4),
        (1_048_576, 8, "l8_grad_hess_f32", dict(gradients=True, hessians=True), 4, 13),
        (1_048_576, 8, "l8_grad_hess_f32_slice", dict(gradients=True, hessians=True, kernel="slice"), 4, 13),
        # FP32 Hessians: AUTO runs 10 lanes per point (one per distinct plane)
        # at scaled l_max 7..16 and normalized 6..13, ROW above; the one-lane
        # tile, the 16-lane map and ROW beside it
        (1_048_576, 8, "l8_grad_hess_f32_one_lane",
         dict(gradients=True, hessians=True, kernel="point", launch=(12, 2, 16, 1)), 4, 13),
        (1_048_576, 8, "l8_grad_hess_f32_sixteen_lanes",
         dict(gradients=True, hessians=True, kernel="point", launch=(4, 0, 0, 16)), 4, 13),
        (400_000, 10, "l10_grad_hess_f32_norm_n400k", dict(gradients=True, hessians=True, normalized=True), 4, 13),
        (400_000, 10, "l10_grad_hess_f32_norm_n400k_sixteen_lanes",
         dict(gradients=True, hessians=True, normalized=True, kernel="point", launch=(4, 0, 0, 16)), 4, 13),
        (400_000, 12, "l12_grad_hess_f32_norm_n400k", dict(gradients=True, hessians=True, normalized=True), 4, 13),
        (100_000, 20, "l20_grad_hess_f32_norm_n100k", dict(gradients=True, hessians=True, normalized=True), 4, 13),
        (400_000, 12, "l12_grad_hess_f32_norm_n400k_one_lane",
         dict(gradients=True, hessians=True, normalized=True, kernel="point", launch=(4, 1, 0, 1)), 4, 13),
        (400_000, 12, "l12_grad_hess_f32_norm_n400k_row",
         dict(gradients=True, hessians=True, normalized=True, kernel="row"), 4, 13),
        (200_000, 15, "l15_grad_hess_f32_n200k", dict(gradients=True, hessians=True), 4, 13),
        (200_000, 15, "l15_grad_hess_f32_n200k_row", dict(gradients=True, hessians=True, kernel="row"), 4, 13),
        (200_000, 16, "l16_grad_hess_f32_n200k", dict(gradients=True, hessians=True), 4, 13),
        (200_000, 16, "l16_grad_hess_f32_n200k_row", dict(gradients=True, hessians=True, kernel="row"), 4, 13),
        (200_000, 13, "l13_grad_hess_f32_norm_n200k", dict(gradients=True, hessians=True, normalized=True), 4, 13),
        (200_000, 13, "l13_grad_hess_f32_norm_n200k_row",
         dict(gradients=True, hessians=True, normalized=True, kernel="row"), 4, 13),
        (200_000, 14, "l14_grad_hess_f32_norm_n200k", dict(gradients=True, hessians=True, normalized=True), 4, 13),
        (200_000, 14, "l14_grad_hess_f32_norm_n200k_ten_lanes",
         dict(gradients=True, hessians=True, normalized=True, kernel="point", launch=(3, 0, 0, 10)), 4, 13),
        (1_000_000, 10, "l10_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 10, "l10_grad_bf16_n1M", dict(gradients=True, out_dtype=torch.bfloat16), 2, 4),
        # l_max 12..16 (AUTO: 4 lanes per point, one per output plane) against
        # the best one-lane-per-point shapes measured on this GPU
        (1_000_000, 12, "l12_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 12, "l12_grad_f32_n1M_one_lane", dict(gradients=True, kernel="point", launch=(16, 1, 0, 1)), 4, 4),
        (1_000_000, 13, "l13_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 14, "l14_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 15, "l15_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 16, "l16_grad_f32_n1M", dict(gradients=True), 4, 4),
        (1_000_000, 16, "l16_grad_f32_n1M_one_lane", dict(gradients=True, kernel="point", launch=(8, 2, 0, 1)), 4, 4),
        (1_000_000, 16, "l16_grad_bf16_n1M", dict(gradients=True, out_dtype=torch.bfloat16), 2, 4),
        # the paper's GPU table sizes (10k / 100k points, l_max = 8)
        (10_000, 8, "l8_values_f64_n10k", dict(), 8, 1),
        (10_000, 8, "l8_values_f64_n10k_normalized", dict(normalized=True), 8, 1),
        (10_000, 8, "l8_grad_f32_n10k", dict(gradients=True), 4, 4),
        (100_000, 8, "l8_values_f32_n100k", dict(), 4, 1),
        (100_000, 8, "l8_grad_f32_n100k", dict(gradients=True), 4, 4),
        (100_000, 8, "l8_grad_f64_n100k", dict(gradients=True), 8, 4),
        # the high-degree precision-sweep sizes, normalized (AUTO: ROW for FP32
        # arithmetic, DEGREE for FP64 arithmetic), and the other families
        (200_000, 20, "l20_grad_f32_norm_n200k", dict(gradients=True, normalized=True), 4, 4),
        (200_000, 30, "l30_grad_f32_norm_n200k", dict(gradients=True, normalized=True), 4, 4),
        (200_000, 50, "l50_grad_f32_norm_n200k", dict(gradients=True, normalized=True), 4, 4),
        (200_000, 63, "l63_grad_f32_norm_n200k", dict(gradients=True, normalized=True), 4, 4),
        (200_000, 20, "l20_grad_f32_norm_n200k_slice", dict(gradients=True, normalized=True, kernel="slice"), 4, 4),
        (200_000, 50, "l50_grad_f32_norm_n200k_slice", dict(gradients=True, normalized=True, kernel="slice"), 4, 4),
        (200_000, 20, "l20_grad_f32_norm_n200k_degree", dict(gradients=True, normalized=True, kernel="degree"), 4, 4),
        (200_000, 20, "l20_grad_bf16_norm_n200k", dict(gradients=True, normalized=True, out_dtype=torch.bfloat16), 2, 4),
        (1_000_000, 20, "l20_grad_f32_n1M", dict(gradients=True), 4, 4),
        (200_000, 50, "l50_grad_mixed_norm_n200k", dict(gradients=True, normalized=True, qprec="f64"), 4, 4),
        (200_000, 50, "l50_grad_f64_norm_n200k", dict(gradients=True, normalized=True), 8, 4),
        (200_000, 50, "l50_grad_f64_norm_n200k_slice", dict(gradients=True, normalized=True, kernel="slice"), 8, 4),
        (200_000, 50, "l50_grad_f64_norm_n200k_degree_down",
         dict(gradients=True, normalized=True, kernel="degree_down"), 8, 4),
        (1_000_000, 16, "l16_grad_f64_n1M", dict(gradients=True), 8, 4),
        # FP64 with gradients from l_max 9: AUTO runs DEGREE (2 lanes per point)
        (1_000_000, 10, "l10_grad_f64_n1M", dict(gradients=True), 8, 4),
        (1_000_000, 10, "l10_grad_f64_n1M_point", dict(gradients=True, kernel="point"), 8, 4),
        # hard-coded l <= 3 + recursion (POINT_HC, AUTO's FP64 choice up to l_max 8
        # with gradients, 3 for values) against the all-recursion POINT kernel
        (1_000_000, 3, "l3_grad_f64_n1M_point", dict(gradients=True, kernel="point"), 8, 4),
        (1_000_000, 3, "l3_grad_f64_n1M_point_hc", dict(gradients=True, kernel="point_hc"), 8, 4),
        (4_194_304, 8, "l8_grad_f64_point", dict(gradients=True, kernel="point"), 8, 4),
        (10_000, 8, "l8_values_f64_n10k_point_hc", dict(kernel="point_hc"), 8, 1),
    ):
        dt = torch.float64 if elem == 8 else torch.float32
        x = torch.from_numpy(inputs.shell_points(n, 0.5, 5.0, seed=2)).to(dev, dt)
        K = (L + 1) ** 2
        if isinstance(kw.get("launch"), tuple):
            from paper_2302_08381_gb300 import _capi as C

            kw = dict(kw, launch=C.make_launch(*kw["launch"]))

        def fn():
            api.spherical_harmonics(x, L, **kw)

        # POINT-family forward variants use the library's autotuner too (as the
        # headline does); value-only / gradient / bf16 / FP64 shapes are tuned
        # separately, Hessian shapes keep their defaults; the other families
        # take their default shapes.
        auto_point = L <= 16 if dt == torch.float32 else L <= 11  # where AUTO runs the POINT kernels
        if auto_point and "kernel" not in kw and "qprec" not in kw and not kw.get("hessians"):
            from paper_2302_08381_gb300 import _capi as C

            sph = torch.empty((n, K), dtype=kw.get("out_dtype", dt) or dt, device=dev)
            dsph = torch.empty((n, 3, K), dtype=sph.dtype, device=dev) if kw.get("gradients") else None
            C.sphericart_autotune(
                x.data_ptr(), n, L, 1 if kw.get("normalized") else 0,
                C.SPH_F64 if dt == torch.float64 else C.SPH_F32,
                C.SPH_OUT_BF16 if kw.get("out_dtype") == torch.bfloat16 else C.SPH_OUT_SAME,
                sph.data_ptr(), dsph.data_ptr() if dsph is not None else None, stream.cuda_stream, 2,
            )
            del sph, dsph

        for _ in range(3):
            fn()
        ms = _events_ms(torch, stream, fn, 10, flush)
        nbytes = n * (3 * (8 if elem == 8 else 4) + K * elem * ddims)
        res[label] = {"n": n, "l_max": L, "ms": ms, "points_per_s": n / (ms * 1e-3),
                      "ns_per_point": ms * 1e6 / n, "achieved_GBs": nbytes / (ms * 1e-3) / 1e9}
        del x
        torch.cuda.empty_cache()
    return res


def run_expansion_leg(torch, np, api, inputs, dev, stream, flush):
    """Eq. expansion fused (harmonics never stored) vs materialised (forward
    writes Y, torch contracts and sums per centre): 100,000 centres with
    ~N(40, 10) points each, l_max = 6, 8 radial channels, FP32."""
    l_max, nr, ncent = 6, 8, 100_000
    rng = np.random.default_rng(610)
    counts = np.clip(rng.normal(40, 10, size=ncent).round(), 0, 120).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    E = int(offs[-1])
    x = torch.from_numpy(inputs.shell_points(E, 0.7, 5.0, seed=611)).to(dev)
    R = torch.from_numpy(inputs.upstream(E, nr * (l_max + 1), seed=612)).to(dev).view(E, nr, l_max + 1)
    o = torch.from_numpy(offs).to(dev)
    c = torch.empty((ncent, nr, (l_max + 1) ** 2), device=dev)

    def fused():
        api.expansion(x, R, o, l_max, out=c)

    def plain():
        return api.materialized_expansion(x, R, o, l_max)

    for _ in range(3):
        fused()
        plain()
    t_f = _events_ms(torch, stream, fused, 10, flush)
    t_p = _events_ms(torch, stream, plain, 5, flush)
    nbytes = E * (12 + nr * (l_max + 1) * 4) + ncent * (8 + nr * (l_max + 1) ** 2 * 4)
    return {
        "workload": f"{ncent} centres, {E} points, l_max={l_max}, n_rad={nr}, FP32",
        "fused_ms": t_f,
        "materialized_ms": t_p,
        "speedup": t_p / t_f,
        "fused_points_per_s": E / (t_f * 1e-3),
        "fused_achieved_GBs": nbytes / (t_f * 1e-3) / 1e9,
        "algorithmic_bytes": nbytes,
    }


def run_e2e(torch, api, inputs, dev, n, L, K, seed):
    """End to end through the public host API: pinned host xyz -> device ->
    kernel -> pinned host sph + dsph (sphericart_compute_host: chunks of
    512Ki points, H2D / kernel / D2H overlapped on three streams).
    Returns seconds per step."""
    xyz_h = torch.from_numpy(inputs.shell_points(n, 0.5, 5.0, seed=seed)).pin_memory()
    sph_h = torch.empty((n, K), dtype=torch.float32, pin_memory=True)
    dsph_h = torch.empty((n, 3, K), dtype=torch.float32, pin_memory=True)
    chunk = 1 << 19
    ws = torch.empty(2 * (chunk + 32) * 4 * (3 + 4 * K) + 4096, dtype=torch.uint8, device=dev)

    def e2e_step():
        api.spherical_harmonics_host(xyz_h, L, False, gradients=True, out=(sph_h, dsph_h), workspace=ws,
                                     chunk_points=chunk, device=dev)

    # The first transfers into freshly pinned buffers (and the first after a
    # CPU write to them) run several times slower on this machine: 3 warm-up
    # steps, then the median of 7 synchronised steps.
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    times = []
    for _ in range(7):
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    return statistics.median(times)


def run_extras(torch, np, api, inputs, dev, stream, n, L, K, sph, dsph, flush):
    out = {}
    out["variants"] = run_variants_leg(torch, api, inputs, dev, stream, flush)

    # ---- fused recompute-backward vs materialise-then-contract (l_max = 6)
    Lb = BWD_L
    Kb = (Lb + 1) ** 2
    xb_np = inputs.shell_points(BWD_N, 0.7, 6.0, seed=3)
    gb_np = inputs.upstream(BWD_N, Kb, seed=33)
    vb_np = inputs.upstream(BWD_N, 3, seed=34)
    xb = torch.from_numpy(xb_np).to(dev)
    gb = torch.from_numpy(gb_np).to(dev)
    vb = torch.from_numpy(vb_np).to(dev)
    sb = torch.empty((BWD_N, Kb), device=dev)
    db = torch.empty((BWD_N, 3, Kb), device=dev)
    dx = torch.empty_like(xb)

    def fused():
        api.spherical_harmonics(xb, Lb, False, out=(sb,))
        api.backward(xb, gb, Lb, out=dx)

    def plain():
        api.spherical_harmonics(xb, Lb, False, gradients=True, out=(sb, db))
        return torch.einsum("nik,nk->ni", db, gb)

    def fused_bwd_only():
        api.backward(xb, gb, Lb, out=dx)

    for _ in range(3):
        fused()
        plain()
    t_fused = _events_ms(torch, stream, fused, 10, flush)
    t_plain = _events_ms(torch, stream, plain, 10, flush)
    t_bwd = _events_ms(torch, stream, fused_bwd_only, 10, flush)
    t_dbwd = _events_ms(torch, stream, lambda: api.double_backward(xb, gb, vb, Lb), 10, flush)
    fused()
    dx_plain = plain()
    torch.cuda.synchronize()
    diff = float((dx.double() - dx_plain.double()).abs().max() / dx_plain.double().abs().max())
    del sb, db, gb, vb, xb, dx, dx_plain
    out["batch"] = run_batch_leg(torch, np, api, inputs, dev, stream, flush)
    out["expansion"] = run_expansion_leg(torch, np, api, inputs, dev, stream, flush)
    from paper_2302_08381_gb300 import _capi as C

    out["arith_peaks"] = {
        "fp32_tflops": C.sphericart_fma_peak(C.SPH_F32, stream.cuda_stream, 3),
        "fp64_tflops": C.sphericart_fma_peak(C.SPH_F64, stream.cuda_stream, 3),
        "method": "sphericart_fma_peak: 8 independent FMA chains per thread, 64 warps per SM, best of 3 runs "
        "of ~5 ms (2 flops per FMA)",
    }
    bwd_bytes = BWD_N * (12 + Kb * 4 + 12)
    dbwd_bytes = BWD_N * (12 + Kb * 4 + 12 + Kb * 4 + 12)
    out["backward"] = {
        "workload": f"N={BWD_N}, l_max={Lb}, |r|~U[0.7,6], g~N(0,1), FP32",
        "fused_fwd_plus_bwd_ms": t_fused,
        "plain_fwd_dsph_plus_einsum_ms": t_plain,
        "speedup_fused_vs_plain": t_plain / t_fused,
        "fused_bwd_kernel_ms": t_bwd,
        "fused_bwd_achieved_GBs": bwd_bytes / (t_bwd * 1e-3) / 1e9,
        "double_backward_ms": t_dbwd,
        "double_backward_achieved_GBs": dbwd_bytes / (t_dbwd * 1e-3) / 1e9,
        "max_rel_diff_fused_vs_plain": diff,
        "stated_error": "both within 2e-5 (max-relative) of the FP64 oracle on sampled points of this "
        "workload and within 1e-5 of central differences (h=1e-3, FP64): tests/test_backward_gpu.py",
    }
    return out


if __name__ == "__main__":
    main()
