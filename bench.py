"""Benchmark of the TTNS real-time sweep on GB300.

One "step" = one symmetric one-site TDVP sweep (S(dt/2) then S*(dt/2)) of the
whole tree.  Default workload: the singlet-fission-shaped tree (5 electronic
states, root with 4 chains of 20 sites, local dim 10, bond dim 20, dt 0.5 fs),
seeded synthetic parameters, mixed precision (contractions in FP32 arithmetic,
Lanczos / QR / gauge moves in FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU (torchrun); a
single tree does not shard, so every rank advances its own replica ("replicas
only", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

# DRAM bytes (read + write) of one k_sweep launch (one headline step), from one ncu capture
# of dram__bytes_read.sum + dram__bytes_write.sum for this kernel build (mean of two launches)
KSWEEP_DRAM_BYTES_PER_STEP = 664.14e6

METRIC = "ttns_sweeps_per_s"
UNIT = "sweeps/s"
WORKLOAD = "sf_5state_4x20_d10_D20"
# the headline tree, and the same tree with 4-site chains (same root, same kernels) used as
# the small case for detailed profiler captures
WORKLOADS = {
    "sf_5state_4x20_d10_D20": dict(L=20),
    "sf_5state_4x4_d10_D20": dict(L=4),
}


def make_problem(name: str):
    from paper_1710_01362_gb300 import workloads as W
    if name == WORKLOAD:
        return W.sf_5state_4x20()
    return W.singlet_fission(seed=2, n_env=4, L=WORKLOADS[name]["L"], d=10, D=20, n_modes=40, dt=0.5,
                             n_steps=400, name=name)


def _peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle(problem, n_warm: int, n_steps: int):
    """The FP64 CPU oracle on a bounded sample of the workload (whole sweeps)."""
    from oracle.ttns import TTNS
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    st = TTNS(problem)
    for _ in range(n_warm):
        st.step(problem.dt)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        st.step(problem.dt)
    dt = time.perf_counter() - t0
    return n_steps / dt, cores, dt


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1710_01362_gb300 import workloads as W
    p = W.sf_5state_4x20()
    warm = min(args.warmup, 1)
    n = max(1, min(args.steps, 6))
    value, cores, secs = cpu_oracle(p, warm, n)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": n, "warmup": warm, "ms_per_step": 1e3 * secs / n, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "n_el": 5, "chains": 4, "chain_len": 20, "local_dim": 10,
                   "bond_dim": 20, "dt_fs": p.dt},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} full sweeps after {warm} warm-up sweep(s) of the headline tree"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--plain-cluster-launch", action="store_true",
                    help="launch the persistent kernel without the cooperative attribute (profiler runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1710_01362_gb300 import build, shard, ttns
    from paper_1710_01362_gb300 import workloads as W
    if rank == 0 or world > 1:
        build.build()
    p = make_problem(args.workload)
    L = WORKLOADS[args.workload]["L"]
    stream = torch.cuda.Stream(device=dev)
    prec = ttns.TTNS_MIXED if args.precision == "mixed" else ttns.TTNS_FP64
    K, Wm = args.steps, max(args.warmup, 3)
    lf = 1 if args.plain_cluster_launch else 0

    with torch.cuda.stream(stream):
        tree = ttns.Tree(p, precision=prec, record=True, max_record=K + Wm + 8, stream=stream.cuda_stream,
                         launch_flags=lf)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
        for _ in range(Wm):
            tree.step(p.dt, 1)
        tree.sync()
        c0 = tree.counters()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        shard.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        for k in range(K):
            flush.zero_()                      # untimed: evicts L2 between steps
            ev[k][0].record(stream)
            tree.step(p.dt, 1)                 # one persistent launch = one sweep
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        tree.sync()
        times = [a.elapsed_time(b) for a, b in ev]  # ms
        c1 = tree.counters()
        shard.barrier()
        total_ms = shard.max_over_ranks(float(sum(times)))  # the slowest replica's time
        value = shard.aggregate_rate(K, world, total_ms * 1e-3)

        # populations vs the oracle's stored trajectory (steps 1..Wm+K)
        pop_err = None
        gpath = os.path.join(HERE, "tests", "golden", args.workload + ".json")
        if os.path.exists(gpath):
            with open(gpath) as f:
                gd = json.load(f)
            tr = tree.trajectory()
            pops = np.real(np.einsum("kii->ki", tr))
            ref = np.array(gd["populations"])[1:1 + len(pops)]
            pop_err = float(np.abs(pops[: len(ref)] - ref).max())

        tree.close()

        # end to end through the public API from host data: the timed region builds the tree
        # from the host-side Hamiltonian parameters (operator tables and initial state copied
        # host -> device), runs K steps, reads rho_S into pinned host memory after every step,
        # and frees the tree
        rho_host = torch.empty(2 * p.n_el * p.n_el, dtype=torch.float64, pin_memory=True)
        rho_np = rho_host.numpy()
        plan = ttns.plan([p], precision=prec)
        h2d = 16 * plan["pool_complex"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t2 = ttns.Tree(p, precision=prec, stream=stream.cuda_stream, launch_flags=lf)
        for _ in range(K):
            t2.step(p.dt, 1)
            ttns.lib().ttns_reduced_density_matrix(t2.h, 0, ttns._dptr(rho_np))
        t2.close()
        e2e_s = shard.max_over_ranks(time.perf_counter() - t0)
        e2e_value = shard.aggregate_rate(K, world, e2e_s)

    flops = c1["contraction_flops"] - c0["contraction_flops"]
    iters = c1["krylov_iters"] - c0["krylov_iters"]
    peaks, peak_kind = _peaks()
    fp32_peak_tflops = 152 * 128 * 2 * 2070e6 / 1e12  # FP32 FMA units x 2 flops x max SM clock
    achieved = flops / (total_ms * 1e-3) / 1e12 / world if total_ms > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak_tflops,
            "traffic": KSWEEP_DRAM_BYTES_PER_STEP if args.workload == WORKLOAD else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "kernel": "k_sweep (whole sweep, one persistent launch)",
            "peak_note": "FP32 SIMT FMA peak from unit counts and max clock (152 SMs x 128 lanes x 2 x 2.07 GHz)"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 contractions + f64 Lanczos/QR" if prec == ttns.TTNS_MIXED else "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "n_el": 5, "chains": 4, "chain_len": L, "local_dim": 10, "bond_dim": 20,
                   "dt_fs": p.dt, "precision": args.precision, "l2": "flushed (256 MB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": 16 * p.n_el * p.n_el,
                "note": f"timed: ttns_build_tree from host parameters ({h2d} B uploaded), {K} x (ttns_step + "
                        "rho_S read to pinned host memory), ttns_free"},
        "gpu_launches": K,
        "clocks": clk,
        "roofline": roof,
        "contraction_tflops": achieved,
        "krylov_iters_per_step": iters / K,
        "max_pop_err_vs_oracle": pop_err,
        "peaks": peak_kind,
    }
    if rank == 0 and world == 1 and not args.no_fp64_compare and prec == ttns.TTNS_MIXED:
        with torch.cuda.stream(stream):
            t64 = ttns.Tree(p, precision=ttns.TTNS_FP64, stream=stream.cuda_stream, launch_flags=lf)
            t64.step(p.dt, 2)
            t64.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n64 = max(2, K // 5)
            a.record(stream)
            t64.step(p.dt, n64)
            b.record(stream)
            torch.cuda.synchronize()
            out["fp64_path_sweeps_per_s"] = n64 / (a.elapsed_time(b) * 1e-3)
            t64.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, secs = cpu_oracle(p, 0, 2)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "2 full sweeps of the same tree from t = 0 (FP64 numpy oracle)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
