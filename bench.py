"""Benchmark of the TTNS real-time sweep on GB300.

One "step" = one symmetric one-site TDVP sweep (S(dt/2) then S*(dt/2)) of the whole
tree, one persistent kernel launch.  Default workload: the largest single-GPU
configuration, the entanglement-renormalisation tree (5 electronic states, a balanced
binary tree of 7 ER nodes over 8 chains of 60 sites, local dim 20, bond dim 40, dt 0.25
fs) with BF16X3 tensor-core contractions (FP32 accumulation) and FP64 Lanczos / QR /
gauge moves, seeded synthetic parameters.  The same line carries the singlet-fission
star tree (4 chains x 20 sites, 3xTF32) as a secondary measurement.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload NAME] [--precision bf16x3|tf32x3|fp32|fp64]

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU (torchrun).  A single tree
does not shard, so every rank advances its own replica ("replicas only", weak scaling);
the batched workload (256 spin-boson trees) is split by tree across the ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "ttns_sweeps_per_s"
UNIT = "sweeps/s"
HEADLINE = "sf_er_5state_8x60_d20_D40"
SECONDARY = "sf_5state_4x20_d10_D20"
BATCHED = "batched_spin_boson_256"

# per workload: problem factory, default precision, default timed / warm-up steps, and the
# JSON config.  The *_small entries are the same trees with short chains (same node shapes,
# same kernels) for profiler captures.
WORKLOADS = {
    HEADLINE: dict(kind="single", prec="bf16x3", steps=8, warmup=3,
                   config=dict(n_el=5, tree="ER: root + 7 ER nodes", chains=8, chain_len=60, local_dim=20,
                               bond_dim=40, dt_fs=0.25)),
    "sf_er_5state_8x12_d20_D40": dict(kind="single", prec="bf16x3", steps=8, warmup=3,
                                      config=dict(n_el=5, tree="ER: root + 7 ER nodes", chains=8, chain_len=12,
                                                  local_dim=20, bond_dim=40, dt_fs=0.25)),
    SECONDARY: dict(kind="single", prec="tf32x3", steps=30, warmup=3,
                    config=dict(n_el=5, tree="star root", chains=4, chain_len=20, local_dim=10, bond_dim=20,
                                dt_fs=0.5)),
    "sf_5state_4x4_d10_D20": dict(kind="single", prec="tf32x3", steps=30, warmup=3,
                                  config=dict(n_el=5, tree="star root", chains=4, chain_len=4, local_dim=10,
                                              bond_dim=20, dt_fs=0.5)),
    BATCHED: dict(kind="batched", prec="tf32x3", steps=3, warmup=3,
                  config=dict(n_trees=256, n_el=2, chains=1, chain_len="10-40", local_dim=4, bond_dim="12-24",
                              dt_fs=0.5)),
}
PRECISIONS = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "fp32": 3}
DTYPE = {"fp64": "f64", "tf32x3": "tf32x3 (contractions) + f64 (Lanczos) + double-single (QR, gauge)",
         "bf16x3": "bf16x3 (contractions) + f64 (Lanczos) + double-single (QR, gauge)",
         "fp32": "f32 (contractions) + f64 (Lanczos) + double-single (QR, gauge)"}


def make_problems(name: str):
    from paper_1710_01362_gb300 import workloads as W
    if name == HEADLINE:
        return [W.sf_er_5state_8x60()]
    if name == "sf_er_5state_8x12_d20_D40":
        return [W.sf_er_5state_8x60(L=12, n_steps=40)]
    if name == SECONDARY:
        return [W.sf_5state_4x20()]
    if name == "sf_5state_4x4_d10_D20":
        return [W.singlet_fission(seed=2, n_env=4, L=4, d=10, D=20, n_modes=40, dt=0.5, n_steps=400, name=name)]
    if name == BATCHED:
        return [W.batched_spin_boson(s) for s in range(1000, 1256)]
    raise KeyError(name)


def _peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


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


def host_info():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count() or 1, "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


def _oracle_sweeps(problem, n_warm: int, n_steps: int):
    from oracle.ttns import TTNS
    st = TTNS(problem)
    for _ in range(n_warm):
        st.step(problem.dt)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        st.step(problem.dt)
    return time.perf_counter() - t0


def _oracle_problem(name: str):
    from paper_1710_01362_gb300 import workloads as W
    if name == HEADLINE:
        return W.sf_er_5state_8x60(L=12, n_steps=40), (1 + 7 + 8 * 12) / (1 + 7 + 8 * 60)
    return make_problems(name)[0], 1.0


def _oracle_child(name: str, n_warm: int, n_steps: int) -> None:
    p, _ = _oracle_problem(name)
    print(json.dumps({"seconds": _oracle_sweeps(p, n_warm, n_steps)}), flush=True)


def cpu_oracle(name: str, n_warm: int = 0, n_steps: int = 1):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload: whole sweeps of
    the same tree, or for the 8 x 60 ER tree of the same tree with 12-site chains (every
    chain-site node has the same shape, so the per-sweep cost scales with the node count,
    488 / 104), timed in a child process on one thread (BLAS thread pools set to 1) and here
    on all threads of the host."""
    info = host_info()
    p, scale = _oracle_problem(name)
    if name == HEADLINE:
        sample = f"{n_steps} sweep(s) after {n_warm} warm-up of the same ER tree with 12-site chains; " \
                 "sweeps/s extrapolated to 60-site chains by the node count (104 / 488)"
    else:
        sample = f"{n_steps} full sweep(s) after {n_warm} warm-up of the same tree"
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", name, str(n_warm), str(n_steps)],
                       capture_output=True, text=True, env=env, cwd=HERE)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    t1 = json.loads(lines[-1])["seconds"] if r.returncode == 0 and lines else None
    tall = _oracle_sweeps(p, n_warm, n_steps)
    vall = n_steps / tall * scale
    v1 = n_steps / t1 * scale if t1 else None
    best_single = v1 is not None and v1 > vall
    return {"value": v1 if best_single else vall, "unit": UNIT, "cores": 1 if best_single else info["nproc"],
            "kind": "oracle", "sample": sample, "single_thread": v1, "all_threads": vall, "nproc": info["nproc"],
            "cpu_model": info["cpu_model"], "seconds": (t1 or 0.0) + tall}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    spec = WORKLOADS[name]
    if spec["kind"] != "single":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single trees only"}))
        return
    n = max(1, min(args.steps, 2))
    warm = min(args.warmup, 1) if name != HEADLINE else 0
    cb = cpu_oracle(name, warm, n)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": n, "warmup": warm, "ms_per_step": 1e3 / cb["value"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": dict(workload=name, **spec["config"]),
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(tree, stream, dt, K, flush, torch):
    """K steps, each bracketed by CUDA events on the tree's stream, L2 flushed before each."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()                      # untimed: evicts L2 between steps
        ev[k][0].record(stream)
        tree.step(dt, 1)                   # one persistent launch = one sweep
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_single(name, prec, K, Wm, dev, stream, lf, torch, shard, ttns, world, want_clocks=True):
    """Device-resident timing of one tree (replicated on every rank), end to end through the
    public API from host data, and the parity against the oracle's stored trajectory."""
    p = make_problems(name)[0]
    with torch.cuda.stream(stream):
        tree = ttns.Tree(p, precision=prec, record=True, max_record=K + Wm + 8, stream=stream.cuda_stream,
                         launch_flags=lf)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
        for _ in range(Wm):
            tree.step(p.dt, 1)
        tree.sync()
        c0 = tree.counters()
        shard.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index) if want_clocks else None
        if clocks:
            clocks.start()
        times = time_steps(tree, stream, p.dt, K, flush, torch)
        clk = clocks.stop() if clocks else None
        tree.sync()
        c1 = tree.counters()
        shard.barrier()
        total_ms = shard.max_over_ranks(float(sum(times)))
        pop_err = None
        gpath = os.path.join(HERE, "tests", "golden", name + ".json")
        if os.path.exists(gpath):
            with open(gpath) as f:
                gd = json.load(f)
            tr = tree.trajectory()
            pops = np.real(np.einsum("kii->ki", tr))
            ref = np.array(gd["populations"])[1:1 + len(pops)]
            pop_err = float(np.abs(pops[: len(ref)] - ref).max())
        pops_end = tree.populations().tolist()
        occ_end = tree.occupations()
        tree.close()
        del flush

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
    return dict(p=p, times=times, total_ms=total_ms, c0=c0, c1=c1, clocks=clk, pop_err=pop_err, pops_end=pops_end,
                occ_end=occ_end, h2d=h2d, e2e_s=e2e_s,
                value=shard.aggregate_rate(K, world, total_ms * 1e-3),
                e2e_value=shard.aggregate_rate(K, world, e2e_s))


def roofline(res, prec_name, world):
    """The dominant (only) kernel, k_sweep: useful contraction flops (the sum-of-products terms,
    8 real flops per complex multiply-add, device-counted Krylov iterations) per launch over its
    CUDA-event time, against the tensor peak of the contraction dtype."""
    peaks, kind = _peaks()
    K = len(res["times"])
    flops = res["c1"]["contraction_flops"] - res["c0"]["contraction_flops"]
    achieved = flops / (res["total_ms"] * 1e-3) / 1e12 / world if res["total_ms"] > 0 else 0.0
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    if prec_name == "bf16x3":
        peak, note = bf16, f"measured bf16 dense, sustained ({kind})"
    elif prec_name == "tf32x3":
        peak, note = bf16 * 1.1 / 2.25, f"measured bf16 sustained x nominal tf32/bf16 ratio 1.1/2.25 ({kind})"
    else:
        peak, note = 152 * 128 * 2 * 2070e6 / 1e12, "FP32 SIMT FMA peak from unit counts and max clock"
    return {"bound": "tensor" if prec_name in ("bf16x3", "tf32x3") else "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
            "traffic": None, "kernel": "k_sweep (whole sweep, one persistent launch)",
            "flops_per_launch": flops / K, "peak_note": note,
            "issued_tensor_flops_factor": 6 if prec_name == "bf16x3" else (3 if prec_name == "tf32x3" else 0)}


def precision_study(name, prec, pname, N, stream, lf, torch, ttns):
    """The workload run N steps in the given precision and in FP64 on the GPU, one after the
    other: the largest population difference at every step (reported per eighth of the run),
    the occupations every N/8 steps, and both paths' device time per step."""
    p = make_problems(name)[0]
    every = max(1, N // 8)
    runs = {}
    for label, pr in ((pname, prec), ("fp64", ttns.TTNS_FP64)):
        with torch.cuda.stream(stream):
            t = ttns.Tree(p, precision=pr, record=True, max_record=N, stream=stream.cuda_stream, launch_flags=lf)
            occ, ms = [], 0.0
            done = 0
            while done < N:
                n = min(every, N - done)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                t.step(p.dt, n)
                b.record(stream)
                torch.cuda.synchronize()
                ms += a.elapsed_time(b)
                done += n
                occ.append(t.occupations())
                # progress (a partial record survives an interrupted run)
                print(json.dumps({"study_progress": label, "steps_done": done, "ms_per_step": ms / done,
                                  "populations": t.populations().tolist()}), flush=True)
            tr = t.trajectory(max_steps=N)
            runs[label] = dict(pops=np.real(np.einsum("kii->ki", tr)), occ=np.array(occ), ms_per_step=ms / N,
                               norm_dev=float(np.abs(np.real(np.einsum("kii->k", tr)) - 1).max()))
            t.close()
    a, b = runs[pname], runs["fp64"]
    d = np.abs(a["pops"] - b["pops"]).max(axis=1)
    docc = np.abs(a["occ"] - b["occ"]).reshape(len(a["occ"]), -1).max(axis=1)
    return {"study": "precision", "workload": name, "steps": N, "dt_fs": p.dt, "precision": pname,
            "max_pop_diff": float(d.max()), "max_pop_diff_per_eighth": [float(x) for x in d.reshape(-1, every).max(axis=1)]
            if N % every == 0 else [float(d.max())],
            "max_occ_diff": float(docc.max()), "occ_diff_every": every, "max_occ_diff_per_eighth": docc.tolist(),
            "max_occupation": float(b["occ"].max()),
            "ms_per_step": {pname: a["ms_per_step"], "fp64": b["ms_per_step"]},
            "trace_dev": {pname: a["norm_dev"], "fp64": b["norm_dev"]},
            "populations_end": {pname: a["pops"][-1].tolist(), "fp64": b["pops"][-1].tolist()}}


def run_batched(name, prec, K, Wm, dev, stream, lf, torch, shard, ttns, rank, world):
    """256 independent trees split by tree across the ranks; value = tree-sweeps of all ranks
    over the slowest rank's time."""
    probs = make_problems(name)
    lo, hi = shard.shard_range(len(probs), rank, world)
    mine = probs[lo:hi]
    with torch.cuda.stream(stream):
        tree = ttns.Tree(mine, precision=prec, stream=stream.cuda_stream, cluster_ctas=4, launch_flags=lf)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
        for _ in range(Wm):
            tree.step(mine[0].dt, 1)
        tree.sync()
        shard.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        times = time_steps(tree, stream, mine[0].dt, K, flush, torch)
        clk = clocks.stop()
        tree.sync()
        shard.barrier()
        total_ms = shard.max_over_ranks(float(sum(times)))
        tree.close()
    return dict(times=times, total_ms=total_ms, clocks=clk, n_trees=len(probs), mine=(lo, hi),
                value=len(probs) * K / (total_ms * 1e-3))


def main():
    if len(sys.argv) == 5 and sys.argv[1] == "--oracle-child":
        return _oracle_child(sys.argv[2], int(sys.argv[3]), int(sys.argv[4]))
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: the workload's default)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="", choices=[""] + sorted(PRECISIONS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--plain-cluster-launch", action="store_true",
                    help="launch the persistent kernel without the cooperative attribute (profiler runs)")
    ap.add_argument("--precision-study", type=int, default=0, metavar="N",
                    help="instead of the benchmark: N steps of the workload in its precision and in FP64, "
                         "populations of every step and occupations every N/8 steps compared (one JSON line)")
    args = ap.parse_args()
    spec = WORKLOADS[args.workload]
    if args.steps <= 0:
        args.steps = spec["steps"]
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
    build.build()
    stream = torch.cuda.Stream(device=dev)
    pname = args.precision or spec["prec"]
    prec = PRECISIONS[pname]
    K, Wm = args.steps, max(args.warmup, 3)
    lf = 1 if args.plain_cluster_launch else 0

    if spec["kind"] == "batched":
        res = run_batched(args.workload, prec, K, Wm, dev, stream, lf, torch, shard, ttns, rank, world)
        out = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
               "ms_per_step": res["total_ms"] / K, "higher_is_better": True, "scaling": "strong",
               "vs_baseline": None, "dtype": DTYPE[pname], "data": "synthetic (seeded)",
               "config": dict(workload=args.workload, precision=pname, parallelism=f"trees split over {world} rank(s)",
                              l2="flushed (256 MB write) before every step", **spec["config"]),
               "gpu_launches": K, "clocks": res["clocks"],
               "note": "value = tree-sweeps of all 256 trees per second (one step advances every tree)"}
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    if args.precision_study > 0:
        if rank == 0:
            print(json.dumps(precision_study(args.workload, prec, pname, args.precision_study, stream, lf, torch, ttns)),
                  flush=True)
        return

    res = run_single(args.workload, prec, K, Wm, dev, stream, lf, torch, shard, ttns, world)
    c0, c1 = res["c0"], res["c1"]
    iters = c1["krylov_iters"] - c0["krylov_iters"]
    roof = roofline(res, pname, world)
    out = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": res["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[pname], "data": "synthetic (seeded)",
        "config": dict(workload=args.workload, precision=pname, l2="flushed (256 MB write) before every step",
                       parallelism="replicas" if world > 1 else "single GPU", **spec["config"]),
        "e2e": {"value": res["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": res["h2d"] / K,
                "d2h_bytes_per_step": 16 * res["p"].n_el ** 2,
                "note": f"timed: ttns_build_tree from host parameters ({res['h2d']} B uploaded), {K} x (ttns_step + "
                        "rho_S read to pinned host memory), ttns_free"},
        "gpu_launches": K,
        "clocks": res["clocks"],
        "roofline": roof,
        "contraction_tflops": roof["achieved"],
        "krylov_iters_per_step": iters / K,
        "max_pop_err_vs_oracle": res["pop_err"],
    }
    if rank == 0 and world == 1 and not args.no_fp64_compare and prec != 0:
        # the plain FP64 GPU path on the same tree and the same number of steps: its speed and
        # the largest population / occupation difference at the end
        p = res["p"]
        n64 = Wm + K
        with torch.cuda.stream(stream):
            t64 = ttns.Tree(p, precision=ttns.TTNS_FP64, stream=stream.cuda_stream, launch_flags=lf)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t64.step(p.dt, Wm)
            a.record(stream)
            t64.step(p.dt, K)
            b.record(stream)
            torch.cuda.synchronize()
            pops64 = t64.populations()
            occ64 = t64.occupations()
            out["fp64_path"] = {"sweeps_per_s": K / (a.elapsed_time(b) * 1e-3), "steps": n64,
                                "max_pop_diff": float(np.abs(np.array(res["pops_end"]) - pops64).max()),
                                "max_occ_diff": float(np.abs(res["occ_end"] - occ64).max())}
            t64.close()
    if rank == 0 and world == 1 and not args.no_secondary and args.workload == HEADLINE:
        sp = WORKLOADS[SECONDARY]
        r2 = run_single(SECONDARY, PRECISIONS[sp["prec"]], sp["steps"], 3, dev, stream, lf, torch, shard, ttns, 1,
                        want_clocks=False)
        out["secondary"] = {"workload": SECONDARY, "precision": sp["prec"], "value": r2["value"], "unit": UNIT,
                            "ms_per_step": r2["total_ms"] / sp["steps"], "e2e": r2["e2e_value"],
                            "max_pop_err_vs_oracle": r2["pop_err"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle(args.workload, 0, 1)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
