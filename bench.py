"""Benchmark: trajectory bond-updates/s at chi_max = 128, mixed precision vs
plain FP64, with the observable error between them.

Workload (the chi = 128 configuration): 1D Haar brickwork circuits, one per
system size n in {24, 48, 64} (the size of each trajectory is drawn uniformly
from that set, seeded), depth 32, two-qubit depolarizing p = 0.005 after each
gate (with probability p both qubits are fully depolarized, each by its
optimal unraveling), chi_max = 128, truncation cutoff 1e-12 (mixed) / 1e-20
(FP64).  Synthetic inputs; no dataset.

A step is one circuit layer applied to every trajectory of the batch (one pass
of the whole hot path: centre moves, contraction, unraveling and sampling on
both qubits, Gram + eigensolve, truncation, error bookkeeping).  Before the
timed steps the states are pre-evolved (untimed) so that the middle bonds sit
at chi_max.  One bond update = one gate on one trajectory.  The MPS state of
the batch is far larger than the 129 MB L2, so every step streams it from HBM.

--impl reference runs the CPU oracle (oracle/, numpy FP64) on the host cores
for a bounded sample of the same workload and prints its own line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "trajectory bond-updates/s at chi=128, mixed vs plain FP64; observable error"
UNIT = "bond-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lemps", choices=["lemps", "reference"])
    ap.add_argument("--traj", type=int, default=4096, help="mixed-precision trajectories in the batch (one wave)")
    ap.add_argument("--fp64-traj", type=int, default=128, help="FP64 comparator trajectories")
    ap.add_argument("--pre-layers", type=int, default=10, help="untimed layers before warm-up")
    ap.add_argument("--depth", type=int, default=32)
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-sample-s", type=float, default=20.0, help="target CPU seconds for the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sizes", default="24,48,64", help="system sizes to include (profiling cases use one)")
    return ap.parse_args()


T_START = time.time()


def log(msg):
    sys.stderr.write(f"[bench {time.time() - T_START:7.1f}s] {msg}\n")
    sys.stderr.flush()


# --- clocks -----------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- workload -----------------------------------------------------------------------

def workload(args):
    from paper_2508_05745_gb300 import inputs as I
    w = I.workload_uneven(seed=args.seed, n_traj=16384, depth=args.depth)
    return w


def batch_sizes(n_of_traj, total):
    labels = n_of_traj[:total]
    return {int(n): int(np.sum(labels == n)) for n in (24, 48, 64)}


def gates_in(circ, layers):
    return [len(circ.layers[l].left_qubits) for l in layers]


# --- the GPU arm ------------------------------------------------------------------------

def trajectory_offsets(rank, per_rank, sizes):
    """Replicas: disjoint global trajectory ids for every (rank, size handle).
    Handle i of rank r starts at (r * len(sizes) + i) * per_rank; the Philox
    counters are keyed by these ids, so no two handles share a trajectory."""
    return {n: (rank * len(sizes) + i) * per_rank for i, n in enumerate(sorted(sizes))}


def combine_over_ranks(torch, dist, ms, updates, device):
    """Job time = the slowest rank's (max), bond updates summed over ranks."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def run_arm(L, torch, w, sizes, precision, args, pre, warm, steps, profile_step=False, e2e=False, offsets=None,
            barrier=None):
    """Create one Simulation per system size, pre-evolve, warm up, time `steps`
    layers.  Returns dict with timing, per-kernel profile and the sims."""
    cutoff = 1e-12 if precision == "mixed" else 1e-20
    # One CUDA stream per system size: the handles are independent, so their
    # kernels may overlap on the GPU.  The timed region is bracketed on the
    # launching stream, which every handle's stream joins before the stop event.
    sims = {}
    for n, b in sizes.items():
        if b == 0:
            continue
        sims[n] = L.Simulation(n, args.chi, b, seed=args.seed, precision=precision, cutoff=cutoff,
                               traj_offset=(offsets or {}).get(n, 0),
                               log_capacity=w["circuits"][n].n_gates, stream=torch.cuda.Stream())
    stream = torch.cuda.current_stream()

    def step(l):
        for n, s in sims.items():
            s.apply_layer(w["circuits"][n].layers[l])

    def fork(ev):
        for s in sims.values():
            s.stream.wait_event(ev)

    def join():
        for s in sims.values():
            e = torch.cuda.Event()
            e.record(s.stream)
            stream.wait_event(e)

    for l in range(pre + warm):
        step(l)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    t0 = l0 = pre + warm
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    fork(ev0)
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler select these launches
    for l in range(t0, t0 + steps):
        step(l)
    torch.cuda.nvtx.range_pop()
    join()
    ev1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ms = ev0.elapsed_time(ev1)
    updates = sum(sum(gates_in(w["circuits"][n], range(t0, t0 + steps))) * s.B for n, s in sims.items())
    out = dict(ms=ms, updates=updates, sims=sims, next_layer=t0 + steps, steps=steps)
    if e2e:
        # end to end through the public API: host gate arrays copied in every
        # apply_layer call, branch indices of the layer read back to the host.
        l1 = out["next_layer"]
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        h2d = d2h = 0
        for l in range(l1, l1 + steps):
            for n, s in sims.items():
                layer = w["circuits"][n].layers[l]
                s.apply_layer(layer)
                h2d += layer.gates.nbytes + layer.kraus.nbytes + layer.left_qubits.nbytes
            for s in sims.values():
                g_last = s.gates_applied - 1
                s.sample_branch(g_last, 1)
                d2h += 4 * s.B
        torch.cuda.synchronize()
        el = time.perf_counter() - t_start
        upd = sum(sum(gates_in(w["circuits"][n], range(l1, l1 + steps))) * s.B for n, s in sims.items())
        out.update(e2e_value=upd / el, h2d=h2d // steps, d2h=d2h // steps)
        out["next_layer"] = l1 + steps
    if profile_step:
        # per-kernel CUDA events; the handles run one after another here so
        # that no kernel's duration includes another handle's work
        l2 = out["next_layer"]
        torch.cuda.synchronize()
        work = {}
        for n, s in sims.items():
            _, bonds = s.export_mps(0)
            for k, v in layer_work(w["circuits"][n].layers[l2].left_qubits, bonds, args.chi).items():
                work[k] = work.get(k, 0.0) + v * s.B
        out["profile_work"] = work
        for s in sims.values():
            s.profile(True)
        torch.cuda.nvtx.range_push("profiled_layer")
        for n, s in sims.items():
            s.apply_layer(w["circuits"][n].layers[l2])
            torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        prof = {}
        for s in sims.values():
            for k, (kms, cnt) in s.profile(False, collect=True).items():
                a, b = prof.get(k, (0.0, 0))
                prof[k] = (a + kms, b + cnt)
        out["profile"] = prof
        out["profile_updates"] = sum(len(w["circuits"][n].layers[l2].left_qubits) * s.B for n, s in sims.items())
        out["next_layer"] = l2 + 1
    return out


def observable_error(res_m, res_d, bf_by_n):
    """Per-observable |mixed - FP64| over the FP64 trajectories (same ids)."""
    errs = {"z": [], "zz": [], "s_half": []}
    for n, rd in res_d.items():
        rm = res_m[n]
        k = bf_by_n[n]
        errs["z"].append(np.abs(rm["z"][:k] - rd["z"][:k]).ravel())
        errs["zz"].append(np.abs(rm["zz"][:k] - rd["zz"][:k]).ravel())
        errs["s_half"].append(np.abs(rm["s_half"][:k] - rd["s_half"][:k]).ravel())
    out = {}
    for k, v in errs.items():
        v = np.concatenate(v) if v else np.zeros(1)
        out[k] = {"median_abs": float(np.median(v)), "max_abs": float(np.max(v))}
    return out


# --- CPU oracle baseline -------------------------------------------------------------------

def _oracle_worker(job):
    n, traj, seed, chi, depth, pre, budget_s = job
    from oracle import trajectories as T
    from paper_2508_05745_gb300 import inputs as I
    w = I.workload_uneven(seed=seed, n_traj=16, depth=depth)
    circ = w["circuits"][n]
    marks = []
    t_start = time.perf_counter()

    class Stop(Exception):
        pass

    def cb(_):
        marks.append(time.perf_counter())
        if len(marks) > pre and marks[-1] - marks[pre - 1] > budget_s:
            raise Stop

    try:
        T.mps_trajectory(circ, traj, seed, chi_max=chi, cutoff=1e-20, layer_callback=cb)
    except Stop:
        pass
    done = len(marks)
    if done <= pre:
        return 0, 0.0
    upd = sum(len(circ.layers[l].left_qubits) for l in range(pre, done))
    return upd, marks[done - 1] - marks[pre - 1]


def cpu_baseline(args, pre_layers, budget_s):
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    # one BLAS thread per worker: set before the spawned children import numpy
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    jobs = [(48, t, args.seed, args.chi, args.depth, pre_layers, budget_s) for t in range(cores)]
    ctx = mp.get_context("spawn")
    try:
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    upd = sum(r[0] for r in res)
    secs = sum(r[1] for r in res)
    rate = upd / (secs / cores) if secs > 0 else 0.0
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} trajectories of the n=48 circuit run in parallel (spawn pool, 1 thread each); "
                      f"layers {pre_layers}.. timed per layer for ~{budget_s:.0f} s each; "
                      f"rate = updates / (summed timed seconds / cores)"}


# --- main ----------------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return main_reference(args)
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    from paper_2508_05745_gb300 import build, lemps as L
    build.build()
    w = workload(args)
    # replicas: rank r takes trajectories [r*B, (r+1)*B) of the global sample
    per_rank = args.traj
    labels = w["n_of_traj"][rank * per_rank:(rank + 1) * per_rank]
    want = [int(x) for x in args.sizes.split(",")]
    if len(want) == 3:
        sizes = {int(n): int(np.sum(labels == n)) for n in (24, 48, 64)}
    else:
        sizes = {n: per_rank // len(want) for n in want}
    log(f"sizes {sizes}")
    offsets = trajectory_offsets(rank, per_rank, sizes)
    barrier = None
    if world > 1:
        import torch.distributed as dist
        barrier = dist.barrier
    clocks = ClockSampler(local)
    clocks.start()
    mixed = run_arm(L, torch, w, sizes, "mixed", args, args.pre_layers, args.warmup, args.steps,
                    profile_step=True, e2e=not args.no_e2e, offsets=offsets, barrier=barrier)
    log(f"mixed arm: {mixed['updates']} updates in {mixed['ms']:.1f} ms")
    clk = clocks.stop()
    ms = mixed["ms"]
    if world > 1:
        import torch.distributed as dist
        ms, total_updates = combine_over_ranks(torch, dist, ms, mixed["updates"], "cuda")
    else:
        total_updates = mixed["updates"]
    value = total_updates / (ms / 1000.0)

    # FP64 comparator on the first trajectories of each size, same layers
    fp64 = None
    obs_err = None
    if not args.no_fp64 and rank == 0:
        bf = {n: min(b, max(1, args.fp64_traj * b // max(1, sum(sizes.values())))) for n, b in sizes.items() if b}
        d = run_arm(L, torch, w, bf, "fp64", args, args.pre_layers, args.warmup, args.steps)
        fp64 = d["updates"] / (d["ms"] / 1000.0)
        log(f"fp64 arm: {d['updates']} updates in {d['ms']:.1f} ms")
        # bring the mixed sims to the same depth as the FP64 sims and compare
        res_d = {}
        for n, s in d["sims"].items():
            res_d[n] = s.measure()
        # mixed sims advanced further (e2e + profile steps): rerun a mixed arm at equal depth
        mm = run_arm(L, torch, w, bf, "mixed", args, args.pre_layers, args.warmup, args.steps)
        res_m = {n: s.measure() for n, s in mm["sims"].items()}
        obs_err = observable_error(res_m, res_d, bf)
        log("observable error done")
        for s in list(d["sims"].values()) + list(mm["sims"].values()):
            s.destroy()
    prof = mixed["profile"]
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    total_prof = sum(v[0] for v in prof.values())
    rl = roofline(prof, mixed["profile_work"], args)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (FP64 unraveling/weights)", "data": "synthetic",
        "config": {"workload": "uneven: n~U{24,48,64}, depth 32 Haar brickwork, 2q depolarizing p=0.005, chi_max=128",
                   "trajectories_per_gpu": per_rank, "by_n": sizes, "pre_layers": args.pre_layers,
                   "step": "one layer over the batch", "l2": "state >> 129 MB L2 (streamed from HBM each step)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fp64_value": fp64, "mixed_over_fp64": (value / fp64) if fp64 else None,
        "observable_error_mixed_vs_fp64": obs_err,
        "e2e": {"value": mixed.get("e2e_value"), "unit": UNIT, "h2d_bytes_per_step": mixed.get("h2d"),
                "d2h_bytes_per_step": mixed.get("d2h")},
        "gpu_launches": gpu_launches(prof, args.steps, mixed["profile_updates"], mixed["updates"]),
        "kernel_share": {k: round(v[0] / total_prof, 4) for k, v in prof.items() if total_prof > 0},
        "roofline": rl, "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.pre_layers, args.cpu_sample_s)
        log("cpu baseline done")
    for s in mixed["sims"].values():
        s.destroy()
    if rank == 0:
        print(json.dumps(line))


def gpu_launches(prof, steps, prof_updates, updates):
    launches = sum(v[1] for v in prof.values())  # launches of one profiled step
    return int(launches * steps)


# Algorithmic work, in complex multiply-adds (1 CMAC = 8 real flops), of one
# layer for one trajectory, per kernel kind, from the bond dimensions b[] of
# the state before the layer (each split is assumed to grow the bond to
# min(chi, 2 dl, 2 dr)).  Gate on (q, q+1) with dl, dm, dr = b[q], b[q+1],
# b[q+2]; n_g = 2 d_s is the Gram side chosen by the next gate, d_o the other:
#   contract  (2 dl x dm)(dm x 2 dr):                 4 dl dm dr
#   gram      one triangle of n_g x n_g, K = 2 d_o:   n_g^2 d_o
#   eig       Hermitian tridiagonalization (2/3) n_g^3, back-transformation
#             of keep vectors n_g^2 keep
#   split     U^dagger Theta and the residual:        4 keep n_g d_o
#   move      per centre move, Householder QR of m x n (m n^2 - n^3 / 3),
#             explicit Q (m r^2 - r^3 / 3), triangular merge into the
#             neighbour (r n d_next, half of the r x n by n x 2 d_next product)
def _qr_work(m, n, d_next):
    r = min(m, n)
    return (m * n * n - n ** 3 / 3.0) + (m * r * r - r ** 3 / 3.0) + r * n * d_next


def layer_work(left_qubits, bonds, chi):
    b = [int(x) for x in bonds]
    nq = len(b) - 1
    w = {"contract": 0.0, "gram": 0.0, "eig": 0.0, "split": 0.0, "move": 0.0}
    qs = [int(q) for q in left_qubits]
    for i, q in enumerate(qs):
        if i > 0:
            p = qs[i - 1]
            if q > p:   # centre at p+1 moves right to q
                for k in range(p + 1, q):
                    w["move"] += _qr_work(2 * b[k], b[k + 1], b[min(k + 2, nq)])
            else:       # centre at p moves left to q+1
                for k in range(p, q + 1, -1):
                    w["move"] += _qr_work(2 * b[k + 1], b[k], b[max(k - 1, 0)])
        dl, dm, dr = b[q], b[q + 1], b[q + 2]
        right = (qs[i + 1] > q) if i + 1 < len(qs) else (i == 0 or qs[i - 1] < q)
        ds, do = (dl, dr) if right else (dr, dl)
        ng = 2 * ds
        keep = min(chi, 2 * dl, 2 * dr)
        w["contract"] += 4.0 * dl * dm * dr
        w["gram"] += ng * ng * do
        w["eig"] += (2.0 / 3.0) * ng ** 3 + ng * ng * keep
        w["split"] += 4.0 * keep * ng * do
        b[q + 1] = keep
    return w


# DRAM bytes (read + write) of one ncu capture of the kernel as it is now
# (profiles/<kernel>_chi128_n48_b152.md); remove an entry when its kernel changes.
NCU_TRAFFIC = {
    "eig": {"bytes": 243.2e6,
            "note": "one k_heev launch at the n_Gram=256 gate (gate 12 of layer 8), 152 trajectories, dram read "
                    "115.7 MB + write 127.5 MB: 1.60 MB per trajectory against ~1.5 MB of algorithmic bytes (G read, "
                    "reflectors written and read back, U written); bench launches mix gate sizes, so this is the "
                    "full-size launch, not the average"},
}


def fp32_peak_tflops():
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        sm_max = json.load(open(peaks_path)).get("sm_max_mhz", sm_max)
    # FP32 SIMT peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x clock
    return 152 * 128 * 2 * sm_max * 1e6 / 1e12


def roofline(prof, work, args, fp64=False):
    """Per kernel kind: achieved TFLOP/s = algorithmic flops of the profiled
    layer (layer_work over every trajectory, from the actual bond dimensions)
    / the summed CUDA-event time of that kind's launches; the dominant kind is
    reported."""
    peak = fp32_peak_tflops() / (64.0 if fp64 else 1.0)
    rows = {}
    for kind, (ms, cnt) in prof.items():
        if kind not in work or ms <= 0:
            continue
        flops = 8.0 * work[kind]
        ach = flops / (ms / 1000.0) / 1e12
        rows[kind] = {"ms": ms, "launches": cnt, "avg_launch_ms": ms / max(cnt, 1), "gflop": flops / 1e9,
                      "achieved_tflops": ach, "frac": ach / peak}
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0]
    r = rows.get(dom, {})
    cap = NCU_TRAFFIC.get(dom)
    return {"kernel": dom, "bound": "alu", "achieved": r.get("achieved_tflops"), "peak": peak, "unit": "TFLOP/s",
            "frac": r.get("frac"), "traffic": cap["bytes"] if cap else None,
            "traffic_note": cap["note"] if cap else None, "avg_launch_ms": r.get("avg_launch_ms"),
            "peak_note": "FP32 SIMT peak derived from 152 SMs x 128 lanes x 2 x max SM clock (MEASURED_PEAKS sm_max_mhz); of derived",
            "work_note": "algorithmic complex multiply-adds of the profiled layer from the bond dimensions "
                         "before it (bench.py layer_work), 8 flops each",
            "kernels": rows}


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(args, args.pre_layers, args.cpu_sample_s)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "uneven: n~U{24,48,64}, depth 32 Haar brickwork, 2q depolarizing p=0.005, chi_max=128"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
