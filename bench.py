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
both qubits, Gram + eigensolve, truncation, error bookkeeping).  Before any
warm-up or timed step the states are pre-evolved (untimed) so that the middle
bonds sit at chi_max.  Every warm-up and timed step is a layer of the depth-32
circuit: when the layers after the pre-evolution run out, the handles are
created afresh and pre-evolved again, untimed (`layer_plan`).  One bond update
= one gate on one trajectory.  The MPS state of the batch is far larger than
the 129 MB L2, so every step streams it from HBM.

--impl reference runs the C++ FP64 oracle (oracle/mps_oracle.cpp, OpenMP) on
the host cores for a bounded sample of the same workload and prints its own
line; the CPU baseline of the main line is the same oracle.
--gpus N without a launcher-provided WORLD_SIZE starts N ranks itself through
torch.distributed.run (replicas, one GPU each).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "trajectory bond-updates/s at chi=128, mixed vs plain FP64; observable error"
UNIT = "bond-updates/s"
WORKLOAD = "uneven: n~U{24,48,64}, depth 32 Haar brickwork, 2q depolarizing p=0.005, chi_max=128"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lemps", choices=["lemps", "reference"])
    ap.add_argument("--per-size", type=int, default=152,
                    help="trajectories of each system size per GPU (default: one per SM, so that every per-gate "
                         "launch of a size handle is one full wave of CTAs)")
    ap.add_argument("--traj", type=int, default=0,
                    help="if > 0: that many trajectories per GPU with the sizes drawn by the seeded sample instead")
    ap.add_argument("--fp64-traj", type=int, default=0, help="FP64 comparator trajectories (default: the same batch)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 steps (at most --steps)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--pre-layers", type=int, default=10, help="untimed layers before warm-up")
    ap.add_argument("--depth", type=int, default=32)
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-sample-s", type=float, default=20.0,
                    help="target timed seconds of the CPU oracle baseline (after its untimed pre-evolution)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sizes", default="24,48,64", help="system sizes to include (profiling cases use one)")
    return ap.parse_args(argv)


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


# --- workload and layer plan ------------------------------------------------------

def workload(args):
    from paper_2508_05745_gb300 import inputs as I
    return I.workload_uneven(seed=args.seed, n_traj=16384, depth=args.depth)


def gates_in(circ, layers):
    return [len(circ.layers[l].left_qubits) for l in layers]


class LayerPlan:
    """Hands out the layers of a depth-`depth` circuit for warm-up, timed,
    end-to-end and profiled steps so that every such step is a layer of the
    circuit at index >= `pre` (the pre-evolution puts the middle bonds at
    chi_max first).  When the layers run out, the next request starts with a
    reset: fresh handles, pre-evolved untimed through layers 0..pre-1.

    take(kind, count) returns a list of events ("reset", None), ("pre", l),
    (kind, l); the caller applies them in order."""

    def __init__(self, depth, pre):
        if not 0 <= pre < depth:
            raise ValueError(f"pre-evolution layers ({pre}) must leave at least one layer of the depth-{depth} circuit")
        self.depth, self.pre = depth, pre
        self.pos = depth    # no handles yet: the first request resets

    def take(self, kind, count):
        ev = []
        for _ in range(count):
            if self.pos >= self.depth:
                ev.append(("reset", None))
                ev.extend(("pre", l) for l in range(self.pre))
                self.pos = self.pre
            ev.append((kind, self.pos))
            self.pos += 1
        return ev


def timed_segments(events):
    """Split a list of plan events at the resets: [(untimed events, timed
    layers)], where the untimed events (reset / pre) precede the segment's
    timed layers."""
    segs, pending, run = [], [], []
    for e in events:
        if e[0] in ("reset", "pre"):
            if run:
                segs.append((pending, run))
                pending, run = [], []
            pending.append(e)
        else:
            run.append(e[1])
    if run or pending:
        segs.append((pending, run))
    return segs


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


class Arm:
    """One handle per system size, each on its own CUDA stream (the handles are
    independent, so their kernels may overlap); layers are applied through the
    public API (Simulation.apply_layer -> apply_layer of the C ABI)."""

    def __init__(self, L, torch, w, sizes, precision, args, offsets=None, barrier=None):
        self.L, self.torch, self.w, self.args = L, torch, w, args
        self.sizes = {n: b for n, b in sizes.items() if b > 0}
        self.precision = precision
        self.cutoff = 1e-12 if precision == "mixed" else 1e-20
        self.offsets = offsets or {}
        self.barrier = barrier
        self.sims = {}
        self.plan = LayerPlan(args.depth, args.pre_layers)
        self.resets = 0
        self.tiles = {}       # GEMM tiles per size chosen by the library's autotuner (sim_tiles)
        self.tune_ms = 0.0    # host time sim_create spent tuning (outside every timed region)

    def reset(self):
        torch = self.torch
        for s in self.sims.values():
            s.destroy()
        self.sims = {}
        for n, b in self.sizes.items():
            self.sims[n] = self.L.Simulation(n, self.args.chi, b, seed=self.args.seed, precision=self.precision,
                                             cutoff=self.cutoff, traj_offset=self.offsets.get(n, 0),
                                             log_capacity=self.w["circuits"][n].n_gates, stream=torch.cuda.Stream())
            t = self.sims[n].tiles()
            self.tune_ms += t["tune_ms"]
            self.tiles[n] = t
        self.resets += 1

    def apply(self, l):
        for n, s in self.sims.items():
            s.apply_layer(self.w["circuits"][n].layers[l])

    def untimed(self, events):
        for kind, l in events:
            if kind == "reset":
                self.reset()
            else:
                self.apply(l)

    def updates(self, layers):
        return sum(sum(gates_in(self.w["circuits"][n], layers)) * s.B for n, s in self.sims.items())

    def warmup(self, count):
        self.untimed(self.plan.take("warm", count))
        self.torch.cuda.synchronize()

    def timed(self, count):
        """Time `count` steps with CUDA events on the launching stream, one
        bracket per segment between resets (barrier + synchronize on both
        sides of each); returns (ms, updates, layers)."""
        torch = self.torch
        stream = torch.cuda.current_stream()
        ms, upd, layers = 0.0, 0, []
        for pending, run in timed_segments(self.plan.take("timed", count)):
            self.untimed(pending)
            if not run:
                continue
            torch.cuda.synchronize()
            if self.barrier:
                self.barrier()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for s in self.sims.values():
                s.stream.wait_event(ev0)
            torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler select these launches
            for l in run:
                self.apply(l)
            torch.cuda.nvtx.range_pop()
            for s in self.sims.values():
                e = torch.cuda.Event()
                e.record(s.stream)
                stream.wait_event(e)
            ev1.record(stream)
            torch.cuda.synchronize()
            if self.barrier:
                self.barrier()
            ms += ev0.elapsed_time(ev1)
            upd += self.updates(run)
            layers += run
        return ms, upd, layers

    def e2e(self, count):
        """End to end through the public API: the layer's host gate arrays are
        copied in every apply_layer call and the branch indices of the layer's
        last gate are read back to the host; wall clock around each segment."""
        torch = self.torch
        el, upd, h2d, d2h, nsteps = 0.0, 0, 0, 0, 0
        for pending, run in timed_segments(self.plan.take("e2e", count)):
            self.untimed(pending)
            if not run:
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for l in run:
                for n, s in self.sims.items():
                    layer = self.w["circuits"][n].layers[l]
                    s.apply_layer(layer)
                    h2d += layer.gates.nbytes + layer.kraus.nbytes + layer.left_qubits.nbytes
                for s in self.sims.values():
                    s.sample_branch(s.gates_applied - 1, 1)
                    d2h += 4 * s.B
            torch.cuda.synchronize()
            el += time.perf_counter() - t0
            upd += self.updates(run)
            nsteps += len(run)
        return dict(value=upd / el if el > 0 else None, h2d=h2d // max(nsteps, 1), d2h=d2h // max(nsteps, 1),
                    steps=nsteps)

    def profile_step(self):
        """Per-kernel CUDA events over one further layer; the handles run one
        after another so that no kernel's duration includes another handle's
        work.  Returns ({kind: (ms, launches)}, {kind: algorithmic CMAC}, updates)."""
        torch = self.torch
        ev = self.plan.take("profile", 1)
        self.untimed(ev[:-1])
        l = ev[-1][1]
        torch.cuda.synchronize()
        work = {}
        for n, s in self.sims.items():
            _, bonds = s.export_mps(0)
            for k, v in layer_work(self.w["circuits"][n].layers[l].left_qubits, bonds, self.args.chi).items():
                work[k] = work.get(k, 0.0) + v * s.B
        for s in self.sims.values():
            s.profile(True)
        torch.cuda.nvtx.range_push("profiled_layer")
        for n, s in self.sims.items():
            s.apply_layer(self.w["circuits"][n].layers[l])
            torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        prof = {}
        for s in self.sims.values():
            for k, (kms, cnt) in s.profile(False, collect=True).items():
                a, b = prof.get(k, (0.0, 0))
                prof[k] = (a + kms, b + cnt)
        return prof, work, self.updates([l])

    def measure(self):
        return {n: s.measure() for n, s in self.sims.items()}

    def destroy(self):
        for s in self.sims.values():
            s.destroy()
        self.sims = {}


def branch_logs(arm):
    """Sampled branch of every noise site since the handles were created,
    [B, 2 gates] per size."""
    out = {}
    for n, s in arm.sims.items():
        cols = [s.sample_branch(g, slot) for g in range(s.gates_applied) for slot in (0, 1)]
        out[n] = np.stack(cols, axis=1) if cols else np.zeros((s.B, 0), np.int32)
    return out


def observable_error(res_m, res_d, br_m=None, br_d=None):
    """Per-observable |mixed - FP64| over trajectories with the same ids whose
    sampled branches agree at every noise site (a branch can flip where a
    uniform falls within rounding of a cumulative weight), the number of
    trajectories whose branches differ, and the largest |mean_mixed -
    mean_FP64| / combined standard error over all trajectories."""
    errs = {"z": [], "zz": [], "s_half": []}
    zmax = 0.0
    divergent = 0
    for n, rd in res_d.items():
        rm = res_m[n]
        same = np.ones(len(rd["z"]), bool)
        if br_m is not None:
            same = np.all(br_m[n] == br_d[n], axis=1)
            divergent += int(np.sum(~same))
        for k in errs:
            errs[k].append(np.abs(rm[k] - rd[k])[same].ravel())
        for k, km, ks in (("z", "z_mean", "z_stderr"), ("zz", "zz_mean", "zz_stderr")):
            se = np.sqrt(rm[ks] ** 2 + rd[ks] ** 2)
            ok = se > 0
            if ok.any():
                zmax = max(zmax, float(np.max(np.abs(rm[km] - rd[km])[ok] / se[ok])))
        se = np.hypot(rm["s_half_stderr"], rd["s_half_stderr"])
        if se > 0:
            zmax = max(zmax, abs(rm["s_half_mean"] - rd["s_half_mean"]) / se)
    out = {}
    for k, v in errs.items():
        v = np.concatenate(v) if v else np.zeros(1)
        out[k] = {"median_abs": float(np.median(v)), "max_abs": float(np.max(v))}
    out["max_mean_z_score"] = zmax
    out["branch_divergent_trajectories"] = divergent
    return out


# --- CPU oracle baseline -------------------------------------------------------------------

def _oracle_batches(args, sizes, pre_layers, cores):
    """One C++ oracle batch per system size of the workload (the same seeded
    circuits as the GPU arm), one trajectory per host core, evolved untimed
    through the pre-evolution layers so that the middle bonds sit at chi_max."""
    from oracle import cpp
    from paper_2508_05745_gb300 import inputs as I
    w = I.workload_uneven(seed=args.seed, n_traj=cores, depth=args.depth)
    batches = {}
    for n in sizes:
        b = cpp.Batch(w["circuits"][n], 0, cores, args.seed, args.chi, 1e-20)
        b.run(0, pre_layers, cores)
        batches[n] = b
    return w, batches


def cpu_baseline(args, pre_layers, budget_s):
    """The C++17 FP64 oracle (oracle/mps_oracle.cpp, OpenMP, one trajectory per
    core) on the host cores: for each system size, layers after the untimed
    pre-evolution are timed with all cores until about budget_s / #sizes
    seconds have passed (at least one layer); then one further layer of one
    trajectory of the middle size with one thread gives the 1-core figure.
    rate = bond updates / wall seconds."""
    cores = os.cpu_count() or 1
    sizes = [int(x) for x in args.sizes.split(",")]
    w, batches = _oracle_batches(args, sizes, pre_layers, cores)
    by_n, upd_tot, t_tot = {}, 0, 0.0
    try:
        for n in sizes:
            circ, b = w["circuits"][n], batches[n]
            l, upd, t = pre_layers, 0, 0.0
            while l < args.depth and (l == pre_layers or t < budget_s / len(sizes)):
                t0 = time.perf_counter()
                b.run(l, l + 1, cores)
                t += time.perf_counter() - t0
                upd += cores * len(circ.layers[l].left_qubits)
                l += 1
            by_n[str(n)] = {"bond_updates": upd, "seconds": round(t, 3), "rate": upd / t, "layers": [pre_layers, l]}
            upd_tot += upd
            t_tot += t
        n1 = sizes[len(sizes) // 2]
        l1 = by_n[str(n1)]["layers"][1]
        one = None
        if l1 < args.depth:
            t0 = time.perf_counter()
            batches[n1].run_range(0, 1, l1, l1 + 1, 1)
            t1 = time.perf_counter() - t0
            u1 = len(w["circuits"][n1].layers[l1].left_qubits)
            one = {"value": u1 / t1, "unit": UNIT, "cores": 1, "n": n1, "layer": l1, "bond_updates": u1,
                   "seconds": round(t1, 3)}
    finally:
        for b in batches.values():
            b.close()
    return {"value": upd_tot / t_tot, "unit": UNIT, "cores": cores, "kind": "oracle",
            "impl": "C++17 FP64 oracle (oracle/mps_oracle.cpp), OpenMP over trajectories",
            "by_n": by_n, "one_core": one,
            "sample": f"per n in {sizes}: {cores} trajectories (one per core) pre-evolved untimed through "
                      f"{pre_layers} layers, then whole layers timed with all cores (~{budget_s:.0f} s in all); "
                      f"1-core: one more layer of one n={n1} trajectory on one thread"}


# --- roofline -------------------------------------------------------------------------------

# Algorithmic work, in complex multiply-adds (1 CMAC = 8 real flops), of one
# layer for one trajectory, per kernel kind, from the bond dimensions b[] of
# the state before the layer (each split is assumed to grow the bond to
# min(chi, 2 dl, 2 dr)).  Gate on (q, q+1) with dl, dm, dr = b[q], b[q+1],
# b[q+2]; n_g = 2 d_s is the Gram side the library picks (the smaller one
# when the site capacities cap[q], cap[q+2] differ, else the side that
# leaves the centre next to the following gate), d_o the other:
#   contract  (2 dl x dm)(dm x 2 dr):                 4 dl dm dr
#   gram      one triangle of n_g x n_g, K = 2 d_o:   n_g^2 d_o
#   eig       Hermitian tridiagonalization (2/3) n_g^3 (FP64); the
#   eig_bt    back-transformation of keep vectors n_g^2 keep runs in the same
#             launch, in the storage precision (complex64 in the mixed arm)
#   split     U^dagger Theta and the residual:        4 keep n_g d_o
#   move      per centre move, Householder QR of m x n (m n^2 - n^3 / 3),
#             explicit Q (m r^2 - r^3 / 3), triangular merge into the
#             neighbour (r n d_next, half of the r x n by n x 2 d_next product);
#             the moves before the layer's first gate are not counted
def _qr_work(m, n, d_next):
    r = min(m, n)
    return (m * n * n - n ** 3 / 3.0) + (m * r * r - r ** 3 / 3.0) + r * n * d_next


def split_sides(left_qubits, nq, chi):
    """Per gate of a layer, True when the split uses the left Gram (centre
    moves to q+1), as the library decides it (local layering, capacities
    cap[k] = min(chi, 2^min(k, n-k)))."""
    cap = [min(chi, 2 ** min(k, nq - k)) for k in range(nq + 1)]
    qs = [int(q) for q in left_qubits]
    out = []
    for i, q in enumerate(qs):
        if cap[q] != cap[q + 2]:
            out.append(cap[q] < cap[q + 2])
        else:
            out.append((qs[i + 1] > q) if i + 1 < len(qs) else (i == 0 or qs[i - 1] < q))
    return out


def layer_work(left_qubits, bonds, chi):
    b = [int(x) for x in bonds]
    nq = len(b) - 1
    w = {"contract": 0.0, "gram": 0.0, "eig": 0.0, "eig_bt": 0.0, "split": 0.0, "move": 0.0}
    qs = [int(q) for q in left_qubits]
    sides = split_sides(qs, nq, chi)
    centre = None
    for i, q in enumerate(qs):
        if centre is not None:
            if centre < q:        # the centre moves right to q
                for k in range(centre, q):
                    w["move"] += _qr_work(2 * b[k], b[k + 1], b[min(k + 2, nq)])
            elif centre > q + 1:  # the centre moves left to q+1
                for k in range(centre, q + 1, -1):
                    w["move"] += _qr_work(2 * b[k + 1], b[k], b[max(k - 1, 0)])
        dl, dm, dr = b[q], b[q + 1], b[q + 2]
        right = sides[i]
        ds, do = (dl, dr) if right else (dr, dl)
        ng = 2 * ds
        keep = min(chi, 2 * dl, 2 * dr)
        w["contract"] += 4.0 * dl * dm * dr
        w["gram"] += ng * ng * do
        w["eig"] += (2.0 / 3.0) * ng ** 3
        w["eig_bt"] += ng * ng * keep
        w["split"] += 4.0 * keep * ng * do
        b[q + 1] = keep
        centre = q + 1 if right else q
    return w


# Arithmetic type of each kernel kind in the mixed arm: the eigensolver's
# tridiagonalization works in complex128 on the FP64 pipe (its complex64
# back-transformation, eig_bt, is reported beside it), the others in complex64
# on the FP32 pipe (the contraction partly on the tensor cores).
MIXED_PIPE = {"eig": "fp64", "contract": "fp32", "gram": "fp32", "split": "fp32", "move": "fp32"}


def peaks_tflops():
    """SIMT peaks from unit counts and the maximum SM clock: 152 SMs x 128 FP32
    lanes x 2 flop (FMA) per clock, and the FP64 pipe at 1/64 of that (2 FP64
    FMA per SM and clock: the nominal 1.25 TFLOP/s of GB300 at 2070 MHz)."""
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        sm_max = json.load(open(peaks_path)).get("sm_max_mhz", sm_max)
    fp32 = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    return {"fp32": fp32, "fp64": fp32 / 64.0}


def roofline(prof, work, pipes):
    """Per kernel kind: achieved TFLOP/s = algorithmic flops of the profiled
    layer (layer_work over every trajectory, from the actual bond dimensions)
    / the summed CUDA-event time of that kind's launches, against the peak of
    the pipe it computes on; the dominant kind is reported."""
    peaks = peaks_tflops()
    rows = {}
    for kind, (ms, cnt) in prof.items():
        if kind not in work or ms <= 0:
            continue
        flops = 8.0 * work[kind]
        ach = flops / (ms / 1000.0) / 1e12
        pk = peaks[pipes.get(kind, "fp32")]
        rows[kind] = {"ms": ms, "launches": cnt, "avg_launch_ms": ms / max(cnt, 1), "gflop": flops / 1e9,
                      "achieved_tflops": ach, "pipe": pipes.get(kind, "fp32"), "peak_tflops": pk, "frac": ach / pk}
        if kind == "eig" and "eig_bt" in work:
            rows[kind]["note"] = ("gflop/achieved count the FP64 tridiagonalization only; the same launches "
                                  "also back-transform %.1f GFLOP in the storage precision" % (8.0 * work["eig_bt"] / 1e9))
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0]
    r = rows.get(dom, {})
    return {"kernel": dom, "bound": "alu", "achieved": r.get("achieved_tflops"), "peak": r.get("peak_tflops"),
            "unit": "TFLOP/s", "frac": r.get("frac"), "traffic": None,
            "traffic_note": "DRAM bytes come from ncu captures, which never run inside the bench; "
                            "the per-kernel ncu figures are kept with the profiles",
            "avg_launch_ms": r.get("avg_launch_ms"),
            "peak_note": "of derived: SIMT peak from 152 SMs x 128 FP32 lanes x 2 flop x max SM clock "
                         "(MEASURED_PEAKS sm_max_mhz); FP64 pipe = FP32 / 64",
            "work_note": "algorithmic complex multiply-adds of the profiled layer from the bond dimensions "
                         "before it (bench.py layer_work), 8 flops each; for the eigensolver the FP64 "
                         "tridiagonalization (2/3) n^3 only",
            "kernels": rows}


# --- main ----------------------------------------------------------------------------------

def spawn_ranks(args):
    """--gpus N > 1 without a launcher: run this script under
    torch.distributed.run with N ranks on 127.0.0.1 and pass its output on."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args))
    if args.impl == "reference":
        return main_reference(args)
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps must be >= 1 and --warmup >= 0")
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2508_05745_gb300 import build, lemps as L
    build.build()
    w = workload(args)
    # The batch: --per-size trajectories of each size (a stratified sample of
    # the seeded size draw), or with --traj the first trajectories of the
    # draw; replicas: rank r takes a disjoint block of ids (trajectory_offsets)
    want = [int(x) for x in args.sizes.split(",")]
    if args.traj > 0:
        labels = w["n_of_traj"][(rank * args.traj) % 16384:][:args.traj]
        sizes = {n: int(np.sum(labels == n)) for n in want} if len(want) == 3 else \
            {n: args.traj // len(want) for n in want}
    else:
        sizes = {n: args.per_size for n in want}
    per_rank = sum(sizes.values())
    log(f"sizes {sizes}")
    offsets = trajectory_offsets(rank, per_rank, sizes)
    barrier = None
    if world > 1:
        import torch.distributed as dist
        barrier = dist.barrier

    mixed = Arm(L, torch, w, sizes, "mixed", args, offsets=offsets, barrier=barrier)
    mixed.warmup(args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    ms, updates, layers = mixed.timed(args.steps)
    clk = clocks.stop()
    log(f"mixed arm: {updates} updates in {ms:.1f} ms over layers {layers} ({mixed.resets} handle sets)")
    if world > 1:
        import torch.distributed as dist
        ms, total_updates = combine_over_ranks(torch, dist, ms, updates, "cuda")
    else:
        total_updates = updates
    value = total_updates / (ms / 1000.0)
    e2e = None if args.no_e2e else mixed.e2e(min(args.e2e_steps, args.steps))
    prof, work, prof_updates = mixed.profile_step()
    autotune = tile_summary(mixed)
    observables = merged_observables(mixed.measure(), world)
    mixed.destroy()

    # FP64 comparator: the same path in complex128 on a batch that fills the
    # GPU, and a mixed arm on the same trajectories and layers for the
    # observable error
    fp64 = None
    obs_err = None
    fp64_info = None
    if not args.no_fp64 and rank == 0:
        tot = max(1, sum(sizes.values()))
        bf = {n: max(1, args.fp64_traj * b // tot) for n, b in sizes.items() if b} if args.fp64_traj > 0 else \
            {n: b for n, b in sizes.items() if b}
        k64 = max(1, min(args.fp64_steps, args.steps))
        d = Arm(L, torch, w, bf, "fp64", args, offsets=offsets)
        d.warmup(min(args.warmup, 1))
        d_ms, d_upd, d_layers = d.timed(k64)
        fp64 = d_upd / (d_ms / 1000.0)
        fp64_info = {"trajectories": sum(bf.values()), "by_n": bf, "timed_steps": k64, "ms_per_step": d_ms / k64}
        log(f"fp64 arm: {d_upd} updates in {d_ms:.1f} ms")
        res_d = d.measure()
        br_d = branch_logs(d)
        d.destroy()
        mm = Arm(L, torch, w, bf, "mixed", args, offsets=offsets)
        mm.warmup(min(args.warmup, 1))
        mm.timed(k64)
        res_m = mm.measure()
        br_m = branch_logs(mm)
        mm.destroy()
        obs_err = observable_error(res_m, res_d, br_m, br_d)
        log("observable error done")
    rl = roofline(prof, work, MIXED_PIPE)
    total_prof = sum(v[0] for v in prof.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 contractions (3xTF32 tensor cores where site capacities are 64-128), c128 tridiagonal "
                 "eigensolve with c64 back-transformation, FP64 unraveling/weights", "data": "synthetic",
        "config": {"workload": WORKLOAD, "trajectories_per_gpu": per_rank, "by_n": sizes,
                   "pre_layers": args.pre_layers, "timed_layers": layers, "handle_sets": mixed.resets,
                   "step": "one layer over the batch", "l2": "state >> 129 MB L2 (streamed from HBM each step)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "fp64_value": fp64, "fp64": fp64_info, "mixed_over_fp64": (value / fp64) if fp64 else None,
        "observable_error_mixed_vs_fp64": obs_err,
        "observables": observables,
        "e2e": None if e2e is None else {"value": e2e["value"], "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                                         "d2h_bytes_per_step": e2e["d2h"], "steps": e2e["steps"]},
        "gpu_launches": gpu_launches(prof, args.steps),
        "kernel_share": {k: round(v[0] / total_prof, 4) for k, v in prof.items() if total_prof > 0},
        "roofline": rl, "clocks": clk, "autotune": autotune,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.pre_layers, args.cpu_sample_s)
        log("cpu baseline done")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def tile_summary(arm):
    """How often each GEMM tile shape was chosen, over the gate positions of
    every size (SIMT contraction and the two Gram sides; tensor-core
    positions left out), and the time sim_create spent tuning."""
    out = {}
    for kind, key in (("contract", "contract_simt"), ("gram_left", "gram"), ("gram_right", "gram")):
        for t in arm.tiles.values():
            for bm, bn in t[kind]:
                if bm:
                    d = out.setdefault(key, {})
                    d[f"{bm}x{bn}"] = d.get(f"{bm}x{bn}", 0) + 1
    return {"tiles": out, "tune_ms": round(arm.tune_ms, 1)}


def merged_observables(res, world):
    """Trajectory averages of the states after the mixed arm's last layer, per
    system size: <Z> of the middle qubit, the half-chain entropy (nats) and the
    error bound's mean, merged exactly over the ranks (replicas)."""
    from paper_2508_05745_gb300 import replicas as RP
    out = {}
    for n in sorted(res):
        r = res[n]
        cols = np.column_stack([r["z"][:, n // 2], r["s_half"], r["eps_bound"]])
        if world > 1:
            import torch.distributed as dist
            mean, se = RP.merged_observables(dist, [cols])
        else:
            mean, se = RP.finalize(RP.exact_sums(cols))
        out[str(n)] = {"z_mid": [float(mean[0]), float(se[0])], "s_half": [float(mean[1]), float(se[1])],
                       "eps_hat": float(mean[2]), "trajectories": int(len(cols)) * world}
    return out


def gpu_launches(prof, steps):
    launches = sum(v[1] for v in prof.values())  # launches of one profiled step
    return int(launches * steps)


def main_reference(args):
    """The reference arm: the C++ FP64 oracle on the host cores, --warmup W
    untimed and --steps K timed steps on the same workload; a step is one layer
    of one system size for one trajectory per core (sizes taken in turn, after
    an untimed pre-evolution).  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sizes = [int(x) for x in args.sizes.split(",")]
    w, batches = _oracle_batches(args, sizes, args.pre_layers, cores)
    nxt = {n: args.pre_layers for n in sizes}

    def step(i):
        n = sizes[i % len(sizes)]
        l = nxt[n]
        if l >= args.depth:
            raise SystemExit("reference arm: more steps than the depth-32 circuit has layers after the pre-evolution")
        batches[n].run(l, l + 1, cores)
        nxt[n] = l + 1
        return cores * len(w["circuits"][n].layers[l].left_qubits)

    try:
        for i in range(args.warmup):
            step(i)
        t0 = time.perf_counter()
        upd = sum(step(args.warmup + i) for i in range(args.steps))
        el = time.perf_counter() - t0
    finally:
        for b in batches.values():
            b.close()
    value = upd / el
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
          "impl": "C++17 FP64 oracle (oracle/mps_oracle.cpp), OpenMP over trajectories",
          "sample": f"{args.steps} timed steps (after {args.warmup} untimed), each one layer of one n in {sizes} "
                    f"(in turn) for {cores} trajectories, one per core, after {args.pre_layers} untimed layers"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "device": f"host cores ({cores}); no GPU work",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "trajectories": cores * len(sizes), "by_n": {str(n): cores for n in sizes},
                       "pre_layers": args.pre_layers},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
