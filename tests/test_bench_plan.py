"""The bench's layer scheduling, without a GPU: every warm-up, timed, end-to-end
and profiled step of the depth-32 workload is a layer of the circuit after the
pre-evolution, for the driver's --steps 20 --warmup 5 and for the defaults.
The real Arm class runs against stand-ins for torch.cuda and the library
handle that record which layers each handle received."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2508_05745_gb300 import inputs as I  # noqa: E402


def test_plan_never_passes_the_circuit_depth():
    for depth, pre, warm, steps in [(32, 10, 5, 20), (32, 10, 3, 3), (32, 10, 0, 1), (12, 10, 4, 9), (32, 0, 40, 40)]:
        plan = bench.LayerPlan(depth, pre)
        ev = plan.take("warm", warm) + plan.take("timed", steps) + plan.take("e2e", 5) + plan.take("profile", 1)
        handles, applied = 0, []
        for kind, l in ev:
            if kind == "reset":
                handles += 1
                applied = []
                continue
            assert 0 <= l < depth
            if kind != "pre":
                assert l >= pre, (kind, l)
            applied.append(l)
            # every handle set sees the circuit's layers in order from layer 0
            assert applied == list(range(len(applied)))
        assert sum(k == "timed" for k, _ in ev) == steps
        assert sum(k == "warm" for k, _ in ev) == warm
        assert handles >= 1


def test_plan_rejects_pre_evolution_beyond_depth():
    with pytest.raises(ValueError):
        bench.LayerPlan(10, 10)


def test_segments_split_at_resets():
    plan = bench.LayerPlan(32, 10)
    plan.take("warm", 5)
    segs = bench.timed_segments(plan.take("timed", 20))
    assert [len(run) for _, run in segs] == [17, 3]
    assert segs[0][0] == [] and segs[1][0][0] == ("reset", None)
    assert segs[0][1] == list(range(15, 32)) and segs[1][1] == [10, 11, 12]


# --- stand-ins -------------------------------------------------------------------------

class _Event:
    clock = [0.0]

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        _Event.clock[0] += 1.0
        self.t = _Event.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t


class _Stream:
    cuda_stream = 0

    def wait_event(self, ev):
        pass


def _fake_torch():
    cuda = types.SimpleNamespace(
        Event=_Event, Stream=_Stream, current_stream=lambda: _Stream(), synchronize=lambda: None,
        nvtx=types.SimpleNamespace(range_push=lambda name: None, range_pop=lambda: None))
    return types.SimpleNamespace(cuda=cuda)


class _Sim:
    created = []

    def __init__(self, n, chi, B, seed=0, precision="mixed", cutoff=None, traj_offset=0, log_capacity=0,
                 stream=None):
        self.n, self.B, self.stream, self.layers, self.gates_applied = n, B, stream, [], 0
        self.circ = None
        _Sim.created.append(self)

    def apply_layer(self, layer):
        # the layer object must be the next layer of this size's circuit
        self.layers.append(layer)
        self.gates_applied += len(layer.left_qubits)

    def sample_branch(self, g, s):
        assert 0 <= g < self.gates_applied
        return np.zeros(self.B, np.int32)

    def export_mps(self, t):
        return None, np.full(self.n + 1, 2, np.int32)

    def profile(self, enable, collect=False):
        return {k: (1.0, 1) for k in ("move", "contract", "unravel", "gram", "eig", "split", "other")} if collect else None

    def tiles(self):
        t = np.tile(np.array([[64, 64]], np.int32), (self.n - 1, 1))
        c = t.copy()
        c[self.n // 2] = 0   # a tensor-core position
        return {"contract": c, "gram_left": t, "gram_right": t, "tune_ms": 1.5 if len(_Sim.created) == 1 else 0.0}

    def measure(self):
        return {}

    def destroy(self):
        pass


@pytest.mark.parametrize("steps,warmup", [(20, 5), (3, 3)])
def test_arm_runs_the_driver_schedule(steps, warmup):
    args = bench.parse(["--steps", str(steps), "--warmup", str(warmup)])
    w = I.workload_uneven(seed=0, n_traj=64, depth=args.depth)
    L = types.SimpleNamespace(Simulation=_Sim)
    _Sim.created = []
    arm = bench.Arm(L, _fake_torch(), w, {24: 3, 48: 2, 64: 1}, "mixed", args)
    arm.warmup(args.warmup)
    ms, upd, layers = arm.timed(args.steps)
    assert len(layers) == steps and all(args.pre_layers <= l < args.depth for l in layers)
    e2e = arm.e2e(min(args.e2e_steps, args.steps))
    assert e2e["steps"] == min(args.e2e_steps, args.steps)
    prof, work, pu = arm.profile_step()
    assert pu > 0 and work["eig"] > 0
    for s in _Sim.created:
        circ = w["circuits"][s.n]
        # each handle received a prefix of its circuit's layers, in order
        assert len(s.layers) <= len(circ.layers)
        assert all(a is b for a, b in zip(s.layers, circ.layers))
    expect = sum(sum(len(w["circuits"][n].layers[l].left_qubits) for l in layers) * b
                 for n, b in {24: 3, 48: 2, 64: 1}.items())
    assert upd == expect
    tiles = bench.tile_summary(arm)
    assert tiles["tune_ms"] == 1.5
    assert tiles["tiles"]["gram"] == {"64x64": 2 * (23 + 47 + 63)}
    assert tiles["tiles"]["contract_simt"] == {"64x64": 22 + 46 + 62}


def test_work_model_follows_the_gram_side_rule():
    """The bench's algorithmic-work model picks the split's Gram side as the
    library does: the smaller Gram where the site capacities around the pair
    differ, else the side that leaves the centre next to the following gate.
    On a saturated n=24, chi=128 state the eigensolver work of an ascending
    layer is then sum_q (2/3) min(2 cap_q, 2 cap_q+2)^3."""
    n, chi = 24, 128
    cap = [min(chi, 2 ** min(k, n - k)) for k in range(n + 1)]
    asc = list(range(0, n - 1, 2))
    sides = bench.split_sides(asc, n, chi)
    assert sides == [q < 16 for q in asc]
    desc = list(range(1, n - 1, 2))[::-1]
    assert bench.split_sides(desc, n, chi) == [q < 7 for q in desc]
    w = bench.layer_work(asc, cap, chi)
    expect = sum((2.0 / 3.0) * min(2 * cap[q], 2 * cap[q + 2]) ** 3 for q in asc)
    assert abs(w["eig"] - expect) <= 1e-12 * expect
