"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds none of the simulation method's arithmetic.  It only draws
circuits and channel descriptions, so that the CPU oracle and the GPU library
receive the same problem through their own interfaces:

* Haar-random two-qubit gates (Mezzadri's QR recipe for the circular unitary
  ensemble), used for the random brickwork circuits of Sec. VI (Fig. 8 and the
  random-circuit blocks figure).
* Kraus sets of the single-qubit channels the paper works with: depolarizing
  (App. A.4, the Pauli "mixed-unitary" set), amplitude damping (App. A.4,
  "Orthogonal" set) and dephasing in the paper's convention
  (1 - p/2) rho + (p/2) Z rho Z (Sec. II, channel descriptions).
* The RZZ / RX kicked-Ising gates and the random two-site tensors of the
  differentiation workload.

Gate convention: a two-qubit gate on (q, q+1) is a 4x4 complex matrix whose
row/column index is 2*s_q + s_{q+1}.  Kraus operators are 2x2, K[s', s].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

PAULI_I = np.eye(2, dtype=np.complex128)
PAULI_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PAULI_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PAULI_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


@dataclasses.dataclass
class Layer:
    """One circuit layer: two-qubit gates on disjoint neighbouring pairs, each
    followed by the layer's single-qubit noise channel on both gated qubits.

    ``coin_p`` < 1 means the noise acts only with that probability per gate
    (the reading used for two-qubit depolarizing noise: with probability p both
    qubits are fully depolarized, otherwise nothing happens)."""
    left_qubits: np.ndarray            # (n_gates,) int32, gate k acts on (q, q+1)
    gates: np.ndarray                  # (n_gates, 4, 4) complex128
    kraus: np.ndarray                  # (r, 2, 2) complex128
    coin_p: float = 1.0


@dataclasses.dataclass
class Circuit:
    n_qubits: int
    layers: List[Layer]

    @property
    def n_gates(self) -> int:
        return int(sum(len(l.left_qubits) for l in self.layers))


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random d x d unitary: QR of a complex Ginibre matrix with the phases
    of R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def depolarizing_kraus(p: float) -> np.ndarray:
    """{sqrt(1-3p/4) I, sqrt(p)/2 X, sqrt(p)/2 Y, sqrt(p)/2 Z} (App. A.4)."""
    return np.stack([math.sqrt(1.0 - 0.75 * p) * PAULI_I,
                     0.5 * math.sqrt(p) * PAULI_X,
                     0.5 * math.sqrt(p) * PAULI_Y,
                     0.5 * math.sqrt(p) * PAULI_Z])


def amplitude_damping_kraus(gamma: float) -> np.ndarray:
    """{[[1,0],[0,sqrt(1-g)]], [[0,sqrt(g)],[0,0]]} (App. A.4, "Orthogonal")."""
    k0 = np.array([[1.0, 0.0], [0.0, math.sqrt(1.0 - gamma)]], dtype=np.complex128)
    k1 = np.array([[0.0, math.sqrt(gamma)], [0.0, 0.0]], dtype=np.complex128)
    return np.stack([k0, k1])


def dephasing_kraus(p: float) -> np.ndarray:
    """{sqrt(1-p/2) I, sqrt(p/2) Z}: the paper's convention (Sec. II)."""
    return np.stack([math.sqrt(1.0 - 0.5 * p) * PAULI_I, math.sqrt(0.5 * p) * PAULI_Z])


def projective_dephasing_kraus(p: float) -> np.ndarray:
    """"Projective" unraveling of the dephasing channel (appendix on common
    unravelings): {sqrt(1-p) I, sqrt(p) |0><0|, sqrt(p) |1><1|}."""
    p0 = np.array([[1.0, 0.0], [0.0, 0.0]], dtype=np.complex128)
    p1 = np.array([[0.0, 0.0], [0.0, 1.0]], dtype=np.complex128)
    return np.stack([math.sqrt(1.0 - p) * PAULI_I, math.sqrt(p) * p0, math.sqrt(p) * p1])


def projective_depolarizing_kraus(p: float) -> np.ndarray:
    """"Projective" unraveling of the depolarizing channel (appendix on common
    unravelings): {sqrt(1-p) I, sqrt(p/2) |a><b| for a, b in {0, 1}} (five
    operators, |0><0|, |0><1|, |1><0|, |1><1| in that order)."""
    ops = [math.sqrt(1.0 - p) * PAULI_I]
    for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)):
        e = np.zeros((2, 2), dtype=np.complex128)
        e[a, b] = 1.0
        ops.append(math.sqrt(0.5 * p) * e)
    return np.stack(ops)


def compose_kraus(second: np.ndarray, first: np.ndarray) -> np.ndarray:
    """Kraus set of the channel 'first, then second': {S_a F_b}."""
    return np.stack([s @ f for s in second for f in first])


def rzz(theta: float) -> np.ndarray:
    """exp(-i theta/2 Z(x)Z) as a 4x4 matrix."""
    d = np.exp(-0.5j * theta * np.array([1, -1, -1, 1]))
    return np.diag(d).astype(np.complex128)


def rx(phi: float) -> np.ndarray:
    """exp(-i phi/2 X)."""
    c, s = math.cos(0.5 * phi), math.sin(0.5 * phi)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def brickwork_bonds(n: int, layer_index: int) -> np.ndarray:
    """Left qubits of the gates of a brickwork layer.  Even layers act on bonds
    (0,1),(2,3),...; odd layers on (1,2),(3,4),....  Even layers are listed in
    ascending order and odd layers in descending order (a zig-zag sweep); gates
    of one layer act on disjoint pairs, so the order does not change the
    channel, and both simulators apply the gates in the listed order."""
    start = layer_index % 2
    q = np.arange(start, n - 1, 2, dtype=np.int32)
    return q if layer_index % 2 == 0 else q[::-1].copy()


def random_brickwork(n: int, depth: int, kraus: np.ndarray, seed: int,
                     coin_p: float = 1.0) -> Circuit:
    """Brickwork circuit with Haar-random two-qubit gates (one circuit shared by
    every trajectory)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4C45, n, depth]))
    layers = []
    for l in range(depth):
        q = brickwork_bonds(n, l)
        g = np.stack([haar_unitary(rng, 4) for _ in q]) if len(q) else np.zeros((0, 4, 4), np.complex128)
        layers.append(Layer(q, g, np.asarray(kraus, np.complex128), coin_p))
    return Circuit(n, layers)


def kicked_ising(n: int, depth: int, kraus: np.ndarray, coin_p: float, seed: int) -> Circuit:
    """Kicked-Ising type circuit: per period RZZ(pi/4 + N(0,0.05)) on all bonds
    (even sub-layer, then odd sub-layer, each RZZ followed by the noise), then
    RX(U[0,pi]) on every qubit.  A period's RX layer is folded into the next
    period's even-bond RZZ gates (exact, no noise acts in between); the last
    period's RX layer becomes a final noiseless layer of RX (x) RX gates on the
    even bonds (n even)."""
    assert n % 2 == 0
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4B49, n, depth]))
    layers = []
    pending_rx: Optional[np.ndarray] = None
    for t in range(depth):
        for sub in range(2):
            q = brickwork_bonds(n, sub)
            gates = []
            for qq in q:
                g = rzz(math.pi / 4 + 0.05 * rng.standard_normal())
                if sub == 0 and pending_rx is not None:
                    g = g @ np.kron(pending_rx[qq], pending_rx[qq + 1])
                gates.append(g)
            layers.append(Layer(q, np.stack(gates), np.asarray(kraus, np.complex128), coin_p))
        pending_rx = np.stack([rx(rng.uniform(0.0, math.pi)) for _ in range(n)])
    q = brickwork_bonds(n, 0)
    layers.append(Layer(q, np.stack([np.kron(pending_rx[a], pending_rx[a + 1]) for a in q]),
                        np.asarray(kraus, np.complex128), 0.0))
    return Circuit(n, layers)


# --- The five workloads ----------------------------------------------------

def workload_small_exact(seed: int = 0) -> dict:
    """n=8, depth 8 Haar brickwork, single-qubit depolarizing p=0.02 on both
    gated qubits after each gate, chi_max=16 (exact), 256 trajectories."""
    circ = random_brickwork(8, 8, depolarizing_kraus(0.02), seed)
    return dict(circuit=circ, chi_max=16, n_traj=256, seed=seed)


def workload_ad_dephasing(seed: int = 0, n_traj: int = 4096) -> dict:
    """n=32, depth 20 Haar brickwork; amplitude damping gamma=0.01 followed by
    dephasing p=0.01 composed into one four-operator channel; chi_max=64."""
    kr = compose_kraus(dephasing_kraus(0.01), amplitude_damping_kraus(0.01))
    circ = random_brickwork(32, 20, kr, seed)
    return dict(circuit=circ, chi_max=64, n_traj=n_traj, seed=seed)


def workload_uneven(seed: int = 0, n_traj: int = 16384, depth: int = 32) -> dict:
    """16384 trajectories with n drawn uniformly from {24, 48, 64}, depth 32 Haar
    brickwork, two-qubit depolarizing p=0.005 after each gate, chi_max=128.
    Returns one circuit per system size and the per-trajectory size labels."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x554E]))
    sizes = np.array([24, 48, 64])
    n_of_traj = sizes[rng.integers(0, 3, size=n_traj)]
    circuits = {int(n): random_brickwork(int(n), depth, depolarizing_kraus(1.0), seed, coin_p=0.005)
                for n in sizes}
    return dict(circuits=circuits, n_of_traj=n_of_traj, chi_max=128, seed=seed)


def workload_adjoint(seed: int = 0, batch: int = 8192, chi: int = 64,
                     dtype=np.complex128) -> dict:
    """Independent local unraveling problems: normalized complex Gaussian two-site
    tensors (chi, 2, 2, chi), depolarizing p ~ U[0.005, 0.05], Gaussian Hermitian
    H (entries N(0,1) + i N(0,1), symmetrized)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4144, batch, chi]))
    th = rng.standard_normal((batch, chi, 2, 2, chi)) + 1j * rng.standard_normal((batch, chi, 2, 2, chi))
    th /= np.sqrt(np.sum(np.abs(th) ** 2, axis=(1, 2, 3, 4), keepdims=True))
    p = rng.uniform(0.005, 0.05, size=batch)
    a = rng.standard_normal((batch, 4, 4)) + 1j * rng.standard_normal((batch, 4, 4))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    return dict(theta=th.astype(dtype), p=p, H=h)


def workload_kicked_ising(seed: int = 0, n_traj: int = 2048) -> dict:
    """n=128, depth 40 kicked-Ising circuit, two-qubit depolarizing p=0.01 after
    each RZZ, chi_max=512."""
    circ = kicked_ising(128, 40, depolarizing_kraus(1.0), 0.01, seed)
    return dict(circuit=circ, chi_max=512, n_traj=n_traj, seed=seed)
