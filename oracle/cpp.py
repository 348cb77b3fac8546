"""ctypes binding of the plain C++17 FP64 oracle (``oracle/mps_oracle.cpp``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  The C++ oracle is the
MPS trajectory of ``oracle.trajectories.mps_trajectory`` (Sec. IV.A layering,
Alg. 1 noise sites with the optimal unraveling of Sec. IV.B / App. F.2, the
SVD split and truncation of Sec. II, the error bound of Thm. 1 / App. B)
restated in C++ with its own Jacobi eigensolver, one-sided Jacobi SVD and
Householder QR, and OpenMP over trajectories.  It is the timed CPU baseline.

``build()`` compiles it with g++ (``-fopenmp``) into ``oracle/_build``; the
tests and the benchmark call ``load()``, which builds on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mps_oracle.cpp")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle_mps.so")

MODES = {"optimal": 0, "given": 1, "haar_optimal": 2}
LAYERINGS = {"local": 0, "global": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fcx-limited-range", "-o", tmp, SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the C++ oracle failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    D, I, I64, U64, P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    lib.oracle_uniform.restype = D
    lib.oracle_uniform.argtypes = [U64, U64, U64, U64]
    lib.oracle_optimal_unraveling.restype = I
    lib.oracle_optimal_unraveling.argtypes = [P, P, I, P, P]
    lib.oracle_batch_create.restype = P
    lib.oracle_batch_create.argtypes = [I, I, P, P, P, P, P, P, I64, I64, U64, I, D, I, I, D]
    lib.oracle_batch_run.restype = I
    lib.oracle_batch_run.argtypes = [P, I, I, I]
    lib.oracle_batch_run_range.restype = I
    lib.oracle_batch_run_range.argtypes = [P, I64, I64, I, I, I]
    lib.oracle_batch_results.restype = I
    lib.oracle_batch_results.argtypes = [P, P, P, P, P, P, P, I]
    lib.oracle_batch_layer.restype = I
    lib.oracle_batch_layer.argtypes = [P]
    lib.oracle_batch_max_bond.restype = I
    lib.oracle_batch_max_bond.argtypes = [P]
    lib.oracle_batch_destroy.restype = None
    lib.oracle_batch_destroy.argtypes = [P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def uniform(seed: int, traj: int, gate: int, slot: int) -> float:
    return load().oracle_uniform(seed, traj, gate, slot)


def optimal_unraveling(rho_a: np.ndarray, kraus: np.ndarray):
    """(kraus_out, W) of the C++ oracle, as ``oracle.unravel.optimal_unraveling``."""
    kraus = np.ascontiguousarray(kraus, dtype=np.complex128)
    r = kraus.shape[0]
    rp = max(r, 4)
    rho = np.ascontiguousarray(rho_a, dtype=np.complex128)
    out = np.zeros((rp, 2, 2), dtype=np.complex128)
    w = np.zeros((rp, rp), dtype=np.complex128)
    got = load().oracle_optimal_unraveling(_ptr(rho), _ptr(kraus), r, _ptr(out), _ptr(w))
    assert got == rp
    return out, w


class Batch:
    """Trajectories traj0 .. traj0 + n_traj - 1 of one circuit, advanced layer
    by layer (``run``) with OpenMP over trajectories."""

    def __init__(self, circuit, traj0: int, n_traj: int, seed: int, chi_max: int, cutoff: float = 1e-20,
                 mode: str = "optimal", layering: str = "local", eps_max: float = 4.0):
        self.lib = load()
        self.n = circuit.n_qubits
        self.n_layers = len(circuit.layers)
        self.n_traj = n_traj
        gb, left, gates, kb, kraus, coin = [0], [], [], [0], [], []
        for layer in circuit.layers:
            lq = [int(q) for q in layer.left_qubits]
            left += lq
            gates += [np.asarray(g, dtype=np.complex128).reshape(4, 4) for g in layer.gates]
            gb.append(gb[-1] + len(lq))
            k = np.asarray(layer.kraus, dtype=np.complex128).reshape(-1, 2, 2)
            kraus.append(k)
            kb.append(kb[-1] + k.shape[0])
            coin.append(float(layer.coin_p))
        self._keep = [np.asarray(gb, np.int32), np.asarray(left if left else [0], np.int32),
                      np.ascontiguousarray(np.stack(gates) if gates else np.zeros((1, 4, 4)), dtype=np.complex128),
                      np.asarray(kb, np.int32),
                      np.ascontiguousarray(np.concatenate(kraus) if kraus else np.zeros((1, 2, 2)),
                                           dtype=np.complex128),
                      np.asarray(coin if coin else [1.0], np.float64)]
        g, l_, ga, k_, kr, c = self._keep
        self.n_gates = int(gb[-1])
        self.h = self.lib.oracle_batch_create(self.n, self.n_layers, _ptr(g), _ptr(l_), _ptr(ga), _ptr(k_),
                                              _ptr(kr), _ptr(c), traj0, n_traj, seed, chi_max, cutoff,
                                              MODES[mode], LAYERINGS[layering], eps_max)
        if not self.h:
            raise ValueError("oracle_batch_create refused its arguments")
        self.layer = 0

    def run(self, l0: int, l1: int, threads: int = 0) -> None:
        if self.lib.oracle_batch_run(self.h, l0, l1, threads) != 0:
            raise ValueError(f"oracle_batch_run({l0}, {l1}) refused (batch at layer {self.layer})")
        self.layer = l1

    def run_range(self, i0: int, i1: int, l0: int, l1: int, threads: int = 0) -> None:
        """Advance trajectories i0 .. i1-1 only (each at layer l0) to layer l1."""
        if self.lib.oracle_batch_run_range(self.h, i0, i1, l0, l1, threads) != 0:
            raise ValueError(f"oracle_batch_run_range({i0}, {i1}, {l0}, {l1}) refused")

    def results(self, threads: int = 0) -> dict:
        n, B = self.n, self.n_traj
        layer = self.lib.oracle_batch_layer(self.h)
        if layer < 0:
            raise ValueError("oracle_batch_results: the trajectories are not at one common layer")
        z = np.zeros((B, n))
        zz = np.zeros((B, n - 1))
        s = np.zeros(B)
        eps = np.zeros(B)
        br = np.zeros((B, 2 * int(self._keep[0][layer])), dtype=np.int32)   # two noise sites per gate run
        gap = np.zeros(B)
        if self.lib.oracle_batch_results(self.h, _ptr(z), _ptr(zz), _ptr(s), _ptr(eps), _ptr(br), _ptr(gap),
                                         threads) != 0:
            raise ValueError("oracle_batch_results: the trajectories are not at one common layer")
        return {"z": z, "zz": zz, "s_half": s, "eps_bound": eps, "branch": br, "min_gap": gap}

    def max_bond(self) -> int:
        return self.lib.oracle_batch_max_bond(self.h)

    def close(self) -> None:
        if self.h:
            self.lib.oracle_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mps_trajectories(circuit, traj0: int, n_traj: int, seed: int, chi_max: int, cutoff: float = 1e-20,
                     mode: str = "optimal", layering: str = "local", eps_max: float = 4.0, threads: int = 0) -> dict:
    """Every trajectory of the circuit, run to the end; dict of per-trajectory
    z, zz, s_half, eps_bound and branch arrays."""
    b = Batch(circuit, traj0, n_traj, seed, chi_max, cutoff, mode, layering, eps_max)
    try:
        b.run(0, b.n_layers, threads)
        return b.results(threads)
    finally:
        b.close()
