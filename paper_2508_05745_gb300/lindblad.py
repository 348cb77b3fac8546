"""Lindbladian front end: a Trotterized open-system evolution as a noisy
brickwork circuit that `apply_layer` runs (appendix on Trotterized
Lindbladian evolutions; Sec. V.A).

For a chain with nearest-neighbour terms h2[i] on (i, i+1), single-site terms
h1[i] and the same single-site jump processes on every qubit, one time step dt
becomes two layers:

* layer A: gates exp(-i H_{i,i+1} dt) on (0,1), (2,3), ..., followed by the jump
  channel N = exp(L_jump dt) on both qubits of every gate (every qubit, n even);
* layer B: gates exp(-i H_{i,i+1} dt) on (1,2), (3,4), ..., without noise.

H_{i,i+1} = h2[i] + h1[i] (x) I / m_i + I (x) h1[i+1] / m_{i+1}, with m_j the number
of bonds that touch site j (1 at the ends, 2 inside), so that the bond terms sum
to the chain Hamiltonian.  This is a first-order Trotter splitting, like the
appendix's (which places half of the jump channel after each sub-layer; the
library's layers carry one noise channel each and only on gated qubits, which
the end qubits of layer B are not).

The jump channel's Kraus set comes from the eigendecomposition of its Choi
matrix, built from the 4x4 superoperator exp(L_jump dt) of

  L_jump = sum_j g_j (c_j (x) c_j^* - 1/2 c_j^dag c_j (x) I - 1/2 I (x) c_j^T c_j^*)

(vectorization |rho>> = (rho (x) I)|Omega>); the eigenvectors give orthogonal
Kraus operators.  Host-side numpy: circuit construction, not the hot path.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .inputs import Circuit, Layer

PAULI_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PAULI_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PAULI_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
SIGMA_MINUS = np.array([[0, 1], [0, 0]], dtype=np.complex128)   # |0><1|
PROJ_0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)


def jump_superoperator(jumps, dt: float) -> np.ndarray:
    """exp(L_jump dt) (4x4) for jumps [(gamma, c)] acting on one qubit."""
    eye = np.eye(2)
    gen = np.zeros((4, 4), dtype=np.complex128)
    for g, c in jumps:
        c = np.asarray(c, dtype=np.complex128)
        cdc = c.conj().T @ c
        gen += g * (np.kron(c, c.conj()) - 0.5 * np.kron(cdc, eye) - 0.5 * np.kron(eye, cdc.T))
    return sla.expm(gen * dt)


def jump_kraus(jumps, dt: float, tol: float = 1e-14) -> np.ndarray:
    """Orthogonal Kraus set [r, 2, 2] of exp(L_jump dt) from the eigenvectors of
    its Choi matrix J = sum_{ab} |a><b| (x) N(|a><b|); eigenvalues below tol are
    dropped (r <= 4)."""
    sup = jump_superoperator(jumps, dt)
    choi = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            e = np.zeros((2, 2), dtype=np.complex128)
            e[a, b] = 1.0
            choi += np.kron(e, (sup @ e.reshape(-1)).reshape(2, 2))
    lam, vecs = np.linalg.eigh(0.5 * (choi + choi.conj().T))
    ops = []
    for i in np.argsort(lam)[::-1]:
        if lam[i] <= tol:
            continue
        v = vecs[:, i] * np.sqrt(lam[i])
        # |K>> = sum_a |a> (x) K|a>, i.e. v[2 a + c] = K[c, a]
        ops.append(v.reshape(2, 2).T)
    return np.stack(ops)


def bond_hamiltonians(n: int, h2, h1):
    """H_{i,i+1} for i = 0..n-2 with each site term shared among the bonds that
    touch it."""
    h2 = [np.asarray(h2, np.complex128)] * (n - 1) if np.ndim(h2) == 2 else [np.asarray(x, np.complex128) for x in h2]
    h1 = [np.asarray(h1, np.complex128)] * n if np.ndim(h1) == 2 else [np.asarray(x, np.complex128) for x in h1]
    m = [1 if i in (0, n - 1) else 2 for i in range(n)]
    eye = np.eye(2)
    return [h2[i] + np.kron(h1[i], eye) / m[i] + np.kron(eye, h1[i + 1]) / m[i + 1] for i in range(n - 1)]


def trotter_circuit(n: int, h2, h1, jumps, dt: float, steps: int) -> Circuit:
    """Noisy brickwork circuit of `steps` first-order Trotter steps of length dt
    (two layers each, see the module docstring).  n must be even so that layer
    A reaches every qubit.  h2: one 4x4 or n-1 of them; h1: one 2x2 or n of
    them; jumps: [(gamma, c)] on every qubit."""
    if n < 2 or n % 2:
        raise ValueError("the Lindblad front end needs an even number of qubits")
    hb = bond_hamiltonians(n, h2, h1)
    gates = [sla.expm(-1j * h * dt) for h in hb]
    kraus = jump_kraus(jumps, dt)
    ident = np.eye(2, dtype=np.complex128)[None]
    qa = np.arange(0, n - 1, 2, dtype=np.int32)
    qb = np.arange(1, n - 1, 2, dtype=np.int32)
    layers = []
    for _ in range(steps):
        layers.append(Layer(qa, np.stack([gates[q] for q in qa]), kraus, 1.0))
        if len(qb):
            layers.append(Layer(qb, np.stack([gates[q] for q in qb]), ident, 0.0))
    return Circuit(n, layers)


def heisenberg_amplitude_damping(n: int = 16, gamma: float = 0.002, dt: float = 0.1, steps: int = 60) -> Circuit:
    """The Hamiltonian of the paper's fixed-unraveling comparison (Sec. VI.A):
    H = sum_i Y_i Y_{i+1} + 0.35 X_i + 0.35 Y_i + 0.5 Z_i, with amplitude-damping
    jumps c = |0><1| of rate gamma on every qubit."""
    h1 = 0.35 * PAULI_X + 0.35 * PAULI_Y + 0.5 * PAULI_Z
    return trotter_circuit(n, np.kron(PAULI_Y, PAULI_Y), h1, [(gamma, SIGMA_MINUS)], dt, steps)


def random_lindbladian(n: int, seed: int, gamma: float = 0.01, dt: float = 0.1, steps: int = 20) -> Circuit:
    """A random Lindbladian (Sec. VI.A, averages over random Hamiltonians):
    Gaussian Hermitian bond and site terms (GUE-like, unit scale) and one
    complex Gaussian jump operator shared by all qubits, normalized to unit
    operator norm, of rate gamma; seeded."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4C49, n]))

    def herm(d):
        a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        return 0.5 * (a + a.conj().T)

    h2 = [herm(4) for _ in range(n - 1)]
    h1 = [herm(2) for _ in range(n)]
    c = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    c /= np.linalg.norm(c, 2)
    return trotter_circuit(n, h2, h1, [(gamma, c)], dt, steps)
