"""Oracle: exact Lindbladian evolution of small chains (test infrastructure only;
the library never imports this module).

FP64 numpy/scipy restatement of the superoperator of the appendix on
Trotterized Lindbladian evolutions: the density matrix vectorized as
|rho>> = (rho (x) I)|Omega>, generator

  L = -i (H (x) I - I (x) H^T) + sum_j g_j (c_j (x) c_j^* - 1/2 c_j^dag c_j (x) I
                                            - 1/2 I (x) c_j^T c_j^*),

and rho(t) = exp(L t) |rho(0)>> by a dense matrix exponential (n <= 5).  It also
gives the single-site jump channel exp(L_j dt) as a 4x4 superoperator and its
Choi matrix, from which any Kraus set of the channel can be checked.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def vec(rho: np.ndarray) -> np.ndarray:
    """|rho>> = (rho (x) I)|Omega>: entry (i, j) of rho at index i * d + j."""
    return np.asarray(rho, dtype=np.complex128).reshape(-1)


def unvec(v: np.ndarray, d: int) -> np.ndarray:
    return v.reshape(d, d)


def site_operator(op: np.ndarray, site: int, n: int) -> np.ndarray:
    """op acting on `site` (qubit 0 = most significant) of an n-qubit chain."""
    return np.kron(np.kron(np.eye(2 ** site), op), np.eye(2 ** (n - site - 1)))


def bond_operator(op4: np.ndarray, site: int, n: int) -> np.ndarray:
    """4x4 op on sites (site, site + 1)."""
    return np.kron(np.kron(np.eye(2 ** site), op4), np.eye(2 ** (n - site - 2)))


def superoperator(h: np.ndarray, jumps) -> np.ndarray:
    """The generator L above for Hamiltonian h (d x d) and jump list
    [(gamma, c)] of d x d operators."""
    d = h.shape[0]
    eye = np.eye(d)
    lsup = -1j * (np.kron(h, eye) - np.kron(eye, h.T))
    for g, c in jumps:
        cdc = c.conj().T @ c
        lsup = lsup + g * (np.kron(c, c.conj()) - 0.5 * np.kron(cdc, eye) - 0.5 * np.kron(eye, cdc.T))
    return lsup


def chain_generator(n: int, h2, h1, jumps) -> np.ndarray:
    """L of a chain: h2[i] (4x4) on bond (i, i+1), h1[i] (2x2) on site i,
    jumps [(site, gamma, c)] with 2x2 c."""
    h = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for i in range(n - 1):
        h += bond_operator(h2[i], i, n)
    for i in range(n):
        h += site_operator(h1[i], i, n)
    full = [(g, site_operator(c, s, n)) for s, g, c in jumps]
    return superoperator(h, full)


def evolve(n: int, h2, h1, jumps, t: float, rho0: np.ndarray) -> np.ndarray:
    """rho(t) = exp(L t) rho0 (exact)."""
    lsup = chain_generator(n, h2, h1, jumps)
    return unvec(sla.expm(lsup * t) @ vec(rho0), 2 ** n)


def choi_of_superoperator(s: np.ndarray) -> np.ndarray:
    """Choi matrix sum_{ab} |a><b| (x) N(|a><b|) of a single-qubit channel given
    by its 4x4 superoperator in the convention of vec()."""
    choi = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            e = np.zeros((2, 2), dtype=np.complex128)
            e[a, b] = 1.0
            choi += np.kron(e, unvec(s @ vec(e), 2))
    return choi


def choi_of_kraus(kraus) -> np.ndarray:
    """The same Choi matrix from a Kraus set."""
    choi = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            e = np.zeros((2, 2), dtype=np.complex128)
            e[a, b] = 1.0
            choi += np.kron(e, sum(k @ e @ k.conj().T for k in kraus))
    return choi
