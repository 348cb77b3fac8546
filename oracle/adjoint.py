"""Oracle: expected branch entanglement as a function of the Kraus-mixing unitary.

For a target qubit with reduced state rho_A (from a normalized two-site tensor
Theta[a, s1, s2, b], target = s1) and a Kraus set {K_j}, the unitary
U = exp(iH) remixes the set as K'_k = sum_j U[j, k] K_j (Eq. unitarity_kraus).
The cost is the ensemble-averaged target-vs-rest entropy of the induced
ensemble (Eq. def:ensemble-averaged_entanglement):

    E(H) = sum_k p_k S(sigma_k / p_k),  sigma_k = K'_k rho_A K'_k^dagger,
    p_k = Tr sigma_k.

Its minimum over H is E_oF of the effective two-qubit state (Thm. 2).  The
gradient is taken with respect to the Frobenius inner product on Hermitian
matrices: dE = Re Tr(Gamma^dagger dH), Gamma Hermitian.  The FP64 reference
gradient here is central finite differences over the 16 real parameters of H.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .unravel import unraveling_entropy


def reduced_target(theta: np.ndarray) -> np.ndarray:
    """rho_A[s, t] = sum_{a, s2, b} Theta[a, s, s2, b] Theta*[a, t, s2, b]."""
    th = np.asarray(theta, dtype=np.complex128)
    return np.einsum('asxb,atxb->st', th, th.conj())


def remix(h: np.ndarray, kraus: np.ndarray) -> np.ndarray:
    u = sla.expm(1j * np.asarray(h, dtype=np.complex128))
    return np.einsum('jk,jab->kab', u, np.asarray(kraus, dtype=np.complex128))


def expected_entropy(h: np.ndarray, rho_a: np.ndarray, kraus: np.ndarray) -> float:
    return unraveling_entropy(remix(h, kraus), rho_a)


def hermitian_basis():
    """The 16 real directions of Hermitian 4x4 matrices: E_jj, E_jk + E_kj and
    i (E_jk - E_kj) for j < k, with the weights that turn partial derivatives
    into the Frobenius gradient (1 for diagonal, 1/2 for off-diagonal)."""
    out = []
    for j in range(4):
        e = np.zeros((4, 4), dtype=np.complex128)
        e[j, j] = 1.0
        out.append((e, 1.0, (j, j, 'd')))
    for j in range(4):
        for k in range(j + 1, 4):
            e = np.zeros((4, 4), dtype=np.complex128)
            e[j, k] = e[k, j] = 1.0
            out.append((e, 0.5, (j, k, 're')))
            e = np.zeros((4, 4), dtype=np.complex128)
            e[j, k] = 1j
            e[k, j] = -1j
            out.append((e, 0.5, (j, k, 'im')))
    return out


def fd_gradient(h: np.ndarray, rho_a: np.ndarray, kraus: np.ndarray, step: float = 1e-6) -> np.ndarray:
    """Central finite differences (FP64) assembled into the Hermitian gradient."""
    g = np.zeros((4, 4), dtype=np.complex128)
    for e, w, (j, k, kind) in hermitian_basis():
        d = (expected_entropy(h + step * e, rho_a, kraus)
             - expected_entropy(h - step * e, rho_a, kraus)) / (2.0 * step)
        if kind == 'd':
            g[j, j] = d
        elif kind == 're':
            g[j, k] += w * d
            g[k, j] += w * d
        else:
            g[j, k] += 1j * w * d
            g[k, j] -= 1j * w * d
    return g


def gradient_descent(h0, rho_a, kraus, steps: int = 50, lr: float = 0.5):
    """Gradient descent H <- H - alpha * Gamma with FD gradients and a
    backtracking step size (oracle of the on-device optimization loop).

    The step size starts at lr; at every step it is halved until the cost
    decreases by at least 1e-4 * alpha * ||Gamma||_F^2 (Armijo's sufficient
    decrease), the step is skipped if alpha falls below 1e-12, and the next
    step starts from twice the final alpha (at most 1e4).  Returns (H, the
    cost after each step)."""
    h = np.array(h0, dtype=np.complex128)
    e = expected_entropy(h, rho_a, kraus)
    alpha = lr
    costs = []
    for _ in range(steps):
        g = fd_gradient(h, rho_a, kraus)
        gg = float(np.sum(np.abs(g) ** 2))
        while True:
            h_try = h - alpha * g
            e_try = expected_entropy(h_try, rho_a, kraus)
            if e_try <= e - 1e-4 * alpha * gg:
                h, e = h_try, e_try
                break
            alpha *= 0.5
            if alpha < 1e-12:
                break
        costs.append(e)
        alpha = min(2.0 * alpha, 1e4)
    return h, np.array(costs)


def u_theta_phi(theta: float, phi: float) -> np.ndarray:
    """Two-parameter real 4x4 unitary of Eq. U_phi_theta."""
    ct, st, cp, sp = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    return np.array([[ct * cp, ct * sp, st * cp, st * sp],
                     [-ct * sp, ct * cp, -st * sp, st * cp],
                     [-st * cp, -st * sp, ct * cp, ct * sp],
                     [st * sp, -st * cp, -ct * sp, ct * cp]], dtype=np.complex128)


def grid_search(rho_a, kraus, n_grid: int = 64):
    """Brute-force minimum of E over the U(theta, phi) family on an n x n grid."""
    best = (np.inf, 0.0, 0.0)
    kraus = np.asarray(kraus, dtype=np.complex128)
    for th in np.linspace(0.0, math.pi, n_grid, endpoint=False):
        for ph in np.linspace(0.0, math.pi, n_grid, endpoint=False):
            u = u_theta_phi(th, ph)
            e = unraveling_entropy(np.einsum('jk,jab->kab', u, kraus), rho_a)
            if e < best[0]:
                best = (e, th, ph)
    return best
