"""Oracle: Monte-Carlo trajectories with the optimal unraveling, plus exact
density-matrix evolution.

* ``dense_trajectory``  state-vector trajectory (n <= ~20): per gate the
  unitary, then for slot t in (q, q+1) the channel unraveling subprocedure of
  Alg. 1 with the Kraus set chosen by ``optimal_unraveling`` (Sec. IV.B).
* ``mps_trajectory``    the same on an MPS in mixed-canonical form with SVD
  split and truncation to chi_max (Sec. II "Matrix product states",
  Sec. IV.A layering option "local": Trunc o N(x)N o U per gate), with the
  per-layer truncation error eps_trunc = sqrt(2 sum_k eps_k) and the trajectory
  bound sum_l 4 eps_trunc (App. B, "Errors based on MPS truncations").
* ``density_evolution`` rho <- G rho G^dagger, then the channel on q and q+1
  (exact reference, n <= ~10).

Qubit 0 is the most significant bit of a state-vector index.  The uniform for
slot s of global gate g in trajectory i is philox.uniform(seed, i, g, s); the
branch is the first i with u * sum(p) < cumsum(p)_i (Alg. 1 "sample").
A gate whose layer has coin_p < 1 first draws u_c at slot 2 and applies its
noise only when u_c < coin_p.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

from . import philox
from .unravel import haar_optimal, optimal_unraveling, unraveling_entropy, von_neumann_entropy

Z = np.diag([1.0, -1.0]).astype(np.complex128)


@dataclasses.dataclass
class TrajectoryRecord:
    branch: List[int]          # per noise site (gate-major, slot-minor); -1 = no noise
    p_branch: List[float]      # probability of the chosen branch
    e_av: List[float]          # E_av of the chosen unraveling at that site
    discarded: List[float]     # per gate discarded weight (MPS only)
    eps_bound: float = 0.0     # per-trajectory error bound (MPS only)
    eps_layers: List[float] = dataclasses.field(default_factory=list)  # per layer 4 sqrt(2 sum eps) (MPS only)
    # per truncating split, the relative gap (w_{chi'} - w_{chi'+1}) / w_1 of
    # the squared Schmidt values at the cut (MPS only): the conditioning of
    # the kept subspace, which moves by about (perturbation / gap)
    cut_gaps: List[float] = dataclasses.field(default_factory=list)
    # worst-case change of the state when a split is computed from the Gram
    # matrix with unit roundoff u instead of by SVD, summed over the splits:
    # {u: bound} for u = 2^-53 and 2^-24 (MPS only; see gram_route_bound)
    gram_bound: dict = dataclasses.field(default_factory=dict)
    z: np.ndarray = None       # <Z_i>
    zz: np.ndarray = None      # <Z_i Z_{i+1}>
    s_half: float = 0.0        # entropy of bond n/2 (nats)
    state: np.ndarray = None   # final dense state (dense path, or MPS contracted when small)


def sample_index(p: np.ndarray, u: float) -> int:
    """First index with u * sum(p) < cumsum(p)."""
    cs = np.cumsum(p)
    thr = u * cs[-1]
    for i, c in enumerate(cs):
        if thr < c:
            return i
    return len(p) - 1


def _choose_kraus(rho_t, kraus, mode):
    """Kraus set sampled at a noise site: as given, the state's locally
    entanglement-optimal remix (Sec. IV.B), or the fixed Haar-optimal remix
    (the Bell state's optimal set, Sec. V.B)."""
    if mode == "given":
        return np.asarray(kraus, np.complex128)
    if mode == "haar_optimal":
        return haar_optimal(kraus)
    if mode != "optimal":
        raise ValueError(f"unknown unraveling mode {mode!r}")
    return optimal_unraveling(rho_t, kraus)[0]


# --- dense state vector ------------------------------------------------------

def apply_2q(psi, g, q, n):
    t = psi.reshape(2 ** q, 4, 2 ** (n - q - 2))
    return np.einsum('ab,xby->xay', g, t).reshape(-1)


def apply_1q(psi, k, q, n):
    t = psi.reshape(2 ** q, 2, 2 ** (n - q - 1))
    return np.einsum('ab,xby->xay', k, t).reshape(-1)


def reduced_1q(psi, q, n):
    t = psi.reshape(2 ** q, 2, 2 ** (n - q - 1))
    return np.einsum('xay,xby->ab', t, t.conj())


def dense_observables(psi, n):
    prob = (np.abs(psi) ** 2).reshape([2] * n)
    z = np.zeros(n)
    zz = np.zeros(n - 1)
    for i in range(n):
        pm = np.moveaxis(prob, i, 0).reshape(2, -1).sum(axis=1)
        z[i] = pm[0] - pm[1]
    for i in range(n - 1):
        m = np.moveaxis(prob, (i, i + 1), (0, 1)).reshape(2, 2, -1).sum(axis=2)
        zz[i] = m[0, 0] - m[0, 1] - m[1, 0] + m[1, 1]
    h = n // 2
    s = _svd(psi.reshape(2 ** h, -1), compute_uv=False)
    lam = s ** 2 / np.sum(s ** 2)
    lam = lam[lam > 0]
    return z, zz, float(-np.sum(lam * np.log(lam)))


def dense_trajectory(circuit, traj: int, seed: int, mode: str = "optimal",
                     layering: str = "local") -> TrajectoryRecord:
    """State-vector trajectory (Alg. 1).  layering "local": each gate is
    followed by the noise on its two qubits, (Trunc N^{(x)2} U)^{(x) n/2};
    "global": all gates of the layer, then the noise on every gated qubit in
    gate order, Trunc^{(x) n-1} N^{(x) n} U^{(x) n/2} (Sec. IV.A, layering
    options).  Both draw the same Philox counters (gate, slot)."""
    if layering not in ("local", "global"):
        raise ValueError(f"unknown layering {layering!r}")
    n = circuit.n_qubits
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    rec = TrajectoryRecord([], [], [], [])
    g_glob = 0
    for layer in circuit.layers:
        if layering == "global":
            for q, gate in zip(layer.left_qubits, layer.gates):
                psi = apply_2q(psi, gate, int(q), n)
        for q, gate in zip(layer.left_qubits, layer.gates):
            q = int(q)
            if layering == "local":
                psi = apply_2q(psi, gate, q, n)
            active = True
            if layer.coin_p < 1.0:
                active = philox.uniform(seed, traj, g_glob, 2) < layer.coin_p
            for slot, t in enumerate((q, q + 1)):
                if not active:
                    rec.branch.append(-1); rec.p_branch.append(1.0); rec.e_av.append(0.0)
                    continue
                rho_t = reduced_1q(psi, t, n)
                kp = _choose_kraus(rho_t, layer.kraus, mode)
                p = np.array([np.vdot(v, v).real for v in (apply_1q(psi, k, t, n) for k in kp)])
                i = sample_index(p, philox.uniform(seed, traj, g_glob, slot))
                rec.branch.append(i); rec.p_branch.append(p[i] / p.sum())
                rec.e_av.append(unraveling_entropy(kp, rho_t / np.trace(rho_t).real))
                psi = apply_1q(psi, kp[i], t, n) / math.sqrt(p[i])
            g_glob += 1
    rec.z, rec.zz, rec.s_half = dense_observables(psi, n)
    rec.state = psi
    return rec


# --- exact density matrix ----------------------------------------------------

def density_evolution(circuit) -> np.ndarray:
    n = circuit.n_qubits
    d = 2 ** n
    rho = np.zeros((d, d), dtype=np.complex128)
    rho[0, 0] = 1.0

    def op2(g, q):
        return np.kron(np.kron(np.eye(2 ** q), g), np.eye(2 ** (n - q - 2)))

    def op1(k, q):
        return np.kron(np.kron(np.eye(2 ** q), k), np.eye(2 ** (n - q - 1)))

    for layer in circuit.layers:
        for q, gate in zip(layer.left_qubits, layer.gates):
            q = int(q)
            g = op2(gate, q)
            rho = g @ rho @ g.conj().T
            noisy = rho
            for t in (q, q + 1):
                ks = [op1(k, t) for k in layer.kraus]
                noisy = sum(k @ noisy @ k.conj().T for k in ks)
            rho = layer.coin_p * noisy + (1.0 - layer.coin_p) * rho
    return rho


def density_observables(rho, n):
    z = np.zeros(n)
    zz = np.zeros(n - 1)
    diag = np.diag(rho).real.reshape([2] * n)
    for i in range(n):
        pm = np.moveaxis(diag, i, 0).reshape(2, -1).sum(axis=1)
        z[i] = pm[0] - pm[1]
    for i in range(n - 1):
        m = np.moveaxis(diag, (i, i + 1), (0, 1)).reshape(2, 2, -1).sum(axis=2)
        zz[i] = m[0, 0] - m[0, 1] - m[1, 0] + m[1, 1]
    return z, zz


# --- MPS trajectory -----------------------------------------------------------

class MPS:
    """Site tensors A[k] of shape (d_k, 2, d_{k+1}) (Eq. def_MPS) kept in
    mixed-canonical form: sites left of ``center`` left-orthonormal, sites right
    of it right-orthonormal."""

    def __init__(self, n):
        self.n = n
        self.a = [np.ones((1, 2, 1), dtype=np.complex128) * np.array([1, 0]).reshape(1, 2, 1)
                  for _ in range(n)]
        self.center = 0

    def move_center(self, target):
        while self.center < target:
            k = self.center
            dl, _, dr = self.a[k].shape
            q, r = np.linalg.qr(self.a[k].reshape(dl * 2, dr))
            self.a[k] = q.reshape(dl, 2, -1)
            self.a[k + 1] = np.einsum('ab,bsc->asc', r, self.a[k + 1])
            self.center += 1
        while self.center > target:
            k = self.center
            dl, _, dr = self.a[k].shape
            q, r = np.linalg.qr(self.a[k].reshape(dl, 2 * dr).T)   # A^T = Q R
            self.a[k] = q.T.reshape(-1, 2, dr)
            self.a[k - 1] = np.einsum('asb,cb->asc', self.a[k - 1], r)
            self.center -= 1

    def to_dense(self):
        psi = self.a[0].reshape(2, -1)
        for k in range(1, self.n):
            psi = np.einsum('xa,asb->xsb', psi, self.a[k]).reshape(-1, self.a[k].shape[2])
        return psi.reshape(-1)

    def observables(self):
        n = self.n
        z = np.zeros(n)
        zz = np.zeros(n - 1)
        s_half = 0.0
        self.move_center(0)
        for k in range(n):
            self.move_center(k)
            a = self.a[k]
            z[k] = np.sum(np.abs(a[:, 0, :]) ** 2) - np.sum(np.abs(a[:, 1, :]) ** 2)
            if k + 1 < n:
                th = np.einsum('asm,mtb->astb', a, self.a[k + 1])
                w = np.sum(np.abs(th) ** 2, axis=(0, 3))
                zz[k] = w[0, 0] - w[0, 1] - w[1, 0] + w[1, 1]
            if k == n // 2 - 1:
                dl, _, dr = a.shape
                s = _svd(a.reshape(dl * 2, dr), compute_uv=False)
                lam = s ** 2 / np.sum(s ** 2)
                lam = lam[lam > 0]
                s_half = float(-np.sum(lam * np.log(lam)))
        return z, zz, s_half


def _pair_tensor(m, q, gate=None):
    """Two-site tensor of sites (q, q+1) with the centre moved onto the pair,
    the gate (4x4 on the two physical indices) applied when given."""
    if m.center < q:
        m.move_center(q)
    elif m.center > q + 1:
        m.move_center(q + 1)
    a, b = m.a[q], m.a[q + 1]
    th = np.einsum('asm,mtb->astb', a, b)
    if gate is not None:
        th = np.einsum('uv,avb->aub', gate, th.reshape(a.shape[0], 4, b.shape[2]))
    return th.reshape(a.shape[0], 2, 2, b.shape[2])


def _svd(a, **kw):
    """numpy's SVD (LAPACK gesdd, divide and conquer).  On gesdd's rare
    non-convergence, the same decomposition by LAPACK gesvd (QR iteration)
    through scipy."""
    try:
        return np.linalg.svd(a, **kw)
    except np.linalg.LinAlgError:
        import scipy.linalg as sla
        return sla.svd(a, lapack_driver="gesvd", **kw)


GRAM_UNITS = (2.0 ** -53, 2.0 ** -24)


def gram_route_bound(w, keep, ng, u):
    """Worst-case norm of the change of a truncated split (Eq.
    MPS_truncation_error keeps the top chi' squared Schmidt values w) when
    the split comes from a Hermitian eigensolve of the n_g x n_g Gram matrix
    in arithmetic of unit roundoff u instead of from the SVD.  The Gram
    route perturbs the squared values by about tau = n_g u w_1, so (i) kept
    values below tau are not resolved at all: their vectors may turn
    completely, moving the state by up to sqrt(their weight); (ii) where the
    cut itself lies above tau, the kept subspace turns by at most tau / (w_chi'
    - w_chi'+1) (Davis-Kahan), moving the state by that times sqrt(w_chi').
    Weights are relative to sum w."""
    r = np.asarray(w, dtype=float) / float(np.sum(w))
    tau = ng * u * r[0]
    kept = r[:keep]
    b = math.sqrt(float(np.sum(kept[kept < tau])))
    if keep < len(r) and r[keep - 1] >= tau:
        gap = r[keep - 1] - r[keep]
        b += math.sqrt(r[keep - 1]) * min(1.0, tau / gap if gap > 0 else 1.0)
    return b


def _split(m, q, th, cap, cutoff, rec):
    """SVD split of the pair (Eq. MPS_truncation_error): keep
    chi' = min(cap, #{s_k^2 > cutoff * sum s^2}) values, renormalize, centre on
    q+1; returns the discarded weight."""
    dl, dr = th.shape[0], th.shape[3]
    u, s, vh = _svd(th.reshape(dl * 2, 2 * dr), full_matrices=False)
    w = s ** 2
    tot = np.sum(w)
    keep = int(min(cap, np.sum(w > cutoff * tot)))
    keep = max(keep, 1)
    eps = float(np.sum(w[keep:]) / tot)
    rec.discarded.append(eps)
    if keep < len(w):
        rec.cut_gaps.append(float((w[keep - 1] - w[keep]) / w[0]))
    for unit in GRAM_UNITS:
        rec.gram_bound[unit] = rec.gram_bound.get(unit, 0.0) + gram_route_bound(w, keep, 2 * max(dl, dr), unit)
    kept = math.sqrt(np.sum(w[:keep]))
    m.a[q] = u[:, :keep].reshape(dl, 2, keep)
    m.a[q + 1] = (s[:keep, None] * vh[:keep, :] / kept).reshape(keep, 2, dr)
    m.center = q + 1
    return eps


def mps_trajectory(circuit, traj: int, seed: int, chi_max: int, cutoff: float = 1e-20,
                   mode: str = "optimal", eps_max: float = 4.0, keep_dense: bool = False,
                   layer_callback=None, layering: str = "local"):
    """One MPS trajectory.  layering "local": after gate (q, q+1) and its
    noise, the two-site tensor is split by SVD keeping chi' = min(chi_max,
    #{s_k^2 > cutoff * sum s^2}) values.  "global" (Sec. IV.A, layering
    options): all gates of the layer are applied and split without the chi_max
    cap, then the noise acts on every gated pair in gate order (re-split
    without the cap), then every bond is truncated to chi_max by a left-to-right
    sweep of two-site splits.  The discarded weights of a layer are summed into
    its eps (Thm. 1) and the state is renormalized after each split.
    layer_callback(l), if given, is called after layer l (used to time the
    oracle per layer)."""
    if layering not in ("local", "global"):
        raise ValueError(f"unknown layering {layering!r}")
    n = circuit.n_qubits
    m = MPS(n)
    rec = TrajectoryRecord([], [], [], [])
    g_glob = 0
    eps_tot = 0.0
    uncapped = 1 << 30
    for layer in circuit.layers:
        eps_layer = 0.0
        if layering == "global":
            for q, gate in zip(layer.left_qubits, layer.gates):
                q = int(q)
                eps_layer += _split(m, q, _pair_tensor(m, q, gate), uncapped, cutoff, rec)
        for q, gate in zip(layer.left_qubits, layer.gates):
            q = int(q)
            th = _pair_tensor(m, q, gate if layering == "local" else None)
            active = True
            if layer.coin_p < 1.0:
                active = philox.uniform(seed, traj, g_glob, 2) < layer.coin_p
            for slot in range(2):
                if not active:
                    rec.branch.append(-1); rec.p_branch.append(1.0); rec.e_av.append(0.0)
                    continue
                if slot == 0:
                    rho_t = np.einsum('asxb,atxb->st', th, th.conj())
                else:
                    rho_t = np.einsum('axsb,axtb->st', th, th.conj())
                kp = _choose_kraus(rho_t, layer.kraus, mode)
                p = np.array([np.trace(k @ rho_t @ k.conj().T).real for k in kp])
                i = sample_index(p, philox.uniform(seed, traj, g_glob, slot))
                rec.branch.append(i); rec.p_branch.append(p[i] / p.sum())
                rec.e_av.append(unraveling_entropy(kp, rho_t / np.trace(rho_t).real))
                op = kp[i] / math.sqrt(p[i])
                if slot == 0:
                    th = np.einsum('us,asxb->auxb', op, th)
                else:
                    th = np.einsum('us,axsb->axub', op, th)
            eps_layer += _split(m, q, th, chi_max if layering == "local" else uncapped, cutoff, rec)
            g_glob += 1
        if layering == "global":
            for k in range(n - 1):
                eps_layer += _split(m, k, _pair_tensor(m, k), chi_max, cutoff, rec)
        eps_tot += 4.0 * math.sqrt(2.0 * eps_layer)
        rec.eps_layers.append(4.0 * math.sqrt(2.0 * eps_layer))
        if layer_callback is not None:
            layer_callback(len(rec.discarded))
    rec.eps_bound = eps_tot if eps_tot <= eps_max - 2.0 else eps_max
    rec.z, rec.zz, rec.s_half = m.observables()
    if keep_dense:
        rec.state = m.to_dense()
    return rec


def trajectory_statistics(values: np.ndarray):
    """Mean and standard error over trajectories (axis 0)."""
    values = np.asarray(values, dtype=np.float64)
    nt = values.shape[0]
    mean = values.mean(axis=0)
    se = values.std(axis=0, ddof=1) / math.sqrt(nt) if nt > 1 else np.zeros_like(mean)
    return mean, se


def error_estimate(eps_bounds: np.ndarray, eps_max: float = 4.0, delta: float = 0.05):
    """(eps_hat_N, Hoeffding buffer) of Thm. 1: eps_hat = mean of the
    per-trajectory bounds, buffer = sqrt(eps_max^2 / (2N) ln(1/delta))."""
    nt = len(eps_bounds)
    return float(np.mean(eps_bounds)), math.sqrt(eps_max ** 2 / (2.0 * nt) * math.log(1.0 / delta))


# --- concentration-improved error bound (Sec. III.C; appendix on concentration) ---

def concentration_weight(kind: str, param: float, k: int, n: int) -> float:
    """Weight of a layer k layers before the last one: alpha^k for a channel
    contracting the trace distance by alpha < 1 per layer ("alpha"), or
    min(sqrt(8 n) (1 - p)^k, 1) for local depolarizing noise of rate p by the
    strong data-processing inequality ("depolarizing")."""
    if kind == "alpha":
        return param ** k
    if kind == "depolarizing":
        return min(math.sqrt(8.0 * n) * (1.0 - param) ** k, 1.0)
    raise ValueError(f"unknown weighting {kind!r}")


def concentrated_bound(eps_layers, kind: str, param: float, n: int, eps_max: float = 4.0) -> float:
    """Per-trajectory concentration-improved bound sum_l w(L - l) eps_approx(l)
    over the trajectory's layers l = 1..L, capped like the plain bound
    (kept when <= eps_max - 2, else eps_max)."""
    big_l = len(eps_layers)
    e = sum(concentration_weight(kind, param, big_l - 1 - l, n) * x for l, x in enumerate(eps_layers))
    return e if e <= eps_max - 2.0 else eps_max


# --- output-distribution sampling (Lemma sampling_reduction) -------------------

SAMPLE_COUNTER_BASE = 1 << 62   # Philox gate word of shot s: SAMPLE_COUNTER_BASE + s


def sample_bitstring_dense(psi: np.ndarray, n: int, seed: int, traj: int, shot: int) -> np.ndarray:
    """One computational-basis bitstring from |psi>, qubit 0 first, by
    sequential conditionals: bit k is 0 when u_k (p0 + p1) < p0, with p_s the
    weight of the prefix extended by s and u_k = Philox(seed; traj,
    SAMPLE_COUNTER_BASE + shot, k).  Sampling every trajectory's final state
    this way samples the unraveled mixed state (Lemma sampling_reduction)."""
    t = psi.reshape([2] * n)
    bits = np.zeros(n, dtype=np.uint8)
    for k in range(n):
        w = np.sum(np.abs(t) ** 2, axis=tuple(range(1, t.ndim)))
        u = philox.uniform(seed, traj, SAMPLE_COUNTER_BASE + shot, k)
        b = 0 if u * (w[0] + w[1]) < w[0] else 1
        bits[k] = b
        t = t[b]
    return bits


def bitstring_probability(psi: np.ndarray, n: int, bits) -> float:
    """Product of the sequential conditionals of a bitstring (equals |<x|psi>|^2
    for a normalized state)."""
    t = psi.reshape([2] * n)
    prob = 1.0
    for k in range(n):
        w = np.sum(np.abs(t) ** 2, axis=tuple(range(1, t.ndim)))
        prob *= w[bits[k]] / (w[0] + w[1])
        t = t[bits[k]]
    return prob
