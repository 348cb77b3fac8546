"""Oracle: entanglement measures and the locally entanglement-optimal unraveling.

FP64 numpy/scipy restatement of Sec. IV.B and App. E-F.  Entropies are in nats
(natural logarithm); the paper writes log2 in App. F and "log" in Sec. II, and
the optimum does not depend on the base.

Conventions
-----------
* Two-qubit vectors are 4-vectors with index 2*t + k, the first factor t being
  the noisy target qubit and the second k the effective partner qubit of
  Sec. IV.B.2.
* Decomposition matrices (App. E): columns are sub-normalized ensemble members,
  rho = w w^dagger.
* Kraus remixing (Eq. unitarity_kraus): K'_k = sum_j W[j, k] K_j.

Canonical choices.  The optimal decomposition is not unique: Takagi vectors
carry signs (and, for equal Takagi values, a real orthogonal mixing; for zero
Takagi values a unitary one), eigenvectors of Re M carry signs (and rotations
inside degenerate eigenspaces), and each choice is optimal but gives different
branch weights.  Depolarizing noise makes such degeneracies structural (three
equal Takagi values and a degenerate pair of Re M for every state; full
depolarization makes all four Takagi values equal).  The oracle and the GPU
library follow the same written rules, so per-trajectory results coincide:
  R1  rho_A eigenpairs are ordered by descending eigenvalue and each
      eigenvector's phase makes <REF2|u_k> real and positive; a degenerate
      rho_A (gap <= DEG_TOL) uses the computational basis;
  R2  reference Gram-Schmidt (RGS): a block of ensemble members A (columns)
      with a real orthogonal freedom A -> A O is replaced by A B, where the
      columns of B are obtained by Gram-Schmidt on the gradients
      g = Re(A^dagger r) of the reference vectors r in REF4 (in order);
      a block with a unitary freedom uses g = A^dagger r and complex
      Gram-Schmidt.  B depends only on the span, not on the basis an
      eigensolver returned;
  R3  RGS is applied to the Takagi vectors x (after Step 1) per block of equal
      Takagi values (real version) and to the block of zero Takagi values
      inside the rank of rho (unitary version), and, in the entangled case,
      to a = y Q per cluster of equal eigenvalues of Re M (real version);
      single columns get their sign (or phase) this way too;
  R4  singular values of phi below RANK_TOL * s_max are treated as zero and
      their columns of v set to zero; Takagi is applied to the leading block;
      Takagi values below ZERO_TOL * s_max are zero, equal values are those
      within DEG_TOL * s_max;
  R5  the separability test is C > 0 exactly, C = s1 - s2 - s3 - s4;
  R6  a target whose reduced state has smaller eigenvalue <= PURE_TOL * trace
      is not entangled with the rest: the Kraus set is returned unchanged
      (W = identity), since every unraveling then has E_av = 0.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

PAULI_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
YY = np.kron(PAULI_Y, PAULI_Y).real.astype(np.complex128)  # real symmetric
H4 = 0.5 * np.array([[1, 1, 1, 1],
                     [1, 1, -1, -1],
                     [1, -1, 1, -1],
                     [1, -1, -1, 1]], dtype=np.complex128)  # App. F, Step 3
U2 = np.diag([1, 1j, 1j, 1j])                                # App. F, Step 2

RANK_TOL = 1e-12
PURE_TOL = 1e-12
DEG_TOL = 1e-9
ZERO_TOL = 1e-10

# Fixed generic reference vectors of the canonical rules R1 and R2.
REF2 = np.array([0.8, 0.36 + 0.48j])
REF4 = np.array([[0.47, 0.31 + 0.22j, -0.18 + 0.53j, 0.26 - 0.52j],
                 [0.12 + 0.44j, 0.58, -0.37 - 0.21j, -0.33 + 0.38j],
                 [-0.29 + 0.35j, 0.14 - 0.41j, 0.62, 0.23 + 0.41j],
                 [0.36 - 0.27j, -0.45 + 0.16j, 0.28 + 0.33j, 0.61],
                 [0.5, -0.5j, 0.5, 0.5j],
                 [0.5j, 0.5, -0.5, 0.5],
                 [1.0, 0.0, 0.0, 0.0],
                 [0.0, 0.0, 0.0, 1.0]])


# --- entanglement measures (Sec. II, App. F) --------------------------------

def von_neumann_entropy(rho: np.ndarray) -> float:
    """-Tr rho ln rho (Eq. def:entanglement_entropy), nats."""
    w = np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))
    w = w[w > 0.0]
    return float(-np.sum(w * np.log(w)))


def entanglement_entropy_2q(psi: np.ndarray) -> float:
    """Entropy of the first qubit of a two-qubit vector (normalizes psi)."""
    m = psi.reshape(2, 2)
    nrm = np.vdot(psi, psi).real
    if nrm <= 0.0:
        return 0.0
    return von_neumann_entropy(m @ m.conj().T / nrm)


def spin_flip_vectors(v: np.ndarray) -> np.ndarray:
    """tilde v = (Y (x) Y) v^* column by column (Eq. spin-flip-vector)."""
    return YY @ v.conj()


def spin_flip_density(rho: np.ndarray) -> np.ndarray:
    return YY @ rho.conj() @ YY


def concurrence(rho: np.ndarray) -> float:
    """Hill-Wootters concurrence through R = sqrt(sqrt(rho) tilde rho sqrt(rho))
    (App. F): C = max(0, l1 - l2 - l3 - l4) with l the eigenvalues of R."""
    rho = 0.5 * (rho + rho.conj().T)
    w, u = np.linalg.eigh(rho)
    s = (u * np.sqrt(np.clip(w, 0.0, None))) @ u.conj().T
    r2 = s @ spin_flip_density(rho) @ s
    lam = np.sqrt(np.clip(np.linalg.eigvalsh(0.5 * (r2 + r2.conj().T)), 0.0, None))
    lam = np.sort(lam)[::-1]
    return float(max(0.0, lam[0] - lam[1] - lam[2] - lam[3]))


def binary_entropy(x: float) -> float:
    """h(x) = -x ln x - (1-x) ln(1-x)."""
    out = 0.0
    for t in (x, 1.0 - x):
        if t > 0.0:
            out -= t * math.log(t)
    return out


def entanglement_of_formation(rho: np.ndarray) -> float:
    """E_oF = h((1 + sqrt(1 - C^2))/2) (Hill-Wootters closed form, App. F)."""
    c = concurrence(rho / np.trace(rho).real)
    return binary_entropy(0.5 * (1.0 + math.sqrt(max(0.0, 1.0 - c * c))))


def ensemble_average_entropy(members: np.ndarray):
    """E_av of a decomposition matrix (columns sub-normalized two-qubit
    vectors), Eq. def:ensemble-averaged_entanglement.  Returns (E_av, p)."""
    p = np.sum(np.abs(members) ** 2, axis=0).real
    e = 0.0
    for k in range(members.shape[1]):
        if p[k] > 0.0:
            e += p[k] * entanglement_entropy_2q(members[:, k])
    return e, p


# --- reduction to the effective two-qubit problem (Sec. IV.B.2) -------------

def effective_state(rho_a: np.ndarray) -> np.ndarray:
    """psi_eff = sqrt(l0) |u0>|0> + sqrt(l1) |u1>|1> from the eigenpairs of the
    target's reduced state (Eqs. schmidt_1_n-1, effective_two_qubit_state)."""
    w, u = np.linalg.eigh(0.5 * (rho_a + rho_a.conj().T))
    order = np.argsort(w)[::-1]
    w, u = np.clip(w[order], 0.0, None), u[:, order]
    if w[0] - w[1] <= DEG_TOL * max(w[0], 1e-300):
        u = np.eye(2, dtype=np.complex128)
    else:
        for k in range(2):
            ov = np.vdot(REF2, u[:, k])
            u[:, k] *= np.conj(ov) / abs(ov)
    psi = np.zeros(4, dtype=np.complex128)
    for k in range(2):
        psi += math.sqrt(w[k]) * np.kron(u[:, k], np.eye(2)[k])
    return psi


def induced_decomposition(kraus: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """phi = sum_j (K_j (x) I)|psi> <j| (Eq. Kraus_to_ensemble in the matrix
    form of App. E); kraus has shape (r, 2, 2)."""
    return np.stack([np.kron(k, np.eye(2)) @ psi for k in kraus], axis=1)


# --- Wootters' optimal decomposition, closed-form version (App. F.2) --------

def unitary_sqrt(w: np.ndarray) -> np.ndarray:
    """Principal square root of a unitary matrix.  A unitary matrix is normal,
    so its complex Schur form w = Z T Z^dagger has a diagonal T (up to
    rounding): the root is Z diag(exp(i theta / 2)) Z^dagger with theta =
    arg T_kk in (-pi, pi], and the branch cut sits at -1, whose root is +i.
    Taking only the diagonal avoids the triangular recurrence of a general
    matrix square root, which is ill-conditioned exactly when eigenvalues
    repeat (the degenerate Takagi values of depolarizing noise)."""
    t, z = sla.schur(np.asarray(w, dtype=np.complex128), output="complex")
    theta = np.angle(np.diag(t))
    theta = np.where(theta <= -math.pi + 1e-12, math.pi, theta)
    return (z * np.exp(0.5j * theta)) @ z.conj().T


def takagi(tau: np.ndarray):
    """Takagi-Autonne factorization tau = U diag(s) U^T of a complex symmetric
    matrix from its SVD: U = U_M sqrt((U_M^T V_M)^*) (App. F.2, Step 1), with
    the principal root of that unitary.  Returns (U, s) with s descending."""
    um, s, vmh = np.linalg.svd(tau)
    vm = vmh.conj().T
    root = unitary_sqrt((um.T @ vm).conj())
    return um @ root, s


def separable_angles(lam: np.ndarray) -> np.ndarray:
    """Phases theta with sum_j exp(2 i theta_j) lam_j = 0
    (Eq. separating_angles_condition), built as the trapezoid of App. F.2:
    theta_1 = 0, theta_4 = pi/2, the legs lam_2, lam_3 closing the gap
    d = lam_1 - lam_4 at height h (Heron's formula, evaluated in Kahan's
    cancellation-free arrangement).  The obtuse-angle test selects the branch
    of theta_3 that closes the polygon: 2 theta_3 = pi + asin(h/lam_3) when
    lam_2 cos(2 theta_2) + lam_1 - lam_4 > 0, else -asin(h/lam_3).  Equal
    values (within DEG_TOL) use the square, theta = (0, pi/4, pi/2, 3pi/4)."""
    l1, l2, l3, l4 = (float(x) for x in lam)
    if l1 - l4 <= DEG_TOL * max(l1, 1e-300):
        return np.array([0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4])
    d = l1 - l4
    a, b, c = sorted((d, l2, l3), reverse=True)
    prod = (a + (b + c)) * (c - (a - b)) * (c + (a - b)) * (a + (b - c))
    area = 0.25 * math.sqrt(max(0.0, prod))
    h = 2.0 * area / d
    a2 = math.pi - math.asin(min(1.0, h / l2)) if l2 > 0.0 else 0.0
    if l3 > 0.0:
        b3 = math.asin(min(1.0, h / l3))
        a3 = math.pi + b3 if l2 * math.cos(a2) + d > 0.0 else -b3
    else:
        a3 = 0.0
    return np.array([0.0, 0.5 * a2, 0.5 * a3, 0.5 * math.pi])


def clusters(vals: np.ndarray, tol: float):
    """Groups of consecutive indices of a descending array whose neighbours
    differ by at most tol * max|vals|."""
    scale = max(float(np.max(np.abs(vals))), 1e-300)
    groups = [[0]]
    for i in range(1, len(vals)):
        if vals[groups[-1][-1]] - vals[i] <= tol * scale:
            groups[-1].append(i)
        else:
            groups.append([i])
    return groups


def reference_basis(members: np.ndarray, complex_freedom: bool) -> np.ndarray:
    """Rule R2: the matrix B (real orthogonal, or unitary when
    complex_freedom) such that members @ B is the canonical basis of the
    block.  Columns of B are Gram-Schmidt orthonormalized gradients
    Re(A^dagger r) (resp. A^dagger r) of the references r in REF4."""
    m = members.shape[1]
    scale = max(float(np.linalg.norm(members)), 1e-300)
    basis = []
    for r in REF4:
        g = members.conj().T @ r
        if not complex_freedom:
            g = g.real.astype(np.complex128)
        for b in basis:
            g = g - np.vdot(b, g) * b
        nrm = np.linalg.norm(g)
        if nrm > 1e-8 * scale * np.linalg.norm(r):
            basis.append(g / nrm)
        if len(basis) == m:
            break
    for k in range(m):           # members of rank < m: complete deterministically
        if len(basis) == m:
            break
        g = np.zeros(m, dtype=np.complex128)
        g[k] = 1.0
        for b in basis:
            g = g - np.vdot(b, g) * b
        nrm = np.linalg.norm(g)
        if nrm > 1e-6:
            basis.append(g / nrm)
    out = np.stack(basis, axis=1)
    return out if complex_freedom else out.real


def wootters(v: np.ndarray, rank: int):
    """Optimal decomposition z = v T of rho = v v^dagger (App. F.2), where the
    columns of v beyond ``rank`` are zero.  Returns (z, T, C)."""
    vt = spin_flip_vectors(v)
    tau = v.conj().T @ vt                       # tau = v^dagger tilde v
    ut = np.eye(4, dtype=np.complex128)
    sig = np.zeros(4)
    if rank > 0:
        u_r, s_r = takagi(tau[:rank, :rank])
        ut[:rank, :rank] = u_r
        sig[:rank] = s_r
    x = v @ ut                                  # x^dagger tilde x = diag(sig)
    if rank > 0:                                # rule R3 on the Takagi vectors
        s1 = sig[0]
        zero = [k for k in range(rank) if sig[k] <= ZERO_TOL * s1]
        nonzero = [k for k in range(rank) if sig[k] > ZERO_TOL * s1]
        for g in (clusters(sig[nonzero], DEG_TOL) if nonzero else []):
            idx = [nonzero[i] for i in g]
            rot = reference_basis(x[:, idx], complex_freedom=False)
            x[:, idx] = x[:, idx] @ rot
            ut[:, idx] = ut[:, idx] @ rot
        if zero:
            rot = reference_basis(x[:, zero], complex_freedom=True)
            x[:, zero] = x[:, zero] @ rot
            ut[:, zero] = ut[:, zero] @ rot
            sig[zero] = 0.0
    c = sig[0] - sig[1] - sig[2] - sig[3]
    if c > 0.0:                                 # entangled: Steps 2 and 3
        y = x @ U2
        yt = spin_flip_vectors(y)
        m = y.conj().T @ yt - c * (y.conj().T @ y)
        mr = 0.5 * (m.real + m.real.T)
        d, q = np.linalg.eigh(mr)
        order = np.argsort(d)[::-1]
        d, q = d[order], q[:, order]
        for g in clusters(d, DEG_TOL):
            q[:, g] = q[:, g] @ reference_basis(y @ q[:, g], complex_freedom=False)
        t = ut @ U2 @ q.astype(np.complex128) @ H4
    else:                                       # separable case
        c = 0.0
        th = separable_angles(sig)
        t = ut @ np.diag(np.exp(1j * th)) @ H4
    return v @ t, t, max(c, 0.0)


def optimal_unraveling(rho_a: np.ndarray, kraus: np.ndarray):
    """Locally entanglement-optimal Kraus set for a target qubit with reduced
    state rho_a (Thm. 2, Sec. IV.B.4): U_opt = U_Wootters U_0 with U_0 from the
    SVD of the induced decomposition (Eq. v_to_phi).

    Returns (kraus_out, W) with kraus_out[k] = sum_j W[j, k] kraus[j]; the
    output has max(r, 4) operators (zero operators pad r < 4)."""
    kraus = np.asarray(kraus, dtype=np.complex128)
    r = kraus.shape[0]
    rp = max(r, 4)
    kpad = np.zeros((rp, 2, 2), dtype=np.complex128)
    kpad[:r] = kraus
    w_rho = np.linalg.eigvalsh(0.5 * (rho_a + rho_a.conj().T))
    if w_rho[0] <= PURE_TOL * max(w_rho.sum(), 1e-300):
        return kpad, np.eye(rp, dtype=np.complex128)
    psi = effective_state(rho_a / np.trace(rho_a).real)
    phi = induced_decomposition(kpad, psi)            # 4 x rp
    uphi, s, vh = np.linalg.svd(phi, full_matrices=True)
    vphi = vh.conj().T                                # rp x rp
    rank = int(np.sum(s > RANK_TOL * s[0]))
    v = np.zeros((4, 4), dtype=np.complex128)
    v[:, :rank] = uphi[:, :rank] * s[:rank]           # v = phi V_phi
    _, t, _ = wootters(v, rank)
    tt = np.eye(rp, dtype=np.complex128)
    tt[:4, :4] = t
    w = vphi @ tt
    kout = np.einsum('jk,jab->kab', w, kpad)
    return kout, w


def haar_optimal(kraus: np.ndarray) -> np.ndarray:
    """The "Haar Optimal" fixed unraveling (Sec. V.B, near-optimal fixed
    unraveling for random circuits): the locally entanglement-optimal Kraus set
    of the Bell state, computed once and used at every site.  The Bell state's
    target has reduced state I/2, whose effective state is Phi+ (rule R1's
    degenerate case picks the computational basis).  By the least-unitary
    corollary (Sec. V.B) the same set minimizes the average unitarity."""
    return optimal_unraveling(0.5 * np.eye(2, dtype=np.complex128), kraus)[0]


def unitarity(k: np.ndarray) -> float:
    """Unitarity of an operator (Eq. def:operator_unitarity): Shannon entropy,
    in bits, of its squared singular values normalized by the squared
    Frobenius norm.  1 for a unitary 2x2 operator, 0 for rank 1; a zero
    operator has no weight and returns 0."""
    k = np.asarray(k, dtype=np.complex128)
    f2 = float(np.sum(np.abs(k) ** 2))
    if f2 <= 0.0:
        return 0.0
    q = np.linalg.svd(k, compute_uv=False) ** 2 / f2
    q = q[q > 0.0]
    return float(-np.sum(q * np.log2(q)))


def unitarity_av(kraus: np.ndarray) -> float:
    """Average unitarity of a Kraus set (least-unitary corollary, Sec. V.B):
    (1/d) sum_i ||K_i||_F^2 unitarity(K_i), d = 2."""
    return float(sum(np.sum(np.abs(k) ** 2) * unitarity(k) for k in np.asarray(kraus)) / 2.0)


def branch_weights(kraus: np.ndarray, rho_a: np.ndarray) -> np.ndarray:
    """p_i = Tr(K_i rho_a K_i^dagger) (Eq. Kraus_to_ensemble)."""
    return np.array([np.trace(k @ rho_a @ k.conj().T).real for k in kraus])


def unraveling_entropy(kraus: np.ndarray, rho_a: np.ndarray) -> float:
    """E_av of the ensemble a Kraus set induces on the target: sum_i p_i S(sigma_i
    / p_i) with sigma_i = K_i rho_a K_i^dagger (the target-vs-rest entropy of each
    branch is the entropy of the branch's reduced target state)."""
    e = 0.0
    for k in kraus:
        sig = k @ rho_a @ k.conj().T
        p = np.trace(sig).real
        if p > 0.0:
            e += p * von_neumann_entropy(sig / p)
    return e
