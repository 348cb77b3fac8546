"""Pins of the oracle's entanglement measures and optimal unraveling against
what the paper fixes: closed forms, printed matrices, invariants and brute
force.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import unravel as U
from oracle import philox
from paper_2508_05745_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_matrices.json")
BELL_PHI_PLUS = np.array([1, 0, 0, 1], dtype=np.complex128) / math.sqrt(2)


def golden(name):
    with open(GOLDEN) as f:
        g = json.load(f)[name]
    if "real" in g:
        return g["scale"] * np.array(g["real"], dtype=np.complex128)
    return g["scale"] * (np.array(g["re"]) + 1j * np.array(g["im"]))


def rand_rho(rng, d=2):
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = a @ a.conj().T
    return r / np.trace(r).real


def choi_state(kraus):
    """(N (x) I)[|Phi+><Phi+|] (App. F.4)."""
    phi = U.induced_decomposition(kraus, BELL_PHI_PLUS)
    return phi @ phi.conj().T


CHANNELS = {
    "depolarizing": (I.depolarizing_kraus(0.02), True),
    "depolarizing_strong": (I.depolarizing_kraus(0.7), True),
    "full_depolarizing": (I.depolarizing_kraus(1.0), True),
    "amplitude_damping": (I.amplitude_damping_kraus(0.3), False),
    "dephasing": (I.dephasing_kraus(0.25), False),
    "ad_then_dephasing": (I.compose_kraus(I.dephasing_kraus(0.01), I.amplitude_damping_kraus(0.01)), False),
}


# --- Philox ------------------------------------------------------------------

def test_philox_matches_numpy_bit_generator():
    """numpy.random.Philox is an independent Philox4x64-10; it increments the
    counter before each block, so its block i uses counter + i + 1."""
    for key, ctr in [((11, 12), (5, 6, 7, 8)), ((2 ** 64 - 1, 0), (2 ** 64 - 2, 3, 0, 2 ** 63)),
                     ((0, 0), (0, 0, 0, 0))]:
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        raw = bg.random_raw(12)
        c = list(ctr)
        for blk in range(3):
            c[0] = (c[0] + 1) % 2 ** 64
            if c[0] == 0:
                c[1] = (c[1] + 1) % 2 ** 64
            assert list(philox.philox4x64_10(c, key)) == [int(x) for x in raw[4 * blk:4 * blk + 4]]


def test_philox_uniform_range_and_moments():
    u = np.array([philox.uniform(7, t, g, s) for t in range(40) for g in range(25) for s in range(2)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)


# --- entropies and concurrence -----------------------------------------------

def test_entropy_product_and_bell():
    assert abs(U.entanglement_entropy_2q(np.array([1, 0, 0, 0], complex))) < 1e-15
    assert abs(U.entanglement_entropy_2q(BELL_PHI_PLUS) - math.log(2)) < 1e-14


@pytest.mark.parametrize("p", [0.0, 0.02, 0.3, 0.9])
def test_choi_dephasing_closed_form(p):
    """Choi state of dephasing: eigenvalues {1-p/2, p/2, 0, 0}, C = 1-p,
    E_oF = h((1 + sqrt((2-p)p))/2) (App. F.4, dephasing proposition)."""
    rho = choi_state(I.dephasing_kraus(p))
    ev = np.sort(np.linalg.eigvalsh(rho))[::-1]
    assert np.allclose(ev, [1 - p / 2, p / 2, 0, 0], atol=1e-14)
    assert abs(U.concurrence(rho) - (1 - p)) < 1e-7
    eof = U.binary_entropy((1 + math.sqrt((2 - p) * p)) / 2)
    assert abs(U.entanglement_of_formation(rho) - eof) < 1e-7


@pytest.mark.parametrize("g", [0.0, 0.01, 0.3, 0.8])
def test_choi_amplitude_damping_closed_form(g):
    """Choi state of AD: R has one non-zero eigenvalue sqrt(1-gamma),
    E_oF = h((1 + sqrt(gamma))/2) (App. F.4)."""
    rho = choi_state(I.amplitude_damping_kraus(g))
    assert abs(U.concurrence(rho) - math.sqrt(1 - g)) < 1e-7
    assert abs(U.entanglement_of_formation(rho) - U.binary_entropy((1 + math.sqrt(g)) / 2)) < 1e-7


@pytest.mark.parametrize("p", [0.0, 0.02, 0.3, 0.6, 0.8])
def test_choi_depolarizing_closed_form(p):
    """Choi state of depolarizing: eigenvalues {1-3p/4, p/4, p/4, p/4},
    C = max(0, 1-3p/2), E_oF = h((2 + sqrt(3) sqrt((4-3p)p))/4) for p <= 2/3."""
    rho = choi_state(I.depolarizing_kraus(p))
    ev = np.sort(np.linalg.eigvalsh(rho))[::-1]
    assert np.allclose(ev, [1 - 3 * p / 4, p / 4, p / 4, p / 4], atol=1e-14)
    assert abs(U.concurrence(rho) - max(0.0, 1 - 1.5 * p)) < 1e-7
    if p <= 2 / 3:
        eof = U.binary_entropy((2 + math.sqrt(3) * math.sqrt((4 - 3 * p) * p)) / 4)
    else:
        eof = 0.0
    assert abs(U.entanglement_of_formation(rho) - eof) < 1e-7


@pytest.mark.parametrize("s,g", [(0.3, 0.1), (0.8, 0.5), (0.6, 0.0)])
def test_ad_on_computational_schmidt_state(s, g):
    """AD on s|00> + sqrt(1-s^2)|11>: C = 2 s sqrt(1-s^2) sqrt(1-gamma), and the
    printed 2x2 unitary reaches E_oF (App. F.4 remark)."""
    psi = np.array([s, 0, 0, math.sqrt(1 - s * s)], dtype=np.complex128)
    kr = I.amplitude_damping_kraus(g)
    phi = U.induced_decomposition(kr, psi)
    rho = phi @ phi.conj().T
    c = 2 * s * math.sqrt(1 - s * s) * math.sqrt(1 - g)
    assert abs(U.concurrence(rho) - c) < 1e-7
    u = golden("ad_computational_optimal_unitary")
    kp = np.einsum('kj,jab->kab', u, kr)      # printed as K'_i' = sum_i U_i'i K_i
    e, _ = U.ensemble_average_entropy(U.induced_decomposition(kp, psi))
    assert abs(e - U.entanglement_of_formation(rho)) < 1e-7


def test_werner_decompositions():
    """Werner state W(l) = l |Psi-><Psi-| + (1-l) I/4 (App. A): computational
    decomposition E_av = l ln2, Bell decomposition E_av = ln2, the printed
    mixing unitary gives E_av = 0 at l = 1/3, and W is separable for l <= 1/3."""
    psi_m = np.array([0, 1, -1, 0], dtype=np.complex128) / math.sqrt(2)
    bell = [np.array([1, 0, 0, 1]) / math.sqrt(2), np.array([1, 0, 0, -1]) / math.sqrt(2),
            np.array([0, 1, 1, 0]) / math.sqrt(2)]
    for lam in (0.2, 1 / 3, 0.7):
        comp = np.stack([math.sqrt(lam) * psi_m] + [0.5 * math.sqrt(1 - lam) * e for e in np.eye(4)], axis=1)
        bellw = np.stack([0.5 * math.sqrt(3 * lam + 1) * psi_m] + [0.5 * math.sqrt(1 - lam) * b for b in bell], axis=1)
        w = lam * np.outer(psi_m, psi_m.conj()) + (1 - lam) * np.eye(4) / 4
        assert np.allclose(comp @ comp.conj().T, w) and np.allclose(bellw @ bellw.conj().T, w)
        assert abs(U.ensemble_average_entropy(comp)[0] - lam * math.log(2)) < 1e-13
        assert abs(U.ensemble_average_entropy(bellw)[0] - math.log(2)) < 1e-13
        wc = max(0.0, (3 * lam - 1) / 2)   # textbook Werner concurrence
        assert abs(U.concurrence(w) - wc) < 1e-7
        if lam <= 1 / 3 + 1e-12:
            assert U.entanglement_of_formation(w) < 1e-12
    lam = 1 / 3
    bellw = np.stack([0.5 * math.sqrt(3 * lam + 1) * psi_m] + [0.5 * math.sqrt(1 - lam) * b for b in bell], axis=1)
    mix = golden("werner_separable_unitary")
    assert np.allclose(mix @ mix.conj().T, np.eye(4))
    z = bellw @ mix.T          # |phi_i> = sum_j U_ij |member_j>
    assert U.ensemble_average_entropy(z)[0] < 1e-12


def test_dephasing_projective_relation():
    """The printed 3x3 matrix maps the mixed-unitary dephasing Kraus set to the
    projective one (Sec. II).  As printed, its (1,3) entry has the wrong sign
    for a unitary (row 1 is then not orthogonal to rows 2 and 3); that entry
    multiplies the zero operator, so the map is unaffected.  Reading: the
    (1,3) entry is -sqrt(p/(2-p))."""
    p = 0.3
    printed13 = math.sqrt(p / (2 - p))
    m = np.array([[math.sqrt((2 - 2 * p) / (2 - p)), 0, printed13],
                  [math.sqrt(p) / math.sqrt(2 * (2 - p)), 1 / math.sqrt(2), math.sqrt((1 - p) / (2 - p))],
                  [math.sqrt(p) / math.sqrt(2 * (2 - p)), -1 / math.sqrt(2), math.sqrt((1 - p) / (2 - p))]])
    k = np.concatenate([I.dephasing_kraus(p), np.zeros((1, 2, 2))])
    want = [math.sqrt(1 - p) * np.eye(2), math.sqrt(p) * np.diag([1, 0]), math.sqrt(p) * np.diag([0, 1])]
    assert np.allclose(np.einsum('ij,jab->iab', m, k), want)
    assert not np.allclose(m @ m.T, np.eye(3))
    m[0, 2] = -printed13
    assert np.allclose(m @ m.T, np.eye(3))
    assert np.allclose(np.einsum('ij,jab->iab', m, k), want)


# --- Wootters building blocks ---------------------------------------------------

def test_takagi_residual(rng):
    for trial in range(50):
        a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        tau = a + a.T
        if trial % 5 == 0:          # degenerate Takagi values
            q = I.haar_unitary(rng, 4)
            tau = q @ np.diag([2.0, 1.0, 1.0, 1.0]) @ q.T
        u, s = U.takagi(tau)
        assert np.allclose(u.conj().T @ u, np.eye(4), atol=1e-12)
        assert np.allclose(u @ np.diag(s) @ u.T, tau, atol=1e-12)
        assert np.all(np.diff(s) <= 1e-15)


def test_unitary_sqrt_is_the_principal_root(rng):
    """The unitary root squares back, its eigenvalues have arguments in
    (-pi/2, pi/2] (principal branch, -1 -> +i), and repeated eigenvalues (the
    degenerate Takagi values of depolarizing noise) cause no loss of accuracy."""
    cases = [I.haar_unitary(rng, 4) for _ in range(20)]
    q = I.haar_unitary(rng, 4)
    cases.append(q @ np.diag(np.exp(1j * np.array([0.3, 0.3, 0.3, -2.0]))) @ q.conj().T)
    cases.append(q @ np.diag([-1.0, -1.0, 1.0, 1j]) @ q.conj().T)
    cases.append(np.eye(4, dtype=complex))
    for w in cases:
        r = U.unitary_sqrt(w)
        assert np.allclose(r @ r, w, atol=1e-13)
        assert np.allclose(r.conj().T @ r, np.eye(4), atol=1e-13)
        ang = np.angle(np.linalg.eigvals(r))
        assert np.all(ang > -np.pi / 2 - 1e-9) and np.all(ang <= np.pi / 2 + 1e-9)
    r = U.unitary_sqrt(-np.eye(2, dtype=complex))
    assert np.allclose(r, 1j * np.eye(2), atol=1e-15)


def test_degenerate_depolarizing_inputs_raise_no_warning():
    """Bell target (reduced state I/2) and depolarizing channels, whose Takagi
    values are degenerate by construction: the optimal unraveling is computed
    without any numerical warning and reaches the closed-form E_oF."""
    import warnings
    for p in (0.02, 0.3, 1.0):
        kr = I.depolarizing_kraus(p)
        with warnings.catch_warnings():
            warnings.simplefilter("error")
            out, _ = U.optimal_unraveling(np.eye(2, dtype=complex) / 2, kr)
            e = U.unraveling_entropy(out, np.eye(2, dtype=complex) / 2)
        assert np.allclose(sum(k.conj().T @ k for k in out), np.eye(2), atol=1e-12)
        assert e >= -1e-14


def test_separable_angles_close_the_polygon(rng):
    """sum_j exp(2 i theta_j) lam_j = 0 (Eq. separating_angles_condition) for
    descending lam with lam_1 <= lam_2 + lam_3 + lam_4, including triangles
    (lam_4 = 0), the square case and cases where the angle at lam_4 is acute."""
    cases = [np.array([1.0, 1.0, 1.0, 1.0]), np.array([1.0, 1.0, 1.0, 0.0]),
             np.array([1.0, 0.6, 0.5, 0.0]), np.array([0.5, 0.5, 0.0, 0.0])]
    while len(cases) < 300:
        lam = np.sort(rng.uniform(0, 1, 4))[::-1]
        if lam[0] <= lam[1:].sum():
            cases.append(lam)
    for lam in cases:
        th = U.separable_angles(lam)
        assert abs(np.sum(np.exp(2j * th) * lam)) < 1e-12 * max(1.0, lam[0])


# --- optimal unraveling ------------------------------------------------------------

@pytest.mark.parametrize("name", list(CHANNELS))
def test_optimal_unraveling_reaches_eof(name, rng):
    """E_av(K') equals the Hill-Wootters E_oF of the effective state (Thm. 2);
    K' is a valid Kraus set of the same channel (Eq. unitarity_kraus)."""
    kraus, full_rank = CHANNELS[name]
    tol = 1e-12 if full_rank else 1e-7   # sqrt(R) route of the pin loses precision at rank < 4
    for _ in range(60):
        rho = rand_rho(rng)
        kp, w = U.optimal_unraveling(rho, kraus)
        assert np.allclose(w.conj().T @ w, np.eye(w.shape[0]), atol=1e-12)
        assert np.allclose(sum(k.conj().T @ k for k in kp), np.eye(2), atol=1e-13)
        sig = rand_rho(rng)
        assert np.allclose(sum(k @ sig @ k.conj().T for k in kp), sum(k @ sig @ k.conj().T for k in kraus), atol=1e-13)
        phi = U.induced_decomposition(kraus, U.effective_state(rho))
        eof = U.entanglement_of_formation(phi @ phi.conj().T)
        assert abs(U.unraveling_entropy(kp, rho) - eof) < tol


@pytest.mark.parametrize("name", ["depolarizing", "amplitude_damping", "ad_then_dephasing"])
def test_no_remix_beats_the_optimum(name, rng):
    """Brute force: Haar-random remixes and the U(theta, phi) grid never go
    below E_av of the optimal unraveling."""
    kraus, _ = CHANNELS[name]
    r = max(4, kraus.shape[0])
    kpad = np.zeros((r, 2, 2), complex)
    kpad[:kraus.shape[0]] = kraus
    for _ in range(8):
        rho = rand_rho(rng)
        best = U.unraveling_entropy(U.optimal_unraveling(rho, kraus)[0], rho)
        for _ in range(200):
            v = I.haar_unitary(rng, r)
            assert U.unraveling_entropy(np.einsum('jk,jab->kab', v, kpad), rho) >= best - 1e-12
        from oracle.adjoint import grid_search
        assert grid_search(rho, kpad, 16)[0] >= best - 1e-12


@pytest.mark.parametrize("name,closed", [
    ("dephasing", lambda p: U.binary_entropy((1 + math.sqrt((2 - p) * p)) / 2)),
    ("amplitude_damping", lambda g: U.binary_entropy((1 + math.sqrt(g)) / 2)),
    ("depolarizing", lambda p: U.binary_entropy((2 + math.sqrt(3) * math.sqrt((4 - 3 * p) * p)) / 4)),
])
def test_optimal_unraveling_on_bell_target(name, closed):
    """A maximally entangled target (rho_A = I/2) gives the Choi state; the
    optimal unraveling reaches the printed E_oF (App. F.4 propositions)."""
    param = {"dephasing": 0.25, "amplitude_damping": 0.3, "depolarizing": 0.02}[name]
    kraus = CHANNELS[name][0]
    kp, _ = U.optimal_unraveling(np.eye(2) / 2, kraus)
    assert abs(U.unraveling_entropy(kp, np.eye(2) / 2) - closed(param)) < 1e-7


@pytest.mark.parametrize("name", list(CHANNELS))
def test_output_independent_of_input_representation(name, rng):
    """The optimal Kraus set depends only on the channel and the state: remixing
    the input Kraus set by any unitary leaves the output unchanged (this pins
    the remix bookkeeping W = V_phi T and the canonical rules)."""
    kraus, _ = CHANNELS[name]
    r = max(4, kraus.shape[0])
    kpad = np.zeros((r, 2, 2), complex)
    kpad[:kraus.shape[0]] = kraus
    for _ in range(20):
        rho = rand_rho(rng)
        k1, _ = U.optimal_unraveling(rho, kpad)
        v = I.haar_unitary(rng, r)
        k2, _ = U.optimal_unraveling(rho, np.einsum('jk,jab->kab', v, kpad))
        assert np.allclose(k1[:4], k2[:4], atol=1e-9)


@pytest.mark.parametrize("name", list(CHANNELS))
def test_canonical_rules_are_well_conditioned(name, rng):
    """A 1e-11 perturbation of rho_A moves the branch weights by O(1e-10): the
    canonical rules pick a continuous branch of the optimal decompositions even
    where the optimum is degenerate."""
    kraus, _ = CHANNELS[name]
    for _ in range(50):
        rho = rand_rho(rng)
        b = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        k1, _ = U.optimal_unraveling(rho, kraus)
        k2, _ = U.optimal_unraveling(rho + 1e-11 * (b + b.conj().T), kraus)
        assert np.abs(U.branch_weights(k1, rho) - U.branch_weights(k2, rho)).max() < 1e-8


def test_pure_target_keeps_kraus_set():
    rho = np.diag([1.0, 0.0]).astype(complex)
    kraus = I.depolarizing_kraus(0.1)
    kp, w = U.optimal_unraveling(rho, kraus)
    assert np.allclose(kp, kraus) and np.allclose(w, np.eye(4))


def test_haar_sampler_two_design_purity(rng):
    """E[Tr rho_1^2] = (2 + 2^{n-1}) / (2^n + 1) for n = 2 (Sec. VI.B, 2-design
    purity): pins the Haar gate sampler of the input generator."""
    vals = []
    for _ in range(20000):
        psi = I.haar_unitary(rng, 4)[:, 0].reshape(2, 2)
        r = psi @ psi.conj().T
        vals.append(np.trace(r @ r).real)
    vals = np.array(vals)
    assert abs(vals.mean() - 4 / 5) < 4 * vals.std() / math.sqrt(vals.size)


# --- fixed unravelings: Haar Optimal, least unitary (Sec. V.B) ------------------

HADAMARD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)


def remix(kraus, u):
    """K'_i = sum_j U_ij K_j (Eq. unitarity_kraus, as the table applies it)."""
    return np.einsum('ij,jab->iab', u, np.asarray(kraus, dtype=np.complex128))


# Haar Optimal sets of the paper's table of unravelings: the Orthogonal set
# rotated by H (dephasing, amplitude damping) or H (x) H (depolarizing).
TABLE_HAAR_OPTIMAL = {
    "dephasing": (lambda p: remix(I.dephasing_kraus(p), HADAMARD),
                  lambda p: U.binary_entropy((1 + math.sqrt((2 - p) * p)) / 2)),
    "amplitude_damping": (lambda g: remix(I.amplitude_damping_kraus(g), HADAMARD),
                          lambda g: U.binary_entropy((1 + math.sqrt(g)) / 2)),
    "depolarizing": (lambda p: remix(I.depolarizing_kraus(p), np.kron(HADAMARD, HADAMARD)),
                     lambda p: U.binary_entropy((2 + math.sqrt(3) * math.sqrt((4 - 3 * p) * p)) / 4)),
}
ORTHOGONAL = {"dephasing": I.dephasing_kraus, "amplitude_damping": I.amplitude_damping_kraus,
              "depolarizing": I.depolarizing_kraus}


def test_unitarity_closed_forms():
    """Eq. def:operator_unitarity: 1 for a unitary, 0 for rank 1, the binary
    entropy of the normalized squared singular values otherwise."""
    assert abs(U.unitarity(np.eye(2)) - 1.0) < 1e-15
    assert abs(U.unitarity(0.3 * I.PAULI_Y) - 1.0) < 1e-15
    assert abs(U.unitarity(np.diag([1.0, 0.0])) - 0.0) < 1e-15
    assert U.unitarity(np.zeros((2, 2))) == 0.0
    g = 0.37
    k0 = I.amplitude_damping_kraus(g)[0]
    q = 1.0 / (2.0 - g)
    assert abs(U.unitarity(k0) - U.binary_entropy(q) / math.log(2)) < 1e-14


def test_average_unitarity_is_bell_entropy_in_bits(rng):
    """For any Kraus set, (1/2) sum ||K||_F^2 unitarity(K) equals E_av of the
    Bell state (reduced state I/2) in bits: (K (x) I)|Phi+> has Schmidt
    coefficients sigma(K) / ||K||_F and branch weight ||K||_F^2 / 2."""
    for trial in range(20):
        r = int(rng.integers(1, 6))
        v = np.linalg.qr(rng.standard_normal((2 * r, 2)) + 1j * rng.standard_normal((2 * r, 2)))[0]
        kraus = v.reshape(r, 2, 2)                      # random channel: isometry blocks
        assert np.allclose(sum(k.conj().T @ k for k in kraus), np.eye(2))
        e_bell = U.unraveling_entropy(kraus, np.eye(2) / 2)
        assert abs(U.unitarity_av(kraus) - e_bell / math.log(2)) < 1e-12


@pytest.mark.parametrize("name", list(TABLE_HAAR_OPTIMAL))
@pytest.mark.parametrize("param", [0.01, 0.2, 0.5])
def test_haar_optimal_matches_the_table(name, param):
    """haar_optimal (the Bell state's optimal remix) and the paper's table set
    both reach the closed-form E_oF of the Choi state at the Bell input, and
    have the same (minimal) average unitarity."""
    table_set, closed = TABLE_HAAR_OPTIMAL[name]
    k_orth = ORTHOGONAL[name](param)
    k_ho = U.haar_optimal(k_orth)
    k_tab = table_set(param)
    half = np.eye(2) / 2
    assert abs(U.unraveling_entropy(k_ho, half) - closed(param)) < 1e-9
    assert abs(U.unraveling_entropy(k_tab, half) - closed(param)) < 1e-9
    assert abs(U.unitarity_av(k_ho) - U.unitarity_av(k_tab)) < 1e-9
    # the channel is unchanged
    rho = rand_rho(np.random.default_rng(7))
    out = lambda ks: sum(k @ rho @ k.conj().T for k in ks)
    assert np.allclose(out(k_ho), out(k_orth), atol=1e-13)


@pytest.mark.parametrize("name", ["dephasing", "depolarizing", "amplitude_damping", "ad_then_dephasing"])
def test_haar_optimal_is_least_unitary(name, rng):
    """Least-unitary corollary: no remix of the Kraus set has a smaller
    average unitarity than the Haar-optimal one (brute force over Haar
    unitaries of the padded set)."""
    kraus = CHANNELS[name][0]
    r = max(len(kraus), 4)
    kpad = np.zeros((r, 2, 2), dtype=np.complex128)
    kpad[:len(kraus)] = kraus
    best = U.unitarity_av(U.haar_optimal(kraus))
    for trial in range(300):
        assert U.unitarity_av(remix(kpad, I.haar_unitary(rng, r))) >= best - 1e-12
    # Orthogonal and Projective fixed sets are not below it either
    assert U.unitarity_av(kraus) >= best - 1e-12


@pytest.mark.parametrize("p", [0.05, 0.4])
def test_projective_sets(p):
    """The Projective sets of the appendix on common unravelings are valid
    Kraus sets of the same channels, and at the Bell input they sit above the
    optimum (dephasing: E_av = (1 - p) ln 2, the identity branch alone)."""
    rho = rand_rho(np.random.default_rng(3))
    half = np.eye(2) / 2
    for proj, orth in ((I.projective_dephasing_kraus(p), I.dephasing_kraus(p)),
                       (I.projective_depolarizing_kraus(p), I.depolarizing_kraus(p))):
        assert np.allclose(sum(k.conj().T @ k for k in proj), np.eye(2))
        assert np.allclose(sum(k @ rho @ k.conj().T for k in proj), sum(k @ rho @ k.conj().T for k in orth))
        assert U.unraveling_entropy(proj, half) >= U.unraveling_entropy(U.haar_optimal(orth), half) - 1e-12
    assert abs(U.unraveling_entropy(I.projective_dephasing_kraus(p), half) - (1 - p) * math.log(2)) < 1e-12
