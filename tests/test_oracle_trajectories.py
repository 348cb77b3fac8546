"""Pins of the oracle's trajectory simulators and error estimator (CPU only)."""
import copy
import math

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import trajectories as T
from oracle import unravel as U
from paper_2508_05745_gb300 import inputs as I


@pytest.fixture(scope="module")
def small():
    return I.workload_small_exact(seed=0)


@pytest.mark.parametrize("mode", ["optimal", "haar_optimal"])
def test_dense_and_mps_agree_without_truncation(small, mode):
    """chi >= 2^{n/2}: the MPS trajectory equals the state-vector trajectory
    on the same Philox stream (two independent implementations of Alg. 1),
    for the adaptive and the fixed Haar-optimal unraveling."""
    c = small["circuit"]
    for tr in range(6):
        d = T.dense_trajectory(c, tr, 0, mode=mode)
        m = T.mps_trajectory(c, tr, 0, 16, keep_dense=True, mode=mode)
        assert d.branch == m.branch
        assert abs(abs(np.vdot(d.state, m.state)) - 1.0) < 1e-12
        assert np.allclose(d.p_branch, m.p_branch, atol=1e-12)
        assert np.allclose(d.z, m.z, atol=1e-12) and np.allclose(d.zz, m.zz, atol=1e-12)
        assert abs(d.s_half - m.s_half) < 1e-11
        assert max(m.discarded) < 1e-20 and m.eps_bound == 0.0


def test_haar_optimal_trajectories_reproduce_density_matrix(small):
    """A fixed unraveling is unbiased too: the Haar-optimal mode's trajectory
    means over 128 trajectories match exact density-matrix evolution (all 15
    z-scores below 4)."""
    c = small["circuit"]
    rho = T.density_evolution(c)
    zr, zzr = T.density_observables(rho, c.n_qubits)
    recs = [T.dense_trajectory(c, tr, 0, mode="haar_optimal") for tr in range(128)]
    mz, sz = T.trajectory_statistics([r.z for r in recs])
    mzz, szz = T.trajectory_statistics([r.zz for r in recs])
    z = np.concatenate([(mz - zr) / sz, (mzz - zzr) / szz])
    assert np.max(np.abs(z)) < 4.0, z


@pytest.mark.slow
def test_trajectory_average_reproduces_density_matrix(small):
    """Unbiasedness (Eq. Kraus_to_ensemble averaged over branches): the mean of
    <Z_i>, <Z_i Z_i+1> over 256 trajectories matches exact density-matrix
    evolution; all 15 z-scores must stay below 4."""
    c = small["circuit"]
    rho = T.density_evolution(c)
    zr, zzr = T.density_observables(rho, c.n_qubits)
    recs = [T.dense_trajectory(c, tr, 0) for tr in range(256)]
    mz, sz = T.trajectory_statistics([r.z for r in recs])
    mzz, szz = T.trajectory_statistics([r.zz for r in recs])
    z = np.concatenate([(mz - zr) / sz, (mzz - zzr) / szz])
    assert np.max(np.abs(z)) < 4.0, z


def test_global_layering_dense_and_mps_agree(small):
    """Global layering (all gates, then all noise, then a truncation sweep,
    Sec. IV.A): the state-vector and MPS implementations agree per
    trajectory when chi >= 2^{n/2}, on the same Philox counters."""
    c = small["circuit"]
    for tr in range(6):
        d = T.dense_trajectory(c, tr, 0, layering="global")
        m = T.mps_trajectory(c, tr, 0, 16, keep_dense=True, layering="global")
        assert d.branch == m.branch
        assert abs(abs(np.vdot(d.state, m.state)) - 1.0) < 1e-12
        assert np.allclose(d.z, m.z, atol=1e-12) and np.allclose(d.zz, m.zz, atol=1e-12)
        assert abs(d.s_half - m.s_half) < 1e-11
        assert max(m.discarded) < 1e-20


def test_global_layering_is_the_same_channel(small):
    """Both layerings realize the same channel (the noise on one pair commutes
    with the gates on the other, disjoint pairs of a layer): the global
    layering's trajectory means over 128 trajectories match the exact
    density-matrix evolution (all 15 z-scores below 4).  Without truncation
    the two layerings give the same trajectory, branch for branch."""
    c = small["circuit"]
    rho = T.density_evolution(c)
    zr, zzr = T.density_observables(rho, c.n_qubits)
    recs = [T.dense_trajectory(c, tr, 0, layering="global") for tr in range(128)]
    mz, sz = T.trajectory_statistics([r.z for r in recs])
    mzz, szz = T.trajectory_statistics([r.zz for r in recs])
    z = np.concatenate([(mz - zr) / sz, (mzz - zzr) / szz])
    assert np.max(np.abs(z)) < 4.0, z
    for tr in range(4):
        loc = T.dense_trajectory(c, tr, 0)
        assert loc.branch == recs[tr].branch
        assert abs(abs(np.vdot(loc.state, recs[tr].state)) - 1.0) < 1e-12


def test_global_layering_discards_less():
    """Truncating after the whole layer's noise discards less weight than
    truncating after each gate (Sec. IV.A, layering options): lower summed
    discarded weight on average and in most of 24 trajectories, for three
    noise strengths and bond caps (fixed seeds)."""
    for p, chi in [(0.05, 4), (0.02, 6), (0.1, 4)]:
        c = I.random_brickwork(10, 8, I.depolarizing_kraus(p), seed=4)
        loc = np.array([sum(T.mps_trajectory(c, tr, 1, chi, cutoff=1e-14).discarded) for tr in range(24)])
        glo = np.array([sum(T.mps_trajectory(c, tr, 1, chi, cutoff=1e-14, layering="global").discarded)
                        for tr in range(24)])
        assert glo.mean() < loc.mean()
        assert np.mean(glo < loc) > 0.75


def test_global_layering_truncates_every_bond():
    """With chi_max below the exact rank, the sweep leaves every bond at most
    chi_max, and the discarded weights enter the error bound."""
    c = I.random_brickwork(10, 6, I.depolarizing_kraus(0.05), seed=4)
    rec = T.mps_trajectory(c, 0, 1, 4, cutoff=1e-14, layering="global")
    assert rec.eps_bound > 0.0 and max(rec.discarded) > 0.0
    m_ref = T.mps_trajectory(c, 0, 1, 4, cutoff=1e-14, layering="global", keep_dense=True)
    psi = m_ref.state
    n = c.n_qubits
    for k in range(1, n):
        rank = np.linalg.matrix_rank(psi.reshape(2 ** k, -1), tol=1e-10)
        assert rank <= 4


def test_given_mode_with_identity_noise_is_unitary(small):
    c = copy.deepcopy(small["circuit"])
    for l in c.layers:
        l.kraus = np.eye(2, dtype=complex)[None]
    d = T.dense_trajectory(c, 0, 0, mode="given")
    psi = np.zeros(2 ** 8, complex)
    psi[0] = 1
    for l in c.layers:
        for q, g in zip(l.left_qubits, l.gates):
            psi = T.apply_2q(psi, g, int(q), 8)
    assert abs(abs(np.vdot(psi, d.state)) - 1) < 1e-13


def test_bell_pair_half_chain_entropy():
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    g = cnot @ np.kron(h, np.eye(2))
    c = I.Circuit(2, [I.Layer(np.array([0], np.int32), g[None], np.eye(2, dtype=complex)[None])])
    for rec in (T.dense_trajectory(c, 0, 0, mode="given"), T.mps_trajectory(c, 0, 0, 4, mode="given")):
        assert abs(rec.s_half - math.log(2)) < 1e-13
        assert np.allclose(rec.z, 0, atol=1e-13) and np.allclose(rec.zz, 1, atol=1e-13)


def test_product_state_entropy_zero():
    c = I.Circuit(4, [I.Layer(np.array([0, 2], np.int32), np.stack([np.eye(4, dtype=complex)] * 2),
                              np.eye(2, dtype=complex)[None])])
    rec = T.mps_trajectory(c, 0, 0, 4, mode="given")
    assert rec.s_half == 0.0 and np.allclose(rec.z, 1.0)


@pytest.mark.slow
def test_error_bound_covers_observable_error():
    """Thm. 1 soundness on a truncated run: |<O>_exact - <O>_trajectories| for
    the single-site Z (||Z|| = 1) is below eps_hat + Hoeffding buffer + 4 s.e."""
    c = I.random_brickwork(6, 6, I.depolarizing_kraus(0.05), seed=3)
    rho = T.density_evolution(c)
    zr, _ = T.density_observables(rho, 6)
    recs = [T.mps_trajectory(c, tr, 11, chi_max=2, cutoff=1e-14) for tr in range(200)]
    eps_hat, buf = T.error_estimate(np.array([r.eps_bound for r in recs]))
    mz, sz = T.trajectory_statistics([r.z for r in recs])
    assert eps_hat > 0.0
    assert np.all(np.abs(mz - zr) <= eps_hat + buf + 4 * sz)


def test_eps_bound_definition():
    """eps_bound = sum_l 4 sqrt(2 sum_k eps_k) if that is <= eps_max - 2 else
    eps_max (App. B, Eq. systematic_error_with_constant_bound)."""
    c = I.random_brickwork(6, 4, I.depolarizing_kraus(0.05), seed=5)
    rec = T.mps_trajectory(c, 0, 1, chi_max=2, cutoff=1e-14, eps_max=1e9)
    per_layer = []
    k = 0
    for l in c.layers:
        per_layer.append(sum(rec.discarded[k:k + len(l.left_qubits)]))
        k += len(l.left_qubits)
    want = sum(4 * math.sqrt(2 * e) for e in per_layer)
    assert abs(rec.eps_bound - want) < 1e-12
    capped = T.mps_trajectory(c, 0, 1, chi_max=2, cutoff=1e-14, eps_max=want + 1.0)
    assert capped.eps_bound == want + 1.0


def test_cut_gaps_are_the_schmidt_gaps_at_the_cut():
    """The recorded cut gap of a truncating split is (w_chi' - w_chi'+1) / w_1
    of the squared Schmidt values of the state being split: for the first
    gate of a circuit, the dense trajectory (same branches) holds that state,
    whose Schmidt values across the gated bond are computed here by an
    independent SVD.  Untruncated runs record no gaps."""
    c = I.random_brickwork(4, 1, I.depolarizing_kraus(0.3), seed=7)
    c = I.Circuit(4, [I.Layer(c.layers[0].left_qubits[:1], c.layers[0].gates[:1], c.layers[0].kraus)])
    q = int(c.layers[0].left_qubits[0])
    dense = T.dense_trajectory(c, 0, 2)
    s = np.linalg.svd(dense.state.reshape(2 ** (q + 1), -1), compute_uv=False)
    w = s ** 2
    rec = T.mps_trajectory(c, 0, 2, chi_max=1, cutoff=1e-14)
    assert rec.branch == dense.branch
    assert len(rec.cut_gaps) == 1
    assert abs(rec.cut_gaps[0] - (w[0] - w[1]) / w[0]) < 1e-12
    full = T.mps_trajectory(I.random_brickwork(6, 3, I.depolarizing_kraus(0.05), seed=5), 0, 1, chi_max=8,
                            cutoff=0.0)
    assert full.cut_gaps == []


def test_complex64_rounding_is_amplified_at_close_cuts(monkeypatch):
    """The reading behind the mixed-precision tolerance: rounding every split's
    output to complex64 (the storage of the mixed path, nothing else changed)
    moves a heavily truncated trajectory (chi = 4, 10 qubits, 10 layers of
    depolarizing brickwork) by far more than eps_32: the kept subspace turns
    by up to ~eps_32 / gap at a cut whose relative gap is small."""
    circ = I.random_brickwork(10, 10, I.depolarizing_kraus(0.05), seed=4)
    plain = T._split

    def split_c64(m, q, th, cap, cutoff, rec):
        e = plain(m, q, th.astype(np.complex64).astype(np.complex128), cap, cutoff, rec)
        m.a[q] = m.a[q].astype(np.complex64).astype(np.complex128)
        m.a[q + 1] = m.a[q + 1].astype(np.complex64).astype(np.complex128)
        return e

    out = []
    for t in (0, 2):
        ref = T.mps_trajectory(circ, t, 3, chi_max=4, cutoff=1e-14)
        monkeypatch.setattr(T, "_split", split_c64)
        r32 = T.mps_trajectory(circ, t, 3, chi_max=4, cutoff=1e-14)
        monkeypatch.setattr(T, "_split", plain)
        assert r32.branch == ref.branch
        err = max(np.abs(r32.z - ref.z).max(), np.abs(r32.zz - ref.zz).max(), abs(r32.s_half - ref.s_half))
        out.append((min(ref.cut_gaps), err))
    (g0, e0), (g2, e2) = out
    assert g0 < 2e-3 and e0 > 5e-6             # ~300 eps_32 at a cut gap of 1.4e-3
    assert all(e < 1e-6 / g for g, e in out)   # within 1e-6 / gap, the GPU tolerance


def test_coin_noise_matches_density_matrix():
    """Probabilistic noise (coin_p < 1, the two-qubit depolarizing reading):
    the trajectory average still reproduces the exact channel."""
    c = I.random_brickwork(4, 4, I.depolarizing_kraus(1.0), seed=9, coin_p=0.3)
    rho = T.density_evolution(c)
    zr, zzr = T.density_observables(rho, 4)
    recs = [T.mps_trajectory(c, tr, 2, chi_max=4) for tr in range(400)]
    mz, sz = T.trajectory_statistics([r.z for r in recs])
    assert np.max(np.abs((mz - zr) / np.maximum(sz, 1e-12))) < 4.0
    assert any(b == -1 for r in recs for b in r.branch) and any(b >= 0 for r in recs for b in r.branch)


# --- adjoint oracle -------------------------------------------------------------------

def test_expected_entropy_identity_remix_and_optimum(rng):
    """E(H=0) is E_av of the given set; E(H) >= E_oF for random H (Thm. 2)."""
    w = I.workload_adjoint(seed=1, batch=4, chi=4)
    for b in range(4):
        rho = A.reduced_target(w["theta"][b])
        kr = I.depolarizing_kraus(w["p"][b])
        assert abs(A.expected_entropy(np.zeros((4, 4)), rho, kr) - U.unraveling_entropy(kr, rho)) < 1e-14
        best = U.unraveling_entropy(U.optimal_unraveling(rho, kr)[0], rho)
        for _ in range(10):
            a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
            assert A.expected_entropy(a + a.conj().T, rho, kr) >= best - 1e-12


def test_fd_gradient_directional_consistency(rng):
    """The Hermitian FD gradient predicts directional changes: for random
    Hermitian directions D, Re Tr(Gamma D) matches a 1e-4 step five-point
    derivative of E along D."""
    w = I.workload_adjoint(seed=2, batch=2, chi=4)
    rho = A.reduced_target(w["theta"][0])
    kr = I.depolarizing_kraus(w["p"][0])
    h = w["H"][0]
    g = A.fd_gradient(h, rho, kr)
    assert np.allclose(g, g.conj().T)
    for _ in range(4):
        a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        d = a + a.conj().T
        e = lambda t: A.expected_entropy(h + t * d, rho, kr)
        s = 1e-4
        deriv = (-e(2 * s) + 8 * e(s) - 8 * e(-s) + e(-2 * s)) / (12 * s)
        assert abs(np.trace(g.conj().T @ d).real - deriv) < 1e-7 * max(1.0, abs(deriv))


def test_gradient_descent_approaches_eof():
    """The backtracking descent never raises the cost, stays above the exact
    optimum E_oF, and after 50 steps sits within 2e-4 nats of the brute-force
    minimum over the U(theta, phi) family (a 24 x 24 grid), which itself lies
    within 1e-4 of E_oF for these problems."""
    w = I.workload_adjoint(seed=3, batch=2, chi=4)
    for b in range(2):
        rho = A.reduced_target(w["theta"][b])
        rho = rho / np.trace(rho).real
        kr = I.depolarizing_kraus(w["p"][b])
        _, costs = A.gradient_descent(w["H"][b], rho, kr, steps=50, lr=0.5)
        best = U.unraveling_entropy(U.optimal_unraveling(rho, kr)[0], rho)
        grid = A.grid_search(rho, kr, 24)[0]
        assert np.all(np.diff(costs) <= 1e-15)
        assert costs[-1] <= A.expected_entropy(w["H"][b], rho, kr) + 1e-12
        assert costs[-1] >= best - 1e-12
        assert grid - best < 1e-4
        assert costs[-1] - grid < 2e-4, (costs[-1] - grid, costs[0] - best)


# --- output-distribution sampling and the concentration-improved bound ---------

def test_sequential_conditionals_give_born_probabilities(rng):
    """The product of the sequential conditionals of every bitstring equals its
    Born probability |<x|psi>|^2 (n = 5, random state)."""
    n = 5
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    psi /= np.linalg.norm(psi)
    for x in range(2 ** n):
        bits = [(x >> (n - 1 - k)) & 1 for k in range(n)]
        assert abs(T.bitstring_probability(psi, n, bits) - abs(psi[x]) ** 2) < 1e-15


def test_sampled_bitstrings_follow_born_rule(rng):
    """20000 shots from a random 4-qubit state: total-variation distance to
    |psi|^2 below 0.02 (the expected TV is about 0.01)."""
    n = 4
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    psi /= np.linalg.norm(psi)
    counts = np.zeros(2 ** n)
    for shot in range(20000):
        b = T.sample_bitstring_dense(psi, n, 5, 0, shot)
        counts[int("".join(map(str, b)), 2)] += 1
    tv = 0.5 * np.sum(np.abs(counts / counts.sum() - np.abs(psi) ** 2))
    assert tv < 0.02, tv


def test_trajectory_samples_reproduce_the_noisy_distribution(small):
    """Lemma sampling_reduction: one shot per trajectory samples the mixed
    state; <Z_i> and <Z_i Z_i+1> estimated from 256 trajectories' bits match
    the exact density matrix within 4 standard errors."""
    c = small["circuit"]
    n = c.n_qubits
    rho = T.density_evolution(c)
    zr, zzr = T.density_observables(rho, n)
    bits = np.array([T.sample_bitstring_dense(T.dense_trajectory(c, tr, 0).state, n, 0, tr, 0)
                     for tr in range(256)])
    sgn = 1.0 - 2.0 * bits
    mz, sz = T.trajectory_statistics(sgn)
    mzz, szz = T.trajectory_statistics(sgn[:, :-1] * sgn[:, 1:])
    z = np.concatenate([(mz - zr) / np.maximum(sz, 1e-3), (mzz - zzr) / np.maximum(szz, 1e-3)])
    assert np.max(np.abs(z)) < 4.0, z


def test_concentration_bound_definitions():
    """alpha = 1 gives the plain bound of Thm. 1; weights <= 1 never raise it;
    the depolarizing weight is 1 for recent layers and sqrt(8n)(1-p)^k once
    that drops below 1."""
    c = I.random_brickwork(10, 6, I.depolarizing_kraus(0.05), seed=4)
    rec = T.mps_trajectory(c, 0, 1, 4, cutoff=1e-14)
    assert len(rec.eps_layers) == 6
    assert abs(T.concentrated_bound(rec.eps_layers, "alpha", 1.0, 10) - rec.eps_bound) < 1e-15
    for a in (0.3, 0.7, 0.95):
        assert T.concentrated_bound(rec.eps_layers, "alpha", a, 10) <= rec.eps_bound + 1e-15
    assert T.concentrated_bound(rec.eps_layers, "alpha", 0.5, 10) < T.concentrated_bound(rec.eps_layers, "alpha", 0.9, 10)
    assert T.concentration_weight("depolarizing", 0.3, 0, 10) == 1.0
    k = 40
    assert abs(T.concentration_weight("depolarizing", 0.3, k, 10) - math.sqrt(80.0) * 0.7 ** k) < 1e-18


def test_svd_fallback_gives_the_same_decomposition(monkeypatch):
    """The oracle's split SVD falls back to LAPACK gesvd when gesdd reports
    non-convergence (seen on one x86 LAPACK at chi=128).  The fallback must give
    the same singular values and a valid factorization: u s vh = a, orthonormal
    columns of u."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((40, 24)) + 1j * rng.standard_normal((40, 24))
    ref = np.linalg.svd(a, compute_uv=False)

    def fail(*args, **kw):
        raise np.linalg.LinAlgError("SVD did not converge")

    monkeypatch.setattr(np.linalg, "svd", fail)
    u, s, vh = T._svd(a, full_matrices=False)
    assert np.allclose(s, ref, atol=1e-12)
    assert np.allclose((u * s) @ vh, a, atol=1e-12)
    assert np.allclose(u.conj().T @ u, np.eye(24), atol=1e-12)
    assert np.allclose(T._svd(a, compute_uv=False), ref, atol=1e-12)


# --- the Gram-route bound recorded for the large-bond-dimension tests ----------------

def test_gram_route_bound_closed_forms():
    """gram_route_bound: zero when every kept value is resolved and nothing is
    cut; sqrt of the unresolved kept weight; the Davis-Kahan term tau / gap
    times sqrt(w_chi') at a resolved cut; a full turn (sqrt(w_chi')) when the
    cut falls between equal values."""
    u = 2.0 ** -53
    assert T.gram_route_bound([3.0, 1.0], 2, 4, u) == 0.0
    w = np.array([1.0, 1e-18, 1e-19])
    assert math.isclose(T.gram_route_bound(w, 3, 4, u), math.sqrt((1e-18 + 1e-19) / w.sum()), rel_tol=1e-12)
    w = np.array([1.0, 0.5, 1e-20])
    r = w / w.sum()
    tau = 4 * u * r[0]
    assert math.isclose(T.gram_route_bound(w, 2, 4, u), math.sqrt(r[1]) * tau / (r[1] - r[2]), rel_tol=1e-12)
    w = np.array([1.0, 0.25, 0.25])
    assert math.isclose(T.gram_route_bound(w, 2, 4, u), math.sqrt(0.25 / 1.5), rel_tol=1e-12)


def test_gram_route_bound_holds_for_a_perturbed_gram_matrix(rng):
    """Davis-Kahan, checked: a two-site matrix Theta with a chosen spectrum
    (a resolved cut with a modest gap), its Gram matrix perturbed by a random
    Hermitian E of norm tau = n_g u ||G|| with u = 2^-24, the top chi' vectors
    of the perturbed matrix kept: the truncated state moves by no more than
    the bound (and by a visible amount, so the check is not vacuous)."""
    n, keep, u = 16, 6, 2.0 ** -24
    s = np.sqrt(np.concatenate([np.linspace(1.0, 0.3, keep), [0.3 - 2e-5], np.linspace(0.1, 0.01, n - keep - 1)]))
    qa, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    qb, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    th = (qa * s) @ qb.conj().T
    th /= np.linalg.norm(th)
    g = th @ th.conj().T
    w = np.sort(np.linalg.eigvalsh(g))[::-1]
    tau = n * u * w[0]
    e = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    e = e + e.conj().T
    e *= tau / np.linalg.norm(e, 2)

    def truncated(mat):
        vals, vecs = np.linalg.eigh(mat)
        p = vecs[:, ::-1][:, :keep]
        return p @ (p.conj().T @ th)

    moved = np.linalg.norm(truncated(g + e) - truncated(g))
    bound = T.gram_route_bound(w, keep, n, u)
    assert 0 < moved <= bound, (moved, bound)
    assert moved > 1e-3 * bound


def test_kicked_ising_gates_and_folding():
    """The kicked-Ising circuit family (the chi_max = 512 workload): RZZ(theta)
    = exp(-i theta/2 Z(x)Z) and RX(phi) = exp(-i phi/2 X) against matrix
    exponentials of their generators; and, without noise (coin 0), the circuit
    with each period's RX kicks folded into the next period's even-bond RZZ
    gates (the last period's kicks as a final layer of RX (x) RX) prepares the
    same state as the periods applied as written, RZZ on the even bonds, on the
    odd bonds, then RX on every qubit, with the same angles."""
    from scipy.linalg import expm
    zz = np.kron(np.diag([1.0, -1.0]), np.diag([1.0, -1.0]))
    x = np.array([[0.0, 1.0], [1.0, 0.0]])
    for th in (0.3, math.pi / 4, -1.1):
        assert np.allclose(I.rzz(th), expm(-0.5j * th * zz), atol=1e-14)
        assert np.allclose(I.rx(th), expm(-0.5j * th * x), atol=1e-14)
    n, depth, seed = 6, 3, 7
    circ = I.kicked_ising(n, depth, I.depolarizing_kraus(1.0), 0.0, seed)
    assert len(circ.layers) == 2 * depth + 1 and circ.layers[-1].coin_p == 0.0
    psi = np.zeros(2 ** n, complex)
    psi[0] = 1.0
    for layer in circ.layers:
        for q, g in zip(layer.left_qubits, layer.gates):
            psi = T.apply_2q(psi, g, int(q), n)
    # the same angles, drawn in the generator's order, applied as written
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4B49, n, depth]))
    ref = np.zeros(2 ** n, complex)
    ref[0] = 1.0
    for _ in range(depth):
        for sub in range(2):
            for q in I.brickwork_bonds(n, sub):
                ref = T.apply_2q(ref, I.rzz(math.pi / 4 + 0.05 * rng.standard_normal()), int(q), n)
        for q in range(n):
            ref = T.apply_1q(ref, I.rx(rng.uniform(0.0, math.pi)), q, n)
    assert np.allclose(psi, ref, atol=1e-12)
