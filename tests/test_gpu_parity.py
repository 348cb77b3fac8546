"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs and Philox stream.  Tolerances: FP64 mode 1e-10 per
trajectory on observables and states, relative to the observable's scale (1
for <Z>, <ZZ> and the entropy in nats; the value itself for the error bound,
with an absolute floor set by the FP64 residual of the discarded weight);
mixed mode 1e-4 per trajectory; trajectory averages of mixed and FP64 within 3
combined standard errors, and averages within 4 standard errors of exact
density-matrix evolution."""
import concurrent.futures
import math
import multiprocessing
import os

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import trajectories as T
from oracle import unravel as U
from paper_2508_05745_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_05745_gb300 import build, lemps
    build.build()
    return lemps


def run_gpu(L, circ, chi, n_traj, seed, precision="fp64", unravel="optimal", cutoff=None, traj_offset=0,
            layering="local", eigvec_fp64=False, big_kernels=False):
    sim = L.Simulation(circ.n_qubits, chi, n_traj, seed=seed, precision=precision, unravel=unravel,
                       cutoff=cutoff, log_capacity=circ.n_gates, traj_offset=traj_offset, layering=layering,
                       eigvec_fp64=eigvec_fp64, big_kernels=big_kernels)
    sim.run(circ)
    res = sim.measure()
    branches = np.zeros((n_traj, 2 * circ.n_gates), dtype=np.int32)
    for g in range(circ.n_gates):
        for s in range(2):
            branches[:, 2 * g + s] = sim.sample_branch(g, s)
    return sim, res, branches


def contract(tensors):
    psi = tensors[0].reshape(2, -1)
    for t in tensors[1:]:
        psi = np.einsum('xa,asb->xsb', psi, t).reshape(-1, t.shape[2])
    return psi.reshape(-1)


# --- K-c: the unraveling kernel ---------------------------------------------------

CHANNELS = {
    "depolarizing": I.depolarizing_kraus(0.02),
    "full_depolarizing": I.depolarizing_kraus(1.0),
    "amplitude_damping": I.amplitude_damping_kraus(0.3),
    "dephasing": I.dephasing_kraus(0.25),
    "ad_then_dephasing": I.compose_kraus(I.dephasing_kraus(0.01), I.amplitude_damping_kraus(0.01)),
    "depolarizing_strong": I.depolarizing_kraus(0.7),
}


@pytest.mark.parametrize("name", list(CHANNELS))
def test_unravel_opt_matches_oracle(L, name):
    rng = np.random.default_rng(7)
    kraus = CHANNELS[name]
    rhos = []
    for i in range(300):
        a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        r = a @ a.conj().T
        rhos.append(r / np.trace(r).real * (0.5 + i % 3))     # any trace
    rhos += [np.eye(2) / 2, np.diag([1.0, 0.0]), np.diag([0.7, 0.3]) + 0j]
    rho = np.stack(rhos).astype(np.complex128)
    kout, e_av = L.unravel_opt(torch.from_numpy(rho).cuda(), torch.from_numpy(kraus).cuda())
    kout, e_av = kout.cpu().numpy(), e_av.cpu().numpy()
    for b in range(len(rho)):
        rn = rho[b] / np.trace(rho[b]).real
        ref, _ = U.optimal_unraveling(rn, kraus)
        assert np.allclose(kout[b], ref[:4], atol=1e-10), (name, b)
        assert abs(e_av[b] - U.unraveling_entropy(ref, rn)) < 1e-12
        assert np.allclose(sum(k.conj().T @ k for k in kout[b]), np.eye(2), atol=1e-12)


# --- full path, exact bond dimension -------------------------------------------------

@pytest.fixture(scope="module")
def small_exact(L):
    w = I.workload_small_exact(seed=0)
    sim, res, br = run_gpu(L, w["circuit"], 16, 256, seed=0)
    states = [contract(sim.export_mps(t)[0]) for t in range(24)]
    sim.destroy()
    return w, res, br, states


def test_small_exact_per_trajectory_fp64(small_exact):
    """n=8 depth-8 depolarizing brickwork, chi=16 (no truncation): every checked
    trajectory has the oracle's branch sequence and state to 1e-10."""
    w, res, br, states = small_exact
    assert res["n_failed"] == 0
    for t in range(24):
        ref = T.dense_trajectory(w["circuit"], t, 0)
        assert list(br[t]) == ref.branch
        assert abs(abs(np.vdot(ref.state, states[t])) - 1.0) < 1e-10
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)
        assert np.allclose(res["zz"][t], ref.zz, atol=1e-10)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-10
    assert np.all(res["eps_bound"] == 0.0)


@pytest.mark.slow
def test_small_exact_averages_match_density_matrix(small_exact):
    w, res, _, _ = small_exact
    rho = T.density_evolution(w["circuit"])
    zr, zzr = T.density_observables(rho, 8)
    z = np.concatenate([(res["z_mean"] - zr) / res["z_stderr"], (res["zz_mean"] - zzr) / res["zz_stderr"]])
    assert np.max(np.abs(z)) < 4.0, z
    m, s = T.trajectory_statistics(res["z"])
    assert np.allclose(m, res["z_mean"], atol=1e-13) and np.allclose(s, res["z_stderr"], atol=1e-13)


def test_small_exact_mixed_precision(L, small_exact):
    """Mixed mode (complex64 storage and contractions, FP64 eigensolver):
    trajectories with the same branch sequence agree with the FP64 oracle to
    1e-4."""
    w, res64, br64, _ = small_exact
    sim, res, br = run_gpu(L, w["circuit"], 16, 256, seed=0, precision="mixed")
    sim.destroy()
    same = np.all(br == br64, axis=1)
    assert same.mean() > 0.95
    for t in np.nonzero(same)[0][:64]:
        ref = T.dense_trajectory(w["circuit"], int(t), 0)
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-4)
        assert np.allclose(res["zz"][t], ref.zz, atol=1e-4)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-4


# --- truncation, uneven bond dimensions ---------------------------------------------

def close(a, b, tol, scale=1.0):
    """|a - b| <= tol * max(|b|, scale), elementwise."""
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), scale))


def bound_tol(ref_bound, precision):
    """Error-bound tolerance.  FP64: 1e-10 relative; the discarded weight of a
    split is the FP64 residual ||Theta - U U^dagger Theta||^2, accurate to a
    few eps_64 of ||Theta||^2, and each layer adds 4 sqrt(2 sum eps), whose
    derivative 2 sqrt(2) / sqrt(sum eps) is at most ~1e8 for the layers where
    anything is discarded, hence the 1e-8 * eps_64-level floor of 1e-12 per
    layer.  Mixed: 1e-4 like the observables."""
    if precision == "mixed":
        return 1e-4 * max(1.0, abs(ref_bound))
    return 1e-10 * abs(ref_bound) + 1e-12 * 10


def mixed_tol(ref):
    """Per-trajectory tolerance of the mixed path against the FP64 oracle.

    Complex64 storage and arithmetic perturb each two-site Gram matrix by
    about eps_32 ||G|| (a few roundings per entry and gate), and the kept
    subspace of a truncating split then turns by about that perturbation over
    the relative gap of the squared Schmidt values at the cut (Davis-Kahan);
    the oracle records those gaps.  So the 1e-4 bar holds wherever every cut
    of the trajectory has a relative gap of at least 1e-2, and a trajectory
    with a closer cut gets 1e-6 / (its smallest gap)."""
    g = min(ref.cut_gaps) if ref.cut_gaps else 1.0
    return max(1e-4, 1e-6 / max(g, 1e-300))


@pytest.mark.parametrize("precision,tol,vec64", [("fp64", 1e-10, True), ("mixed", 1e-4, False), ("mixed", 1e-4, True)])
def test_truncated_run_matches_oracle_mps(L, precision, tol, vec64):
    """Heavy truncation (chi=4, cutoff 1e-14) on a 10-qubit depolarizing
    brickwork: every trajectory has the oracle's branch sequence, and its
    observables and error bound match the oracle's FP64 MPS trajectory (FP64:
    1e-10; mixed: 1e-4, or 1e-6 over the smallest relative cut gap where the
    cut falls between close Schmidt values, see mixed_tol).  The Gram
    eigensolve is FP64 in both modes; the mixed mode is run with its kept
    eigenvectors back-transformed in complex64 (default) and in FP64."""
    circ = I.random_brickwork(10, 10, I.depolarizing_kraus(0.05), seed=4)
    n_traj = 16
    sim, res, br = run_gpu(L, circ, 4, n_traj, seed=3, precision=precision, cutoff=1e-14, eigvec_fp64=vec64)
    sim.destroy()
    errs = []
    loose = 0
    for t in range(n_traj):
        ref = T.mps_trajectory(circ, t, 3, chi_max=4, cutoff=1e-14)
        assert list(br[t]) == ref.branch, t
        if precision == "mixed":
            tol = mixed_tol(ref)
            loose += tol > 1e-4
        errs.append(max(np.abs(res["z"][t] - ref.z).max(), np.abs(res["zz"][t] - ref.zz).max(),
                        abs(res["s_half"][t] - ref.s_half)))
        assert close(res["z"][t], ref.z, tol), (t, errs[-1])
        assert close(res["zz"][t], ref.zz, tol), (t, errs[-1])
        assert close(res["s_half"][t], ref.s_half, tol), (t, errs[-1])
        assert abs(res["eps_bound"][t] - ref.eps_bound) <= bound_tol(ref.eps_bound, precision), \
            (t, res["eps_bound"][t], ref.eps_bound)
    print(f"{precision}: max observable error {max(errs):.3e}; trajectories with a cut gap below 1e-2: {loose}")
    assert res["eps_hat"] > 0


@pytest.mark.slow
def test_ad_dephasing_n32_chi64(L):
    """The AD-then-dephasing workload (n=32, depth 20, chi=64): FP64 GPU
    trajectories equal the oracle MPS trajectories to 1e-10; mixed mode has
    the same branch sequences and matches within 1e-4."""
    w = I.workload_ad_dephasing(seed=0, n_traj=3)
    circ = w["circuit"]
    sim, res, br = run_gpu(L, circ, 64, 3, seed=0)
    sim.destroy()
    simm, resm, brm = run_gpu(L, circ, 64, 3, seed=0, precision="mixed")
    simm.destroy()
    for t in range(2):
        ref = T.mps_trajectory(circ, t, 0, chi_max=64, cutoff=1e-20)
        assert list(br[t]) == ref.branch
        assert close(res["z"][t], ref.z, 1e-10)
        assert close(res["zz"][t], ref.zz, 1e-10)
        assert close(res["s_half"][t], ref.s_half, 1e-10)
        assert abs(res["eps_bound"][t] - ref.eps_bound) <= bound_tol(ref.eps_bound, "fp64")
        assert list(brm[t]) == ref.branch
        assert close(resm["z"][t], ref.z, 1e-4)
        assert close(resm["zz"][t], ref.zz, 1e-4)
        assert close(resm["s_half"][t], ref.s_half, 1e-4)


def test_ad_dephasing_config_against_cpp_oracle(L):
    """The AD-then-dephasing configuration at its shape (n=32, depth 20,
    chi=64, composed 4-Kraus channel), 32 trajectories against the C++ FP64
    oracle on the same Philox streams: every branch sequence equal; FP64
    observables and error bounds to 1e-10; mixed observables to 1e-4, or to
    1e-6 over the trajectory's smallest relative cut gap where a truncation
    falls between close Schmidt values (the conditioning reading of the mixed
    tolerance)."""
    from oracle import cpp
    w = I.workload_ad_dephasing(seed=0, n_traj=32)
    circ = w["circuit"]
    n_traj = 32
    ref = cpp.mps_trajectories(circ, 0, n_traj, 0, 64, 1e-20)
    sim, res, br = run_gpu(L, circ, 64, n_traj, seed=0)
    sim.destroy()
    simm, resm, brm = run_gpu(L, circ, 64, n_traj, seed=0, precision="mixed")
    simm.destroy()
    worst64 = worstm = 0.0
    loose = 0
    for t in range(n_traj):
        assert list(br[t]) == list(ref["branch"][t]), t
        assert list(brm[t]) == list(ref["branch"][t]), t
        e64 = max(np.abs(res["z"][t] - ref["z"][t]).max(), np.abs(res["zz"][t] - ref["zz"][t]).max(),
                  abs(res["s_half"][t] - ref["s_half"][t]))
        assert e64 < 1e-10, (t, e64)
        assert abs(res["eps_bound"][t] - ref["eps_bound"][t]) <= bound_tol(ref["eps_bound"][t], "fp64")
        tol = max(1e-4, 1e-6 / max(ref["min_gap"][t], 1e-300))
        loose += tol > 1e-4
        em = max(np.abs(resm["z"][t] - ref["z"][t]).max(), np.abs(resm["zz"][t] - ref["zz"][t]).max(),
                 abs(resm["s_half"][t] - ref["s_half"][t]))
        assert em < tol, (t, em, tol)
        worst64, worstm = max(worst64, e64), max(worstm, em)
    print(f"config 2 vs C++ oracle: FP64 worst {worst64:.2e}, mixed worst {worstm:.2e}, "
          f"trajectories with a cut gap below 1e-2: {loose}")


@pytest.mark.parametrize("chi", [100, 127])
def test_mixed_non_power_of_two_chi_against_cpp_oracle(L, chi):
    """Mixed mode at chi_max = 100 (even site capacities of 100: the tensor-core
    contraction with ragged tile boxes, K chunks past the slot width) and
    chi_max = 127 (odd capacities: the SIMT contraction), n = 18, depth 12,
    8 trajectories, against the C++ FP64 oracle: the same branches, and
    observables within 1e-4 (or 1e-6 over the smallest relative cut gap)."""
    from oracle import cpp
    circ = I.random_brickwork(18, 12, I.depolarizing_kraus(0.05), seed=11)
    n_traj = 8
    ref = cpp.mps_trajectories(circ, 0, n_traj, 4, chi, 1e-12)
    sim, res, br = run_gpu(L, circ, chi, n_traj, seed=4, precision="mixed", cutoff=1e-12)
    _, bonds = sim.export_mps(0)
    sim.destroy()
    assert bonds.max() == chi
    worst = 0.0
    for t in range(n_traj):
        assert list(br[t]) == list(ref["branch"][t]), t
        tol = max(1e-4, 1e-6 / max(ref["min_gap"][t], 1e-300))
        e = max(np.abs(res["z"][t] - ref["z"][t]).max(), np.abs(res["zz"][t] - ref["zz"][t]).max(),
                abs(res["s_half"][t] - ref["s_half"][t]))
        assert e < tol, (t, e, tol)
        worst = max(worst, e)
    print(f"chi={chi}: mixed worst {worst:.2e}")


def test_coin_noise_full_depolarizing(L):
    """Two-qubit depolarizing reading: with probability p both qubits are fully
    depolarized (optimal unraveling of each), otherwise nothing happens."""
    circ = I.random_brickwork(12, 8, I.depolarizing_kraus(1.0), seed=6, coin_p=0.3)
    sim, res, br = run_gpu(L, circ, 16, 16, seed=9, cutoff=1e-14)
    sim.destroy()
    for t in range(16):
        ref = T.mps_trajectory(circ, t, 9, chi_max=16, cutoff=1e-14)
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-9)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-9
    assert (br == -1).any() and (br >= 0).any()


def test_given_unraveling_mode(L):
    circ = I.random_brickwork(6, 6, I.amplitude_damping_kraus(0.2), seed=2)
    sim, res, br = run_gpu(L, circ, 8, 8, seed=1, unravel="given")
    sim.destroy()
    for t in range(8):
        ref = T.dense_trajectory(circ, t, 1, mode="given")
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)


@pytest.mark.parametrize("kraus", [I.depolarizing_kraus(0.05), I.amplitude_damping_kraus(0.2),
                                   I.dephasing_kraus(0.3)], ids=["depolarizing", "amp_damping", "dephasing"])
def test_haar_optimal_mode(L, kraus):
    """Fixed Haar-optimal unraveling (Sec. V.B): the library remixes the Kraus
    set once for the Bell state and samples it as given; per trajectory equal
    to the oracle's dense trajectory in the same mode (FP64)."""
    circ = I.random_brickwork(6, 6, kraus, seed=5)
    sim, res, br = run_gpu(L, circ, 8, 8, seed=3, unravel="haar_optimal")
    sim.destroy()
    for t in range(8):
        ref = T.dense_trajectory(circ, t, 3, mode="haar_optimal")
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)
        assert np.allclose(res["zz"][t], ref.zz, atol=1e-10)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-10


def test_projective_depolarizing_given_mode(L):
    """The five-operator Projective depolarizing set (appendix on common
    unravelings) sampled as given, per trajectory against the oracle."""
    circ = I.random_brickwork(6, 6, I.projective_depolarizing_kraus(0.1), seed=6)
    sim, res, br = run_gpu(L, circ, 8, 8, seed=2, unravel="given")
    sim.destroy()
    for t in range(8):
        ref = T.dense_trajectory(circ, t, 2, mode="given")
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-10


def test_fixed_mode_inputs_are_validated(L):
    """More than four operators only in the given mode; unknown mode names fail."""
    five = I.Layer(np.array([0], np.int32), np.eye(4, dtype=complex)[None], I.projective_depolarizing_kraus(0.1))
    for mode in ("optimal", "haar_optimal"):
        sim = L.Simulation(4, 4, 2, unravel=mode)
        with pytest.raises(L.LempsError) as e:
            sim.apply_layer(five)
        assert e.value.status == L.LEMPS_EINVAL
        sim.destroy()
    with pytest.raises(ValueError):
        L.Simulation(4, 4, 2, unravel="projective")


def test_global_layering_with_truncation(L):
    """Global layering (all gates, all noise, then a truncation sweep; Sec.
    IV.A) with chi_max below the exact rank: per trajectory equal to the
    oracle's MPS trajectory in the same layering (FP64), error bound included."""
    circ = I.random_brickwork(10, 6, I.depolarizing_kraus(0.05), seed=4)
    sim, res, br = run_gpu(L, circ, 4, 8, seed=1, cutoff=1e-14, layering="global")
    sim.destroy()
    for t in range(8):
        ref = T.mps_trajectory(circ, t, 1, 4, cutoff=1e-14, layering="global")
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-9)
        assert np.allclose(res["zz"][t], ref.zz, atol=1e-9)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-9
        assert abs(res["eps_bound"][t] - ref.eps_bound) < 1e-9
    assert res["eps_bound"].max() > 0.0


def test_global_layering_without_truncation(L):
    """chi >= 2^{n/2}: the global layering equals the dense trajectory (and,
    since the pairs of a layer are disjoint, the local layering)."""
    circ = I.workload_small_exact(seed=0)["circuit"]
    sim, res, br = run_gpu(L, circ, 16, 8, seed=0, layering="global")
    sim.destroy()
    _, loc, brl = run_gpu(L, circ, 16, 8, seed=0)
    for t in range(8):
        ref = T.dense_trajectory(circ, t, 0, layering="global")
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-10
    assert np.array_equal(br, brl)
    assert np.allclose(res["z"], loc["z"], atol=1e-10)


def test_global_layering_limits(L):
    with pytest.raises(L.LempsError) as e:
        L.Simulation(8, 128, 2, layering="global")
    assert e.value.status == L.LEMPS_EINVAL
    with pytest.raises(ValueError):
        L.Simulation(8, 16, 2, layering="sideways")


def test_sample_bitstrings_match_oracle(L):
    """Output-distribution sampling (Lemma sampling_reduction), FP64: every
    shot's bitstring equals the oracle's sequential sampling of the same
    trajectory's dense state on the same Philox counters."""
    circ = I.workload_small_exact(seed=0)["circuit"]
    sim, res, br = run_gpu(L, circ, 16, 8, seed=3)
    bits = sim.sample_bitstrings(4)
    bits2 = sim.sample_bitstrings(4)
    sim.destroy()
    assert np.array_equal(bits, bits2)     # same counters, same state
    n = circ.n_qubits
    for t in range(8):
        psi = T.dense_trajectory(circ, t, 3).state
        for shot in range(4):
            assert np.array_equal(bits[t, shot], T.sample_bitstring_dense(psi, n, 3, t, shot))


def test_sample_bitstrings_reproduce_the_noisy_distribution(L):
    """Mixed precision, one shot per trajectory over 512 trajectories: <Z_i>
    and <Z_i Z_i+1> from the bits match exact density-matrix evolution within
    4 standard errors."""
    circ = I.workload_small_exact(seed=0)["circuit"]
    sim, _, _ = run_gpu(L, circ, 16, 512, seed=6, precision="mixed")
    bits = sim.sample_bitstrings(1)[:, 0, :]
    sim.destroy()
    rho = T.density_evolution(circ)
    zr, zzr = T.density_observables(rho, circ.n_qubits)
    sgn = 1.0 - 2.0 * bits
    mz, sz = T.trajectory_statistics(sgn)
    mzz, szz = T.trajectory_statistics(sgn[:, :-1] * sgn[:, 1:])
    z = np.concatenate([(mz - zr) / np.maximum(sz, 1e-3), (mzz - zzr) / np.maximum(szz, 1e-3)])
    assert np.max(np.abs(z)) < 4.0, z


def test_eps_concentrated_matches_oracle(L):
    """Concentration-improved bound (Sec. III.C): per trajectory equal to the
    oracle's weighting of its per-layer errors; alpha = 1 is the plain bound."""
    circ = I.random_brickwork(10, 6, I.depolarizing_kraus(0.05), seed=4)
    sim, res, _ = run_gpu(L, circ, 4, 8, seed=1, cutoff=1e-14)
    e1, _ = sim.eps_concentrated("alpha", 1.0)
    ea, ha = sim.eps_concentrated("alpha", 0.7)
    ed, _ = sim.eps_concentrated("depolarizing", 0.05)
    with pytest.raises(L.LempsError) as e:
        sim.eps_concentrated("alpha", 0.0)
    assert e.value.status == L.LEMPS_EINVAL
    with pytest.raises(L.LempsError):
        sim.sample_bitstrings(0)
    sim.destroy()
    assert np.allclose(e1, res["eps_bound"], atol=1e-12)
    assert abs(ha - ea.mean()) < 1e-15
    for t in range(8):
        ref = T.mps_trajectory(circ, t, 1, 4, cutoff=1e-14)
        assert abs(ea[t] - T.concentrated_bound(ref.eps_layers, "alpha", 0.7, 10)) < 1e-9
        assert abs(ed[t] - T.concentrated_bound(ref.eps_layers, "depolarizing", 0.05, 10)) < 1e-9
    assert (ea <= e1 + 1e-15).all() and ea.max() > 0.0


def test_traj_offset_shards_reproduce_the_full_run(L):
    """Trajectory ids key the Philox counter, so two shards reproduce one run."""
    circ = I.random_brickwork(6, 4, I.depolarizing_kraus(0.05), seed=8)
    _, full, _ = run_gpu(L, circ, 8, 8, seed=4)
    _, a, _ = run_gpu(L, circ, 8, 4, seed=4)
    _, b, _ = run_gpu(L, circ, 8, 4, seed=4, traj_offset=4)
    assert np.array_equal(np.concatenate([a["z"], b["z"]]), full["z"])


# --- degenerate entanglement spectrum ---------------------------------------------------

def nested_bell_circuit(n_pairs):
    """2 n_pairs qubits; pair i (qubits i, 2 n_pairs - 1 - i) in a Bell state for
    every i, so all n_pairs pairs cross the middle bond: its Schmidt spectrum
    is 2^n_pairs equal values and S(n/2) = n_pairs ln 2.  Each pair is made
    on the middle bond (H, then CNOT) and swapped outwards; no noise (the
    identity as the one Kraus operator, sampled as given)."""
    n = 2 * n_pairs
    mid = n_pairs - 1
    h = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    bell = cnot @ np.kron(h, np.eye(2))
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    ident = np.eye(2, dtype=complex)[None]
    layers = []
    for r in range(n_pairs):
        layers.append(I.Layer(np.array([mid], np.int32), bell[None], ident))
        target = r   # the pair moves out to (r, n - 1 - r)
        for step in range(mid - target):
            a, b = mid - 1 - step, mid + 1 + step
            layers.append(I.Layer(np.array([a, b], np.int32), np.stack([swap, swap]), ident))
    return I.Circuit(n, layers)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_half_chain_entropy_of_a_flat_spectrum(L, precision, tol):
    """Six Bell pairs across the middle bond: 64 equal Schmidt values, S(n/2) =
    6 ln 2 and <Z_i> = 0 exactly (a closed form; the eigensolver meets an
    eigenvalue of multiplicity 64)."""
    circ = nested_bell_circuit(6)
    sim = L.Simulation(12, 64, 4, seed=1, precision=precision, unravel="given")
    sim.run(circ)
    res = sim.measure()
    sim.destroy()
    assert res["n_failed"] == 0
    assert np.allclose(res["s_half"], 6 * np.log(2), atol=tol, rtol=0), res["s_half"] - 6 * np.log(2)
    assert np.allclose(res["z"], 0.0, atol=tol)


# --- waves ------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_waves_equal_one_big_handle(L, precision):
    """Waves (max_traj_in_flight = 8 of 20 trajectories: waves of 8, 8 and 4)
    give the results of one handle holding all 20, per trajectory bit for bit
    (global trajectory ids key the Philox counters), means and standard errors
    to rounding; a layer applied after a measurement reaches every wave."""
    circ = I.random_brickwork(8, 6, I.depolarizing_kraus(0.05), seed=3)
    extra = I.random_brickwork(8, 7, I.depolarizing_kraus(0.05), seed=3).layers[6]
    cut = 1e-14 if precision == "fp64" else 1e-12
    one = L.Simulation(8, 8, 20, seed=7, precision=precision, cutoff=cut, traj_offset=5)
    wav = L.Simulation(8, 8, 20, seed=7, precision=precision, cutoff=cut, traj_offset=5, max_traj_in_flight=8)
    assert one.waves() == (20, 1) and wav.waves() == (8, 3)
    for step in range(2):
        if step == 0:
            one.run(circ)
            wav.run(circ)
        else:
            one.apply_layer(extra)
            wav.apply_layer(extra)
        a, b = one.measure(), wav.measure()
        for key in ("z", "zz", "s_half", "eps_bound", "status"):
            assert np.array_equal(a[key], b[key]), (step, key)
        for key in ("z_mean", "z_stderr", "zz_mean", "zz_stderr"):
            assert np.allclose(a[key], b[key], rtol=1e-12, atol=1e-14), (step, key)
        for key in ("s_half_mean", "s_half_stderr", "eps_hat", "eps_buffer"):
            assert abs(a[key] - b[key]) <= 1e-12 * max(1.0, abs(a[key])), (step, key)
        assert a["eps_hat"] > 0
    with pytest.raises(L.LempsError) as e:
        wav.export_mps(0)
    assert e.value.status == L.LEMPS_ESTATE
    one.destroy()
    wav.destroy()


# --- GEMM tile autotuner ----------------------------------------------------------------

TILE_SHAPES = {"fp64": [(64, 64), (32, 64), (64, 32), (32, 32)],
               "mixed": [(64, 64), (128, 64), (64, 128), (32, 32)]}


@pytest.mark.parametrize("precision,n,chi", [("fp64", 12, 40), ("mixed", 16, 100)])
def test_gemm_tiles_give_identical_results(L, precision, n, chi):
    """Every GEMM tile shape the autotuner can pick (gemm_tile = 1..4) and the
    autotuned choice (gemm_tile = 0) give the same run bit for bit: branch
    sequences, observables, error bounds and MPS tensors.  The circuit (depth
    9 Haar brickwork, depolarizing p = 0.05) drives the middle bonds to chi, so
    the products span several tiles of every shape with ragged edges: Gram
    sides up to 80 (FP64, chi = 40) and 200 (mixed, chi = 100, where the
    middle contractions run on the tensor cores and the outer ones on the
    SIMT kernel)."""
    circ = I.random_brickwork(n, 9, I.depolarizing_kraus(0.05), seed=5)
    runs = []
    for tile in range(5):
        sim = L.Simulation(n, chi, 24, seed=9, precision=precision, log_capacity=circ.n_gates, gemm_tile=tile)
        sim.run(circ)
        res = sim.measure()
        br = np.array([sim.sample_branch(g, s) for g in range(circ.n_gates) for s in range(2)])
        mps = [sim.export_mps(t) for t in (0, 11, 23)]
        tiles = sim.tiles()
        sim.destroy()
        assert res["n_failed"] == 0
        runs.append((res, br, mps, tiles))
    assert max(b.max() for _, b in runs[0][2]) == chi
    shapes = TILE_SHAPES[precision]
    for tile, (res, br, mps, tiles) in enumerate(runs):
        for kind in ("contract", "gram_left", "gram_right"):
            got = {tuple(x) for x in tiles[kind] if tuple(x) != (0, 0)}
            assert got, (tile, kind)
            assert got <= set(shapes), (tile, kind, got)
            if tile > 0:
                assert got == {shapes[tile - 1]}, (tile, kind, got)
        if precision == "mixed":
            assert (tiles["contract"] == 0).all(axis=1).any()   # tensor-core positions
        if tile == 0:
            continue
        ref_res, ref_br, ref_mps, _ = runs[0]
        assert np.array_equal(br, ref_br), tile
        for key in ("z", "zz", "s_half", "eps_bound", "status", "z_mean", "zz_mean"):
            assert np.array_equal(res[key], ref_res[key]), (tile, key)
        for (ts, bonds), (rts, rbonds) in zip(mps, ref_mps):
            assert np.array_equal(bonds, rbonds), tile
            for a, b in zip(ts, rts):
                assert np.array_equal(a, b), tile


def test_autotuner_reuses_its_record(L):
    """The autotuner times each (kernel, capacity triple) once per process:
    a second handle with the same capacities, precision and batch class
    spends no time tuning and gets the same tiles."""
    a = L.Simulation(10, 24, 16, seed=1, precision="fp64")
    b = L.Simulation(10, 24, 16, seed=2, precision="fp64")
    ta, tb = a.tiles(), b.tiles()
    a.destroy()
    b.destroy()
    assert tb["tune_ms"] == 0.0
    for kind in ("contract", "gram_left", "gram_right"):
        assert np.array_equal(ta[kind], tb[kind]), kind
        assert {tuple(x) for x in ta[kind]} <= set(TILE_SHAPES["fp64"])


@pytest.mark.slow
def test_runs_are_deterministic_at_chi128(L):
    """At the benchmark's bond dimension (chi = 128, Gram matrices of 256, so
    the eigensolver runs both its blocked and its packed phase) a run is
    reproducible bit for bit: two handles with the same configuration give
    the same MPS tensors, observables and error bounds, and so does a handle
    that holds the same 12 trajectories in three waves (5, 5 and 2)."""
    circ = I.random_brickwork(16, 12, I.depolarizing_kraus(0.02), seed=8)
    out = []
    for wave in (0, 0, 5):
        sim = L.Simulation(16, 128, 12, seed=4, precision="mixed", max_traj_in_flight=wave)
        sim.run(circ)
        res = sim.measure()
        mps = sim.export_mps(3) if wave == 0 else None
        sim.destroy()
        assert res["n_failed"] == 0
        out.append((res, mps))
    assert out[0][1][1].max() == 128
    for res, _ in out[1:]:
        for key in ("z", "zz", "s_half", "eps_bound", "status"):
            assert np.array_equal(res[key], out[0][0][key]), key
    for a, b in zip(out[0][1][0], out[1][1][0]):
        assert np.array_equal(a, b)


# --- edge cases ---------------------------------------------------------------------

def test_two_qubits_single_trajectory(L):
    circ = I.random_brickwork(2, 5, I.depolarizing_kraus(0.1), seed=3)
    sim, res, br = run_gpu(L, circ, 2, 1, seed=2)
    sim.destroy()
    ref = T.dense_trajectory(circ, 0, 2)
    assert list(br[0]) == ref.branch
    assert np.allclose(res["z"][0], ref.z, atol=1e-10)


def test_odd_n_and_empty_layer(L):
    circ = I.random_brickwork(7, 5, I.depolarizing_kraus(0.05), seed=5)
    circ.layers.insert(2, I.Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4), complex), I.depolarizing_kraus(0.05)))
    sim, res, br = run_gpu(L, circ, 8, 4, seed=6)
    sim.destroy()
    for t in range(4):
        ref = T.dense_trajectory(circ, t, 6)
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)


def test_invalid_inputs_are_rejected(L):
    sim = L.Simulation(4, 4, 2, log_capacity=4)
    bad_kraus = I.Layer(np.array([0], np.int32), np.eye(4, dtype=complex)[None], 1.1 * I.depolarizing_kraus(0.1))
    with pytest.raises(L.LempsError) as e:
        sim.apply_layer(bad_kraus)
    assert e.value.status == L.LEMPS_EINVAL
    overlap = I.Layer(np.array([0, 1], np.int32), np.stack([np.eye(4, dtype=complex)] * 2), I.depolarizing_kraus(0.1))
    with pytest.raises(L.LempsError):
        sim.apply_layer(overlap)
    with pytest.raises(L.LempsError) as e:
        sim.sample_branch(0, 0)
    assert e.value.status == L.LEMPS_ESTATE
    sim.destroy()
    with pytest.raises(L.LempsError):
        L.Simulation(4, 0, 2)
    with pytest.raises(L.LempsError):
        L.Simulation(4, 513, 2)
    big = L.Simulation(20, 512, 1)
    with pytest.raises(L.LempsError) as e:
        big.sample_bitstrings(1)   # the sampler holds bonds of at most 256
    assert e.value.status == L.LEMPS_EINVAL
    big.destroy()


# --- differentiation --------------------------------------------------------------------

@pytest.mark.parametrize("chi,dtype", [(8, np.complex128), (64, np.complex128), (64, np.complex64)])
def test_unravel_grad_matches_oracle(L, chi, dtype):
    w = I.workload_adjoint(seed=11, batch=48, chi=chi, dtype=dtype)
    th = torch.from_numpy(w["theta"]).cuda()
    p = torch.from_numpy(w["p"]).cuda()
    h = torch.from_numpy(w["H"]).cuda()
    cost, grad, rho = L.unravel_grad(th, p, h)
    cost, grad, rho = cost.cpu().numpy(), grad.cpu().numpy(), rho.cpu().numpy()
    tol_rho = 1e-13 if dtype == np.complex128 else 1e-6
    for b in range(0, 48, 3):
        ref_rho = A.reduced_target(w["theta"][b].astype(np.complex128))
        ref_rho /= np.trace(ref_rho).real
        assert np.allclose(rho[b], ref_rho, atol=tol_rho)
        kr = I.depolarizing_kraus(w["p"][b])
        assert abs(cost[b] - A.expected_entropy(w["H"][b], rho[b], kr)) < 1e-12
        fd = A.fd_gradient(w["H"][b], rho[b], kr)
        assert np.allclose(grad[b], fd, atol=1e-7 * max(1.0, np.abs(fd).max())), (b, np.abs(grad[b] - fd).max())


def test_descent_on_device_approaches_optimum(L):
    """50 on-device gradient steps (backtracking step size) from random
    unitaries: the cost never rises, never goes below the exact optimum
    E_oF, follows the oracle's descent for the first five steps, and ends
    within 2e-4 nats of the brute-force minimum over the U(theta, phi) family
    on a 24 x 24 grid (chi = 8)."""
    w = I.workload_adjoint(seed=12, batch=32, chi=8)
    th = torch.from_numpy(w["theta"]).cuda()
    p = torch.from_numpy(w["p"]).cuda()
    h = torch.from_numpy(w["H"]).cuda()
    cost0, _, rho = L.unravel_grad(th, p, h, want_grad=False)
    hn, trace = L.unravel_descend(rho, p, h, steps=50, lr=0.5)
    trace = trace.cpu().numpy()
    rho = rho.cpu().numpy()
    cost0 = cost0.cpu().numpy()
    for b in range(32):
        kr = I.depolarizing_kraus(w["p"][b])
        eof = U.unraveling_entropy(U.optimal_unraveling(rho[b], kr)[0], rho[b])
        assert trace[-1, b] >= eof - 1e-12
        assert trace[-1, b] <= cost0[b] + 1e-12
        assert np.all(np.diff(trace[:, b]) <= 1e-15)
        if b < 8:
            grid = A.grid_search(rho[b], kr, 24)[0]
            assert grid >= eof - 1e-12      # the brute-force family is bounded by the optimum too
            assert trace[-1, b] - grid < 2e-4, (b, trace[-1, b] - grid, cost0[b] - eof)
        if b < 4:
            _, ref_costs = A.gradient_descent(w["H"][b], rho[b], kr, steps=5, lr=0.5)
            assert np.allclose(trace[:5, b], ref_costs, atol=1e-6)


def test_autograd_function_backward(L):
    w = I.workload_adjoint(seed=13, batch=4, chi=8)
    th = torch.from_numpy(w["theta"]).cuda()
    p = torch.from_numpy(w["p"]).cuda()
    h = torch.from_numpy(w["H"]).cuda().requires_grad_(True)
    F = L.UnravelCost.function()
    cost = F.apply(h, th, p)
    cost.sum().backward()
    _, grad, _ = L.unravel_grad(th, p, h.detach())
    assert torch.allclose(h.grad, grad)


# --- Lindbladian front end ----------------------------------------------------------

def test_lindblad_circuit_matches_oracle(L):
    """A Trotterized Heisenberg chain with decay (Lindbladian front end) runs
    through the library: per trajectory equal to the oracle's dense trajectory
    of the same circuit (FP64, no truncation)."""
    from paper_2508_05745_gb300 import lindblad as LB
    circ = LB.heisenberg_amplitude_damping(6, 0.3, 0.1, 4)
    sim, res, br = run_gpu(L, circ, 8, 8, seed=2)
    sim.destroy()
    for t in range(8):
        ref = T.dense_trajectory(circ, t, 2)
        assert list(br[t]) == ref.branch
        assert np.allclose(res["z"][t], ref.z, atol=1e-10)
        assert abs(res["s_half"][t] - ref.s_half) < 1e-10


# --- canonical form after truncation -------------------------------------------------

@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-13)])
def test_canonical_form_after_truncation(L, precision, tol):
    """After truncating layers at chi=128 (Gram matrices of size 256 through the
    whole eigensolver, QR and LQ centre moves), every site left of the
    orthogonality centre is a left isometry and every site right of it a right
    isometry, to the precision's rounding level.  This checks the orthonormality
    of the kept eigenvectors and of the Q factors directly, not through
    observables."""
    circ = I.random_brickwork(16, 16, I.depolarizing_kraus(1.0), 5, coin_p=0.005)
    sim = L.Simulation(16, 128, 8, seed=5, precision=precision, cutoff=1e-12 if precision == "mixed" else 1e-20)
    sim.run(circ)
    assert sim.measure()["n_failed"] == 0
    for t in (0, 3, 7):
        tensors, bonds = sim.export_mps(t)
        assert bonds.max() == 128
        left = [np.abs(np.einsum('asb,asc->bc', a.conj(), a) - np.eye(a.shape[2])).max() for a in tensors]
        right = [np.abs(np.einsum('asb,csb->ac', a, a.conj()) - np.eye(a.shape[0])).max() for a in tensors]
        n = len(tensors)
        centres = [c for c in range(n)
                   if all(left[k] < tol for k in range(c)) and all(right[k] < tol for k in range(c + 1, n))]
        assert centres, (precision, t, np.max(left), np.max(right))
    sim.destroy()


def test_mixed_eigenvector_back_transform_precisions_agree(L):
    """Mixed mode at chi=128 (Gram matrices of size 256) with the kept
    eigenvectors back-transformed in complex64 (default) and in FP64: the same
    branch sequences, and observables that differ by far less than the mixed
    tolerance (the back-transformation adds about n eps_32 to vectors that the
    split rounds to complex64 in either case)."""
    circ = I.random_brickwork(16, 16, I.depolarizing_kraus(1.0), 5, coin_p=0.005)
    out = {}
    for vec64 in (False, True):
        sim, res, br = run_gpu(L, circ, 128, 8, seed=5, precision="mixed", cutoff=1e-12, eigvec_fp64=vec64)
        assert res["n_failed"] == 0
        tensors, bonds = sim.export_mps(0)
        assert bonds.max() == 128
        sim.destroy()
        out[vec64] = (res, br)
    (ra, ba), (rb, bb) = out[False], out[True]
    assert np.array_equal(ba, bb)
    d = max(np.abs(ra["z"] - rb["z"]).max(), np.abs(ra["zz"] - rb["zz"]).max(), np.abs(ra["s_half"] - rb["s_half"]).max())
    print(f"complex64 vs FP64 back-transformation: max observable difference {d:.2e}")
    assert d < 1e-5


# --- the chi=128 benchmark configuration, sampled -------------------------------------

def _oracle_mps_job(args):
    circ, t, seed, chi, cutoff = args
    r = T.mps_trajectory(circ, t, seed, chi_max=chi, cutoff=cutoff)
    return r.branch, r.z, r.zz, r.s_half, r.eps_bound


def oracle_mps_many(circ, trajs, seed, chi, cutoff):
    """The oracle's FP64 MPS trajectories, one process per trajectory (a
    spawn pool: safe after CUDA initialisation in this process)."""
    jobs = [(circ, int(t), seed, chi, cutoff) for t in trajs]
    ctx = multiprocessing.get_context("spawn")
    # one BLAS thread per worker (set before the children import numpy)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with concurrent.futures.ProcessPoolExecutor(min(len(jobs), os.cpu_count() or 1), mp_context=ctx) as ex:
            return list(ex.map(_oracle_mps_job, jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.slow
def test_chi128_workload_sampled_against_oracle(L):
    """The chi=128 benchmark configuration, checked on sampled trajectories.

    The circuit is the n=48 one of the uneven workload (depth-32 Haar brickwork,
    two-qubit depolarizing p=0.005), cut to 14 layers so that the middle bonds
    sit at chi=128 in the later layers.  Mixed precision runs in one handle of
    608 trajectories, the bench's per-size scale of one CTA per trajectory and
    kernel; FP64 runs in a handle of 2.  Sixteen mixed and two FP64
    trajectories are recomputed by the oracle's FP64 MPS trajectory:
    - FP64: equal branch sequences, observables to 1e-10, error bound to
      1e-10 relative (see bound_tol).
    - Mixed: equal branch sequences on all sixteen, observables within 1e-4."""
    w = I.workload_uneven(seed=0, n_traj=8, depth=32)
    full = w["circuits"][48]
    circ = I.Circuit(full.n_qubits, full.layers[:14])
    seed = 11
    sim, res, br = run_gpu(L, circ, 128, 608, seed=seed, precision="mixed", cutoff=1e-12)
    _, bonds = sim.export_mps(0)
    sim.destroy()
    assert bonds.max() == 128 and res["n_failed"] == 0
    refs = oracle_mps_many(circ, range(16), seed, 128, 1e-12)
    worst = 0.0
    for t, (branch, z, zz, s_half, _) in enumerate(refs):
        assert list(br[t]) == branch, t
        worst = max(worst, np.abs(res["z"][t] - z).max(), np.abs(res["zz"][t] - zz).max(), abs(res["s_half"][t] - s_half))
        assert close(res["z"][t], z, 1e-4), t
        assert close(res["zz"][t], zz, 1e-4), t
        assert close(res["s_half"][t], s_half, 1e-4), t
    print(f"mixed chi=128: max observable error over 16 trajectories {worst:.3e}")
    sim, res, br = run_gpu(L, circ, 128, 2, seed=seed, precision="fp64", cutoff=1e-20)
    sim.destroy()
    refs = oracle_mps_many(circ, range(2), seed, 128, 1e-20)
    for t, (branch, z, zz, s_half, eps_bound) in enumerate(refs):
        assert list(br[t]) == branch
        assert close(res["z"][t], z, 1e-10), (t, np.abs(res["z"][t] - z).max())
        assert close(res["zz"][t], zz, 1e-10), (t, np.abs(res["zz"][t] - zz).max())
        assert close(res["s_half"][t], s_half, 1e-10), (t, res["s_half"][t] - s_half)
        assert abs(res["eps_bound"][t] - eps_bound) <= bound_tol(eps_bound, "fp64"), (t, res["eps_bound"][t], eps_bound)


# --- mixed precision against FP64: trajectory averages ---------------------------------

def _mean_z_scores(rm, rd):
    """(mean_mixed - mean_FP64) / sqrt(se_mixed^2 + se_FP64^2) for every
    observable (<Z_i>, <Z_i Z_i+1>, S(n/2)); zero where both errors vanish."""
    zs = []
    for km, ks in (("z_mean", "z_stderr"), ("zz_mean", "zz_stderr")):
        se = np.sqrt(rm[ks] ** 2 + rd[ks] ** 2)
        d = rm[km] - rd[km]
        zs.append(np.where(se > 0, d / np.where(se > 0, se, 1.0), np.where(d == 0, 0.0, np.inf)))
    se = math.hypot(rm["s_half_stderr"], rd["s_half_stderr"])
    d = rm["s_half_mean"] - rd["s_half_mean"]
    zs.append(np.array([d / se if se > 0 else (0.0 if d == 0 else np.inf)]))
    return np.concatenate(zs)


@pytest.mark.slow
@pytest.mark.parametrize("config", ["chi64_ad_dephasing", "chi128_depolarizing"])
def test_mixed_and_fp64_means_agree_within_3_se(L, config):
    """Trajectory-averaged observables of the mixed path agree with those of
    the FP64 path within 3 combined standard errors, over 256 trajectories:
    the chi=64 AD-then-dephasing workload (n=32, depth 20) and the chi=128
    two-qubit depolarizing workload (its n=48 circuit, 12 layers, so that the
    middle bonds reach chi=128)."""
    if config == "chi64_ad_dephasing":
        circ, chi = I.workload_ad_dephasing(seed=0, n_traj=256)["circuit"], 64
    else:
        full = I.workload_uneven(seed=0, n_traj=8, depth=32)["circuits"][48]
        circ, chi = I.Circuit(full.n_qubits, full.layers[:12]), 128
    out = {}
    for precision, cutoff in (("mixed", 1e-12), ("fp64", 1e-20)):
        sim = L.Simulation(circ.n_qubits, chi, 256, seed=21, precision=precision, cutoff=cutoff)
        sim.run(circ)
        out[precision] = sim.measure()
        _, bonds = sim.export_mps(0)
        sim.destroy()
        assert out[precision]["n_failed"] == 0
    assert bonds.max() == chi
    z = _mean_z_scores(out["mixed"], out["fp64"])
    print(f"{config}: |z| max {np.abs(z).max():.3e}, median {np.median(np.abs(z)):.3e} over {z.size} observables")
    assert np.all(np.abs(z) < 3.0), z


# --- bond dimensions above 128 (chi_max up to 512) --------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_global_memory_kernels_match_oracle(L, precision):
    """The global-memory eigensolver and QR centre move, which run where a site
    capacity exceeds 128, forced at every size (big_kernels = 1) on the
    truncated chi = 4 run of test_truncated_run_matches_oracle_mps: the same
    branch sequences and the same bars (FP64 1e-10, mixed mixed_tol)."""
    circ = I.random_brickwork(10, 10, I.depolarizing_kraus(0.05), seed=4)
    n_traj = 16
    sim, res, br = run_gpu(L, circ, 4, n_traj, seed=3, precision=precision, cutoff=1e-14, big_kernels=True)
    sim.destroy()
    for t in range(n_traj):
        ref = T.mps_trajectory(circ, t, 3, chi_max=4, cutoff=1e-14)
        assert list(br[t]) == ref.branch, t
        tol = 1e-10 if precision == "fp64" else mixed_tol(ref)
        assert close(res["z"][t], ref.z, tol), t
        assert close(res["zz"][t], ref.zz, tol), t
        assert close(res["s_half"][t], ref.s_half, tol), t
        assert abs(res["eps_bound"][t] - ref.eps_bound) <= bound_tol(ref.eps_bound, precision), t


@pytest.mark.slow
def test_global_memory_kernels_at_chi128(L):
    """The global-memory kernels forced on the chi = 128 benchmark circuit (the
    n = 48 circuit of the uneven workload, 14 layers, Gram matrices of 256):
    two FP64 trajectories to 1e-10 and eight mixed ones to 1e-4 against the
    oracle's FP64 MPS trajectories, as the on-chip kernels are held in
    test_chi128_workload_sampled_against_oracle."""
    w = I.workload_uneven(seed=0, n_traj=8, depth=32)
    full = w["circuits"][48]
    circ = I.Circuit(full.n_qubits, full.layers[:14])
    seed = 11
    for precision, cutoff, n_traj, tol in (("fp64", 1e-20, 2, 1e-10), ("mixed", 1e-12, 8, 1e-4)):
        sim, res, br = run_gpu(L, circ, 128, n_traj, seed=seed, precision=precision, cutoff=cutoff,
                               big_kernels=True)
        _, bonds = sim.export_mps(0)
        sim.destroy()
        assert bonds.max() == 128 and res["n_failed"] == 0
        refs = oracle_mps_many(circ, range(n_traj), seed, 128, cutoff)
        for t, (branch, z, zz, s_half, eps_bound) in enumerate(refs):
            assert list(br[t]) == branch, (precision, t)
            assert close(res["z"][t], z, tol), (precision, t, np.abs(res["z"][t] - z).max())
            assert close(res["zz"][t], zz, tol), (precision, t)
            assert close(res["s_half"][t], s_half, tol), (precision, t)
            assert abs(res["eps_bound"][t] - eps_bound) <= bound_tol(eps_bound, precision), (precision, t)


def _oracle_gap_job(args):
    circ, t, seed, chi, cutoff = args
    r = T.mps_trajectory(circ, t, seed, chi_max=chi, cutoff=cutoff)
    return r.branch, r.z, r.zz, r.s_half, r.eps_bound, dict(r.gram_bound)


def oracle_jobs(jobs):
    """Oracle MPS trajectories for (circ, t, seed, chi, cutoff) jobs in a spawn
    pool, the host's BLAS threads shared out among the jobs."""
    ctx = multiprocessing.get_context("spawn")
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: str(max(1, (os.cpu_count() or 1) // len(jobs))) for k in keys})
    try:
        with concurrent.futures.ProcessPoolExecutor(min(len(jobs), os.cpu_count() or 1), mp_context=ctx) as ex:
            return list(ex.map(_oracle_gap_job, jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def entropy_tol(b, d):
    """Fannes-Audenaert: reduced states of pure states at distance <= b are
    within trace distance T = min(1, b), so their entropies differ by at most
    T ln(d - 1) + h(T) (d = Schmidt rank bound)."""
    tt = min(1.0, b)
    h = 0.0 if tt in (0.0, 1.0) else -tt * math.log(tt) - (1 - tt) * math.log(1 - tt)
    return tt * math.log(max(d - 1, 1)) + h


LARGE_CHI_CASES = {
    # Haar brickwork whose middle bonds reach 512: Gram matrices up to 1024
    "haar_n20_chi512": (lambda: I.random_brickwork(20, 12, I.depolarizing_kraus(0.01), seed=3), 512),
    # the kicked-Ising family (RZZ(pi/4 + noise), RX kicks, two-qubit
    # depolarizing p = 0.01) at n = 20, 22 periods: bonds truncated at 256
    "kicked_ising_n20_chi256": (lambda: I.kicked_ising(20, 22, I.depolarizing_kraus(1.0), 0.01, seed=2), 256),
}


@pytest.mark.slow
@pytest.mark.parametrize("case", list(LARGE_CHI_CASES))
def test_large_bond_dimensions_against_oracle(L, case):
    """chi_max above 128 (the global-memory eigensolver with Gram matrices up to
    1024 and the global-memory QR): two trajectories per precision against the
    oracle's FP64 MPS trajectories with the same cutoff.  Identical branch
    sequences.  FP64: observables within the worst-case change of a split
    computed from the Gram matrix instead of by SVD, summed over the splits
    (the oracle's gram_bound for unit roundoff 2^-53: unresolved kept weight
    and Davis-Kahan at the cut): 2 b for <Z>, <ZZ> and the error bound, the
    Fannes-Audenaert bound for S(n/2), never below 1e-10.  Mixed: the same
    bound for 2^-24 exceeds 1 here, so the observables are held to the mixed
    target of 1e-4 per trajectory (the error bound to the Gram-route bound).
    The FP64 bounds are loose (the errors printed are far below them); the
    global-memory kernels are held to the strict bars in
    test_global_memory_kernels_match_oracle and _at_chi128."""
    make, chi = LARGE_CHI_CASES[case]
    circ = make()
    seed = 5
    cuts = {"fp64": 1e-20, "mixed": 1e-12}
    units = {"fp64": 2.0 ** -53, "mixed": 2.0 ** -24}
    floors = {"fp64": 1e-10, "mixed": 1e-4}
    jobs = [(circ, t, seed, chi, cuts[p]) for p in ("fp64", "mixed") for t in range(2)]
    refs = oracle_jobs(jobs)
    refs = {"fp64": refs[:2], "mixed": refs[2:]}
    out = {}
    for precision in ("fp64", "mixed"):
        sim, res, br = run_gpu(L, circ, chi, 2, seed=seed, precision=precision, cutoff=cuts[precision])
        _, bonds = sim.export_mps(0)
        sim.destroy()
        assert res["n_failed"] == 0
        assert bonds.max() > 128, bonds
        for t, (branch, z, zz, s_half, eps_bound, gb) in enumerate(refs[precision]):
            assert list(br[t]) == branch, (precision, t)
            b = gb[units[precision]]
            if precision == "fp64":
                tol_o = max(floors[precision], 2 * b)
                tol_s = max(floors[precision], entropy_tol(b, chi))
            else:
                tol_o = tol_s = 1e-4
            err = max(np.abs(res["z"][t] - z).max(), np.abs(res["zz"][t] - zz).max())
            assert err <= tol_o, (precision, t, err, tol_o)
            assert abs(res["s_half"][t] - s_half) <= tol_s, (precision, t, res["s_half"][t] - s_half, tol_s)
            assert abs(res["eps_bound"][t] - eps_bound) <= max(bound_tol(eps_bound, precision), 2 * b)
            print(f"{case} {precision} traj {t}: max bond {bonds.max()}, <Z>/<ZZ> error {err:.2e} (bound {tol_o:.1e}), "
                  f"S error {abs(res['s_half'][t] - s_half):.2e} (bound {tol_s:.1e})")
        out[precision] = res
    mid = circ.n_qubits // 2
    for p in ("mixed", "fp64"):
        print(f"{case} {p}: <Z_{mid}> {out[p]['z'][:, mid]}, S(n/2) {out[p]['s_half']}")
