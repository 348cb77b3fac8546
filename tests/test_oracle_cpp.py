"""The C++17 FP64 oracle (oracle/mps_oracle.cpp) pinned against the Python
oracle and against what the method fixes: the counter-based generator bit for
bit, the optimal Kraus sets to rounding, trajectories without truncation
equal to the dense state-vector trajectory (an independent path: no MPS,
no SVD), truncated MPS trajectories equal to the Python MPS oracle, and the
trajectory average equal to exact density-matrix evolution within 3 standard
errors.  CPU only."""
import numpy as np
import pytest

from oracle import cpp, philox
from oracle import trajectories as T
from oracle import unravel as U
from paper_2508_05745_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def built():
    cpp.build()


def test_uniform_equals_the_python_generator():
    for seed in (0, 7, 2 ** 63 + 5):
        for t, g, s in [(0, 0, 0), (3, 11, 1), (12345, 999, 2), (2 ** 40, 2 ** 33, 1)]:
            assert cpp.uniform(seed, t, g, s) == philox.uniform(seed, t, g, s)


CHANNELS = [I.depolarizing_kraus(0.05), I.depolarizing_kraus(1.0), I.amplitude_damping_kraus(0.2),
            I.compose_kraus(I.dephasing_kraus(0.1), I.amplitude_damping_kraus(0.3)),
            I.projective_depolarizing_kraus(0.2)]


@pytest.mark.parametrize("ci", range(len(CHANNELS)))
def test_optimal_unraveling_equals_the_python_oracle(ci):
    kr = CHANNELS[ci]
    rng = np.random.default_rng(ci)
    states = [0.5 * np.eye(2, dtype=np.complex128), np.diag([1.0, 0.0]).astype(np.complex128),
              np.diag([0.7, 0.3]).astype(np.complex128)]
    for _ in range(60):
        a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        states.append(a @ a.conj().T)
    for rho in states:
        kp, wp = U.optimal_unraveling(rho, kr)
        kc, wc = cpp.optimal_unraveling(rho, kr)
        assert np.abs(kp - kc).max() < 1e-11
        # the remix is unitary (Eq. unitarity_kraus) and keeps the channel
        assert np.allclose(wc.conj().T @ wc, np.eye(wc.shape[0]), atol=1e-12)
        assert np.allclose(sum(k.conj().T @ k for k in kc), np.eye(2), atol=1e-12)


def _compare(circ, chi, cutoff, n_traj, seed, mode="optimal", layering="local", dense=False, tol=1e-12):
    r = cpp.mps_trajectories(circ, 0, n_traj, seed, chi, cutoff, mode, layering)
    for t in range(n_traj):
        ref = (T.dense_trajectory(circ, t, seed, mode) if dense
               else T.mps_trajectory(circ, t, seed, chi, cutoff, mode, layering=layering))
        assert list(r["branch"][t]) == list(ref.branch), t
        assert np.abs(r["z"][t] - ref.z).max() < tol
        assert np.abs(r["zz"][t] - ref.zz).max() < tol
        assert abs(r["s_half"][t] - ref.s_half) < tol
        if not dense:
            assert abs(r["eps_bound"][t] - ref.eps_bound) < max(tol, 1e-9 * ref.eps_bound)


def test_untruncated_trajectories_equal_dense_state_vector():
    _compare(I.random_brickwork(8, 8, I.depolarizing_kraus(0.05), seed=1), 16, 1e-20, 12, 3, dense=True)


def test_untruncated_coin_noise_equals_dense_state_vector():
    _compare(I.random_brickwork(10, 6, I.depolarizing_kraus(0.1), seed=2, coin_p=0.5), 32, 1e-20, 8, 5, dense=True)


def test_truncated_trajectories_equal_python_mps_oracle():
    circ = I.random_brickwork(10, 10, I.depolarizing_kraus(0.05), seed=4)
    _compare(circ, 4, 1e-14, 12, 3, tol=1e-10)
    # the smallest relative cut gap (the conditioning of the truncations)
    r = cpp.mps_trajectories(circ, 0, 12, 3, 4, 1e-14)
    for t in range(12):
        gaps = T.mps_trajectory(circ, t, 3, 4, 1e-14).cut_gaps
        assert abs(r["min_gap"][t] - (min(gaps) if gaps else 1.0)) < 1e-9


@pytest.mark.parametrize("mode,layering", [("given", "local"), ("haar_optimal", "local"), ("optimal", "global")])
def test_modes_and_layering_equal_python_mps_oracle(mode, layering):
    _compare(I.random_brickwork(10, 8, I.depolarizing_kraus(0.05), seed=4), 8, 1e-14, 6, 3, mode, layering,
             tol=1e-10)


def test_trajectory_average_matches_density_matrix_evolution():
    """Unravelings average back to the channel: the mean of <Z_i> over
    trajectories equals the exact density-matrix value within 3 s.e."""
    circ = I.random_brickwork(6, 4, I.depolarizing_kraus(0.3), seed=6)
    n_traj = 600
    r = cpp.mps_trajectories(circ, 0, n_traj, 11, 16, 1e-20)
    zr, zzr = T.density_observables(T.density_evolution(circ), 6)
    m, se = r["z"].mean(0), r["z"].std(0, ddof=1) / np.sqrt(n_traj)
    assert np.all(np.abs(m - zr) <= 3 * se + 1e-12), (m, zr, se)
    m2, se2 = r["zz"].mean(0), r["zz"].std(0, ddof=1) / np.sqrt(n_traj)
    assert np.all(np.abs(m2 - zzr) <= 3 * se2 + 1e-12)


def test_layer_chunks_and_thread_counts_give_the_same_run():
    circ = I.random_brickwork(8, 6, I.depolarizing_kraus(0.05), seed=9)
    a = cpp.Batch(circ, 0, 6, 2, 8, 1e-14)
    a.run(0, 2, 1)
    a.run(2, 6, 3)
    ra = a.results()
    with pytest.raises(ValueError):
        a.run(2, 3)          # the batch is at layer 6
    a.close()
    rb = cpp.mps_trajectories(circ, 0, 6, 2, 8, 1e-14, threads=2)
    for k in ("z", "zz", "s_half", "eps_bound", "branch"):
        assert np.array_equal(ra[k], rb[k]), k


def test_trajectory_offset_selects_the_same_streams():
    circ = I.random_brickwork(8, 5, I.depolarizing_kraus(0.05), seed=3)
    full = cpp.mps_trajectories(circ, 0, 8, 4, 8, 1e-14)
    part = cpp.mps_trajectories(circ, 5, 3, 4, 8, 1e-14)
    for k in ("z", "zz", "s_half", "eps_bound", "branch"):
        assert np.array_equal(full[k][5:], part[k]), k


def test_run_range_advances_only_the_selected_trajectories():
    circ = I.random_brickwork(8, 4, I.depolarizing_kraus(0.05), seed=5)
    a = cpp.Batch(circ, 0, 4, 1, 8, 1e-14)
    a.run_range(1, 3, 0, 4, 2)
    with pytest.raises(ValueError):
        a.results()          # trajectories 0 and 3 are still at layer 0
    a.run_range(0, 1, 0, 4)
    a.run_range(3, 4, 0, 4)
    ra = a.results()
    a.close()
    rb = cpp.mps_trajectories(circ, 0, 4, 1, 8, 1e-14)
    for k in ("z", "zz", "s_half", "eps_bound", "branch"):
        assert np.array_equal(ra[k], rb[k]), k
