"""Pins of the Lindbladian front end (appendix on Trotterized Lindbladian
evolutions) against the oracle's exact superoperator evolution and the
appendix's closed forms (CPU only)."""
import math

import numpy as np
import pytest

from oracle import lindblad as OL
from oracle import trajectories as T
from paper_2508_05745_gb300 import inputs as I
from paper_2508_05745_gb300 import lindblad as LB


@pytest.mark.parametrize("gamma,dt", [(0.2, 0.1), (1.3, 0.25), (0.05, 1.0)])
def test_dephasing_jump_is_the_dephasing_channel(gamma, dt):
    """c = |0><0| at rate gamma gives dephasing of rate p = 1 - exp(-gamma dt / 2)
    in the paper's convention (appendix on typical jump operators)."""
    k = LB.jump_kraus([(gamma, LB.PROJ_0)], dt)
    p = 1.0 - math.exp(-gamma * dt / 2)
    assert np.allclose(OL.choi_of_kraus(k), OL.choi_of_kraus(I.dephasing_kraus(p)), atol=1e-13)


@pytest.mark.parametrize("gamma,dt", [(0.2, 0.1), (1.3, 0.25), (0.05, 1.0)])
def test_decay_jump_is_amplitude_damping(gamma, dt):
    """c = |0><1| at rate gamma gives amplitude damping with
    gamma_AD = 1 - exp(-gamma dt); the Kraus set is the Orthogonal one up to
    phases."""
    k = LB.jump_kraus([(gamma, LB.SIGMA_MINUS)], dt)
    g = 1.0 - math.exp(-gamma * dt)
    assert np.allclose(OL.choi_of_kraus(k), OL.choi_of_kraus(I.amplitude_damping_kraus(g)), atol=1e-13)
    assert len(k) == 2


def test_jump_kraus_is_orthogonal_and_exact(rng):
    """A random jump operator pair: the Kraus set reproduces the oracle's
    superoperator exp(L_jump dt) (through the Choi matrix), is trace preserving
    and orthogonal (Tr K_i^dagger K_j = 0 for i != j)."""
    c1 = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    c2 = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    jumps = [(0.4, c1), (0.7, c2)]
    k = LB.jump_kraus(jumps, 0.3)
    import scipy.linalg as sla
    sup = sla.expm(OL.superoperator(np.zeros((2, 2)), jumps) * 0.3)
    assert np.allclose(OL.choi_of_kraus(k), OL.choi_of_superoperator(sup), atol=1e-12)
    assert np.allclose(sum(x.conj().T @ x for x in k), np.eye(2), atol=1e-12)
    gram = np.array([[np.trace(a.conj().T @ b) for b in k] for a in k])
    assert np.allclose(gram - np.diag(np.diag(gram)), 0, atol=1e-12)


def test_bond_terms_sum_to_the_chain_hamiltonian(rng):
    n = 5
    h2 = [rng.standard_normal((4, 4)) for _ in range(n - 1)]
    h1 = [rng.standard_normal((2, 2)) for _ in range(n)]
    hb = LB.bond_hamiltonians(n, h2, h1)
    total = sum(OL.bond_operator(h, i, n) for i, h in enumerate(hb))
    ref = sum(OL.bond_operator(h2[i], i, n) for i in range(n - 1)) + sum(OL.site_operator(h1[i], i, n) for i in range(n))
    assert np.allclose(total, ref)


def test_trotter_circuit_converges_to_the_lindbladian():
    """The circuit's exact density-matrix evolution approaches exp(L t) rho0 at
    first order in dt: halving dt halves the trace-norm error (n = 4,
    Heisenberg chain with decay, t = 0.8)."""
    n, t = 4, 0.8
    h1 = 0.35 * LB.PAULI_X + 0.35 * LB.PAULI_Y + 0.5 * LB.PAULI_Z
    h2 = np.kron(LB.PAULI_Y, LB.PAULI_Y)
    gamma = 0.5
    rho0 = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    rho0[0, 0] = 1.0
    exact = OL.evolve(n, [h2] * (n - 1), [h1] * n, [(s, gamma, LB.SIGMA_MINUS) for s in range(n)], t, rho0)
    errs = []
    for steps in (8, 16, 32):
        c = LB.trotter_circuit(n, h2, h1, [(gamma, LB.SIGMA_MINUS)], t / steps, steps)
        rho = T.density_evolution(c)
        errs.append(np.sum(np.abs(np.linalg.eigvalsh(rho - exact))))
    assert errs[2] < errs[1] < errs[0] < 0.2
    for a, b in zip(errs, errs[1:]):
        assert 0.35 < b / a < 0.65, errs


def test_workload_builders():
    c = LB.heisenberg_amplitude_damping(6, 0.01, 0.1, 3)
    assert len(c.layers) == 6 and c.layers[0].coin_p == 1.0 and c.layers[1].coin_p == 0.0
    for layer in c.layers:
        for g in layer.gates:
            assert np.allclose(g.conj().T @ g, np.eye(4))
    r = LB.random_lindbladian(6, 3)
    assert np.allclose(sum(k.conj().T @ k for k in r.layers[0].kraus), np.eye(2))
    with pytest.raises(ValueError):
        LB.trotter_circuit(5, np.eye(4), np.eye(2), [(0.1, LB.SIGMA_MINUS)], 0.1, 1)
